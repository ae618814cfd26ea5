// Learned preconditioner for the pressure correction: a 3-level U-Net whose
// 3x3x3 convolutions run on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in tensor memory).  The paper has no learned component; this
// is the build's own solver aid for the pressure system of Eq. contDBS.
//
// Tensors are channels-last BF16: element (voxel v, channel c) at v * C + c,
// voxel v = i + nx (j + ny k).  Channel counts are multiples of 8, so the 8
// channels of one tap are one 16-byte vector.
//
// Convolution as an implicit GEMM: D[v, o] = sum_K A[v, K] B[o, K] with
// K = tap * C_in + i (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)), A the gathered
// neighbourhood (zero outside the box) and B the weights [C_out][27][C_in].
// One CTA of 128 threads owns 128 consecutive voxels (the MMA's M); K runs
// in stages of 64 (four K = 16 MMAs), double buffered: all threads gather
// the next stage into shared memory while the tensor core works on the
// current one.  The FP32 accumulator (128 lanes x C_out columns) lives in
// tensor memory and is read back once, with bias and ReLU fused.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/vos.h"
#include "vos_internal.cuh"
#include "vos_tc.cuh"

namespace vos {
void set_global_error(const char* msg);

static __device__ unsigned long long vos_exec_count = 0;
unsigned long long exec_count_unet() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}

// Set by a tensor-core kernel whose mbarrier wait ran out of time.
static __device__ int g_tc_timeout = 0;

namespace unet {

constexpr int kTM = 128;                    // voxels per CTA (MMA M)
constexpr int kStageK = 64;                 // K elements per stage
constexpr int kStageA = kTM * kStageK * 2;  // bytes of one A stage (16 KB)
constexpr uint64_t kWaitNs = 2000000000ull; // 2 s per mbarrier wait

struct ConvArgs {
  const __nv_bfloat16* x;  // [V][cin]
  const __nv_bfloat16* w;  // [cout][27 * cin]
  const float* bias;       // [cout] or null
  float* yf;               // [V][cout] FP32 output or null
  __nv_bfloat16* yb;       // [V][cout] BF16 output or null
  int nx, ny, nz, cin, cout, relu;
  long long V;
};

__host__ __device__ inline int tmem_cols(int cout) {
  return cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256));
}
inline size_t conv_smem_bytes(int cout) { return 2 * (size_t)kStageA + 2 * (size_t)cout * 128 + 64; }

// Byte offset of (row, K-group g) in a stage: 8-row groups 1024 B apart
// (SBO), K groups of 8 elements 128 B apart (LBO), 16 B per row.
__device__ __forceinline__ uint32_t stage_off(int row, int g) {
  return (uint32_t)((row >> 3) * 1024 + g * 128 + (row & 7) * 16);
}

__global__ void __launch_bounds__(kTM) k_conv3d_tc(ConvArgs a) {
  VOS_COUNT_EXEC();
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int bstage = a.cout * 128;
  unsigned char* sA = smem;
  unsigned char* sB = smem + 2 * kStageA;
  uint64_t* mbar = (uint64_t*)(sB + 2 * bstage);
  uint32_t* slot = (uint32_t*)(mbar + 2);
  const uint32_t ncols = (uint32_t)tmem_cols(a.cout);

  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(&mbar[0]), 1);
    tc::mbar_init(tc::smem_addr(&mbar[1]), 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;

  const long long v = (long long)blockIdx.x * kTM + tid;
  const bool vin = v < a.V;
  const long long plane = (long long)a.nx * a.ny;
  const int vk = vin ? (int)(v / plane) : 0;
  const int vj = vin ? (int)((v - (long long)vk * plane) / a.nx) : 0;
  const int vi = vin ? (int)(v - (long long)vk * plane - (long long)vj * a.nx) : 0;
  const int cg = a.cin >> 3;       // channel groups per tap
  const int G = 27 * cg;           // K groups in total
  const int K = 27 * a.cin;
  const int nst = (G + 7) >> 3;    // stages
  const uint32_t idesc = tc::idesc_bf16_f32(kTM, a.cout);
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;

  for (int c = 0; c < nst; ++c) {
    const int s = c & 1;
    bool okw = true;
    if (c >= 2) {  // the MMAs of stage c - 2 must be done reading buffer s
      okw = tc::mbar_wait(tc::smem_addr(&mbar[s]), phase[s], kWaitNs);
      phase[s] ^= 1u;
    }
    unsigned char* A = sA + s * kStageA;
    unsigned char* B = sB + s * bstage;
#pragma unroll 2
    for (int g = 0; g < 8; ++g) {
      const int gg = c * 8 + g;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (vin && gg < G) {
        const int tap = gg / cg, ch = (gg - tap * cg) * 8;
        const int ii = vi + (tap % 3) - 1, jj = vj + (tap / 3) % 3 - 1, kk = vk + tap / 9 - 1;
        if (ii >= 0 && ii < a.nx && jj >= 0 && jj < a.ny && kk >= 0 && kk < a.nz)
          val = __ldg((const uint4*)(a.x + ((long long)kk * plane + (long long)jj * a.nx + ii) * a.cin + ch));
      }
      *(uint4*)(A + stage_off(tid, g)) = val;
    }
    for (int it = tid; it < a.cout * 8; it += kTM) {
      const int n = it >> 3, g = it & 7, gg = c * 8 + g;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (gg < G) val = __ldg((const uint4*)(a.w + (long long)n * K + gg * 8));
      *(uint4*)(B + stage_off(n, g)) = val;
    }
    tc::fence_proxy_async_smem();
    if (!__syncthreads_and(okw ? 1 : 0)) {  // block-uniform: a wait ran out of time
      ok = false;
      break;
    }
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ad = tc::desc_kmajor(a0 + ks * 256, 128, 1024);
        const uint64_t bd = tc::desc_kmajor(b0 + ks * 256, 128, 1024);
        tc::mma_bf16(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
      }
      tc::commit(tc::smem_addr(&mbar[s]));
    }
  }
  // Wait for the last stage's MMAs (a commit tracks all earlier MMAs of the
  // issuing thread) and for the other buffer's outstanding arrival.
  if (ok) {
    const int sl = (nst - 1) & 1;
    ok = tc::mbar_wait(tc::smem_addr(&mbar[sl]), phase[sl], kWaitNs);
    if (ok && nst >= 2) ok = tc::mbar_wait(tc::smem_addr(&mbar[sl ^ 1]), phase[sl ^ 1], kWaitNs);
  }
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(&g_tc_timeout, 1);
  } else {
    tc::fence_after_sync();
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int n0 = 0; n0 < a.cout; n0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(trow + (uint32_t)n0, r);
      if (vin) {
        float f[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float y = __uint_as_float(r[q]) + (a.bias ? __ldg(a.bias + n0 + q) : 0.0f);
          f[q] = (a.relu && y < 0.0f) ? 0.0f : y;
        }
        if (a.yf) {
          float4* dst = (float4*)(a.yf + v * a.cout + n0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        }
        if (a.yb) {
          __align__(16) __nv_bfloat162 h[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) h[q] = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
          uint4* dst = (uint4*)(a.yb + v * a.cout + n0);
          dst[0] = *(const uint4*)&h[0];
          dst[1] = *(const uint4*)&h[4];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// Host launcher: y = conv3(x, w) (+ bias, ReLU).  Returns a CUDA error.
cudaError_t conv3d(const ConvArgs& a, cudaStream_t st) {
  static bool attr_done = false;
  const size_t sm = conv_smem_bytes(256);
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const long long nb = (a.V + kTM - 1) / kTM;
  if (nb <= 0) return cudaSuccess;
  const double flops = 2.0 * 27.0 * a.cin * a.cout * (double)a.V;
  vlaunch_smem("unet_conv", flops, k_conv3d_tc, dim3((unsigned)nb), dim3(kTM), conv_smem_bytes(a.cout), st, a);
  return cudaGetLastError();
}

bool conv_shape_ok(int cin, int cout) {
  return cin >= 8 && cin % 8 == 0 && cout >= 16 && cout <= 256 && cout % 16 == 0;
}

int take_timeout_flag() {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int));
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(int));
  }
  return v;
}

}  // namespace unet
}  // namespace vos

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace vos;

extern "C" {

int vos_conv3d_bf16(const uint16_t* x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const uint16_t* w,
                    const float* bias, int32_t cout, int32_t relu, float* y_f32, uint16_t* y_bf16, void* stream) {
  if (!x || !w || (!y_f32 && !y_bf16) || nx < 1 || ny < 1 || nz < 1 || !unet::conv_shape_ok(cin, cout)) {
    set_global_error("vos_conv3d_bf16: bad argument (cin a multiple of 8, cout a multiple of 16 in [16, 256])");
    return VOS_EINVAL;
  }
  unet::ConvArgs a;
  a.x = (const __nv_bfloat16*)x;
  a.w = (const __nv_bfloat16*)w;
  a.bias = bias;
  a.yf = y_f32;
  a.yb = (__nv_bfloat16*)y_bf16;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.cin = cin;
  a.cout = cout;
  a.relu = relu ? 1 : 0;
  a.V = (long long)nx * ny * nz;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = unet::conv3d(a, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  if (unet::take_timeout_flag()) {
    set_global_error("vos_conv3d_bf16: a tensor-core wait ran out of time");
    return VOS_ETIMEOUT;
  }
  return VOS_OK;
}

}  // extern "C"
