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
// K = (tap, input channel) (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)), A the
// neighbourhood of v (zero outside the box) and B the weights
// [C_out][27][C_in].  The A operand is never materialised: the MMA
// descriptors point into an input tile in shared memory (see k_conv3d_tc).
// The FP32 accumulator (128 lanes x C_out columns) lives in tensor memory
// and is read back once, with bias and ReLU fused.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
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

constexpr int kTM = 128;                     // output voxels per CTA (MMA M)
constexpr int kTX = 8, kTY = 16;             // output tile: 8 (x) x 16 (y) x 1 (z)
constexpr int kHX = kTX + 2, kHY = kTY + 2;  // input tile with a one-voxel halo
constexpr int kHalo = kHX * kHY * 3;         // 540 voxels
constexpr int kBoxBytes = kHalo * 16;        // one 8-channel group of the tile (8640 B)
constexpr int kPlaneA = 8704;                // the same, padded to a multiple of 128 B (TMA)
constexpr int kStageA = 2 * kPlaneA;         // 16 input channels per stage
constexpr int kBulkChunk = 16384;            // bytes per bulk copy of the weights
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per mbarrier wait

struct ConvArgs {
  const __nv_bfloat16* x;    // [V][cin] (described to the kernel by a TMA tensor map)
  const __nv_bfloat16* img;  // weights in the shared-memory image layout (see conv_image)
  const float* bias;         // [cout] or null
  float* yf;                 // [V][cout] FP32 output or null
  __nv_bfloat16* yb;         // [V][cout] BF16 output or null
  int nx, ny, nz, cin, cout, relu;
  long long V;
};

__host__ __device__ inline int tmem_cols(int cout) {
  return cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256));
}
__host__ __device__ inline int stage_b_bytes(int cout) { return 27 * cout * 32; }
// Stages of 16 input channels, and the buffers they cycle through (one
// buffer when there is one stage: half the shared memory, twice the CTAs).
__host__ __device__ inline int conv_stages(int cin) { return ((cin >> 3) + 1) >> 1; }
__host__ __device__ inline int conv_buffers(int cin) { return conv_stages(cin) >= 2 ? 2 : 1; }
inline size_t conv_smem_bytes(int cin, int cout) {
  return (size_t)conv_buffers(cin) * ((size_t)kStageA + stage_b_bytes(cout)) + 64;
}
// Elements of a conv's weight image: stages x 27 taps x cout x 16 channels.
__host__ __device__ inline long long conv_image_elems(int cin, int cout) { return (long long)conv_stages(cin) * 27 * cout * 16; }

// The weight image: the bytes that the B operand of stage s needs in shared
// memory, stored contiguously so that one bulk copy brings a whole stage.
// Element (output n, tap t, input channel c) sits in stage s = c / 16 at
// byte t*cout*32 + (n/8)*256 + kg*128 + (n%8)*16 + (c%8)*2 with
// kg = (c%16)/8: per tap an N x 16 K-major operand in the no-swizzle
// canonical layout (8-row groups 256 B apart, the two K core matrices
// 128 B apart).  Channels >= cin are zero.
__device__ __forceinline__ void image_decode(long long e, int cout, int& n, int& t, int& c) {
  const int j = (int)(e & 7);
  const int nr = (int)((e >> 3) & 7);
  const int kg = (int)((e >> 6) & 1);
  const long long q = e >> 7;  // (s * 27 + t) * (cout / 8) + n / 8
  const int ng = cout >> 3;
  const int n8 = (int)(q % ng);
  const long long st = q / ng;
  t = (int)(st % 27);
  const int s = (int)(st / 27);
  n = n8 * 8 + nr;
  c = s * 16 + kg * 8 + j;
}

// Image of a forward conv from FP32 weights W[cout][27][cin] (transpose =
// 0), or of its data gradient (transpose = 1: a conv with cin' = cout and
// cout' = cin whose weights are W[c][26 - t][n]).
__global__ void k_image_f32(int wcout, int wcin, int transpose, const float* __restrict__ W,
                            __nv_bfloat16* __restrict__ img) {
  VOS_COUNT_EXEC();
  const int cout = transpose ? wcin : wcout, cin = transpose ? wcout : wcin;
  const long long n_el = conv_image_elems(cin, cout);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (long long)gridDim.x * blockDim.x) {
    int n, t, c;
    image_decode(e, cout, n, t, c);
    float v = 0.0f;
    if (c < cin) v = transpose ? W[((long long)c * 27 + (26 - t)) * wcin + n] : W[((long long)n * 27 + t) * wcin + c];
    img[e] = __float2bfloat16_rn(v);
  }
}
// Image from BF16 weights w[cout][27][cin] (the standalone conv entry point).
__global__ void k_image_bf16(int cout, int cin, const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ img) {
  VOS_COUNT_EXEC();
  const long long n_el = conv_image_elems(cin, cout);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (long long)gridDim.x * blockDim.x) {
    int n, t, c;
    image_decode(e, cout, n, t, c);
    img[e] = (c < cin) ? w[((long long)n * 27 + t) * cin + c] : __float2bfloat16_rn(0.0f);
  }
}

// Implicit-GEMM convolution on the tensor cores.  A CTA owns an 8 x 16 x 1
// output tile (M = 128 rows, row m = (x0 + m % 8, y0 + m / 8)).  K runs
// over stages of 16 input channels.  For a stage, TMA brings the 10 x 18 x 3
// input halo tile of each 8-channel group (two 4-D boxes; out-of-range
// voxels arrive as zeros) into a plane laid out [z][y][x] with 16 bytes per
// voxel, and one bulk copy brings the stage's weight image.  For tap
// (dz, dy, dx) the A operand is the tile itself seen through a descriptor:
// the 8 rows of a core matrix are 8 consecutive x voxels (128 contiguous
// bytes), consecutive 8-row groups are consecutive y rows (SBO = 160 B), the
// two K core matrices are the two channel planes (LBO = 8704 B), and the tap
// shifts the start address.  So a stage costs two TMA boxes, one bulk copy
// and 27 MMAs, with no im2col copy and no loads issued by other threads.
// One thread drives the pipeline: loads of stage c + 1 are in flight while
// the tensor core works on stage c; a buffer is refilled once the commit of
// the MMAs that read it has arrived.  The other threads join for the
// epilogue (TMEM -> registers, bias, ReLU, stores).
__global__ void __launch_bounds__(kTM) k_conv3d_tc(ConvArgs a, const __grid_constant__ CUtensorMap tmx) {
  VOS_COUNT_EXEC();
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int bstage = stage_b_bytes(a.cout);
  const int nbuf = conv_buffers(a.cin);
  unsigned char* sA = smem;
  unsigned char* sB = smem + nbuf * kStageA;
  uint64_t* full = (uint64_t*)(sB + nbuf * bstage);
  uint64_t* empty = full + 2;
  uint32_t* slot = (uint32_t*)(empty + 2);
  int* s_ok = (int*)(slot + 1);
  const uint32_t ncols = (uint32_t)tmem_cols(a.cout);
  const int ncg = a.cin >> 3;          // 8-channel groups of the input
  const int nst = conv_stages(a.cin);  // stages of 16 channels

  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(tc::smem_addr(&full[i]), 1);
      tc::mbar_init(tc::smem_addr(&empty[i]), 1);
    }
    tc::fence_mbar_init();
  }
  if (ncg & 1) {  // an odd channel count leaves the last stage's second plane empty: zero it
    uint4* z = (uint4*)(sA + ((nst - 1) % nbuf) * kStageA + kPlaneA);
    for (int e = tid; e < kPlaneA / 16; e += kTM) z[e] = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_proxy_async_smem();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z;

  if (tid == 0) {
    bool ok = true;
    uint32_t fph[2] = {0u, 0u}, eph[2] = {0u, 0u};
    const uint32_t idesc = tc::idesc_bf16_f32(kTM, a.cout);
    auto issue = [&](int c) {
      const int s = c % nbuf;
      const uint32_t fb = tc::smem_addr(&full[s]);
      const bool two = (2 * c + 1) < ncg;
      tc::mbar_arrive_expect_tx(fb, (uint32_t)((two ? 2 : 1) * kBoxBytes + bstage));
      const uint32_t A = tc::smem_addr(sA + s * kStageA);
      tc::tma_load_4d(A, &tmx, 16 * c, x0 - 1, y0 - 1, z0 - 1, fb);
      if (two) tc::tma_load_4d(A + kPlaneA, &tmx, 16 * c + 8, x0 - 1, y0 - 1, z0 - 1, fb);
      const unsigned char* src = (const unsigned char*)a.img + (size_t)c * bstage;
      const uint32_t B = tc::smem_addr(sB + s * bstage);
      for (int off = 0; off < bstage; off += kBulkChunk) {
        const int n = (bstage - off) < kBulkChunk ? (bstage - off) : kBulkChunk;
        tc::bulk_load(B + off, src + off, (uint32_t)n, fb);
      }
    };
    issue(0);
    if (nst > 1) issue(1);
    for (int c = 0; c < nst && ok; ++c) {
      const int s = c % nbuf;
      ok = tc::mbar_wait(tc::smem_addr(&full[s]), fph[s], kWaitNs);
      fph[s] ^= 1u;
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(sA + s * kStageA), b0 = tc::smem_addr(sB + s * bstage);
      for (int t = 0; t < 27; ++t) {
        const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;  // halo offsets 0..2
        const uint64_t ad = tc::desc_kmajor(a0 + (uint32_t)(((dz * kHY + dy) * kHX + dx) * 16), kPlaneA, kHX * 16);
        const uint64_t bd = tc::desc_kmajor(b0 + (uint32_t)(t * a.cout * 32), 128, 256);
        tc::mma_bf16(tmem, ad, bd, idesc, (c > 0 || t > 0) ? 1u : 0u);
      }
      tc::commit(tc::smem_addr(&empty[s]));
      if (c + nbuf < nst) {  // refill buffer s once the MMAs just issued have read it
        ok = tc::mbar_wait(tc::smem_addr(&empty[s]), eph[s], kWaitNs);
        eph[s] ^= 1u;
        if (ok) issue(c + nbuf);
      }
    }
    // the last commit of each buffer: all MMAs done, no arrival left pending
    for (int s = 0; s < nbuf && ok; ++s)
      if (nst > s) ok = tc::mbar_wait(tc::smem_addr(&empty[(nst - 1 - s) % nbuf]), eph[(nst - 1 - s) % nbuf], kWaitNs);
    *s_ok = ok ? 1 : 0;
    if (!ok) atomicExch(&g_tc_timeout, 1);
  }
  __syncthreads();
  if (*s_ok) {
    tc::fence_after_sync();
    const int m = tid;  // TMEM lane of this thread = output row
    const int ox = x0 + (m & 7), oy = y0 + (m >> 3);
    const bool vin = ox < a.nx && oy < a.ny;
    const long long v = (long long)z0 * ((long long)a.nx * a.ny) + (long long)oy * a.nx + ox;
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

// TMA descriptor of a channels-last BF16 tensor [nz][ny][nx][cin] with
// boxes of 8 channels x 10 x 18 x 3 voxels (the encoder comes from the
// driver through the runtime, so no driver library is linked).
static PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
static cudaError_t make_input_map(CUtensorMap* m, const ConvArgs& a) {
  if (!g_encode_tiled) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&g_encode_tiled, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !g_encode_tiled) {
      g_encode_tiled = nullptr;
      return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
  }
  const cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
  const cuuint64_t strides[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.cin * 2 * a.nx,
                                 (cuuint64_t)a.cin * 2 * a.nx * a.ny};
  const cuuint32_t box[4] = {8, (cuuint32_t)kHX, (cuuint32_t)kHY, 3};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)a.x, dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Host launcher: y = conv3(x, w) (+ bias, ReLU), w given as its image.
cudaError_t conv3d(const ConvArgs& a, cudaStream_t st) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_smem_bytes(96, 96));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (a.V <= 0) return cudaSuccess;
  alignas(64) CUtensorMap tm;
  VOS_CUDA_TRY(make_input_map(&tm, a));
  const dim3 grid((unsigned)((a.nx + kTX - 1) / kTX), (unsigned)((a.ny + kTY - 1) / kTY), (unsigned)a.nz);
  const double flops = 2.0 * 27.0 * a.cin * a.cout * (double)a.V;
  vlaunch_smem("unet_conv", flops, k_conv3d_tc, grid, dim3(kTM), conv_smem_bytes(a.cin, a.cout), st, a, tm);
  return cudaGetLastError();
}

// Build the weight image of a forward (transpose = 0) or data-gradient
// (transpose = 1) conv from FP32 weights.
void conv_image(int wcout, int wcin, int transpose, const float* W, __nv_bfloat16* img, cudaStream_t st) {
  const int cout = transpose ? wcin : wcout, cin = transpose ? wcout : wcin;
  const long long n = conv_image_elems(cin, cout);
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 4096) b = 4096;
  vlaunch("unet_image", 0.0, k_image_f32, (int)b, kThreads, st, wcout, wcin, transpose, W, img);
}

bool conv_shape_ok(int cin, int cout) {
  return cin >= 8 && cin % 8 == 0 && cout >= 16 && cout <= 96 && cout % 16 == 0;
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

namespace vos {
namespace unet {

// ---------------------------------------------------------------------------
// Element-wise and data-movement kernels (CUDA cores).  Flat grid-stride
// loops; every reduction is a fixed-order block / grid sum.
// ---------------------------------------------------------------------------
struct Dims {
  int nx, ny, nz;  // padded network box (multiples of 4)
  int px, py, pz;  // physical box (the pressure unknowns)
};

__device__ __forceinline__ long long phys_index(const Dims& d, long long v, bool& in) {
  const long long plane = (long long)d.nx * d.ny;
  const int k = (int)(v / plane);
  const int j = (int)((v - (long long)k * plane) / d.nx);
  const int i = (int)(v - (long long)k * plane - (long long)j * d.nx);
  in = i < d.px && j < d.py && k < d.pz;
  return i + (long long)d.px * (j + (long long)d.py * k);
}

#define UNET_LOOP(v, n) for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < (n); v += (long long)gridDim.x * blockDim.x)

static int ugrid(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  const long long cap = (long long)g_num_sms * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// inv_rms and rms of a vector from its squared norm (FP64 on one thread).
__global__ void k_rms(const double* rr, double n, float* out) {
  VOS_COUNT_EXEC();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double ms = *rr / n;
    out[0] = ms > 0.0 ? (float)(1.0 / sqrt(ms)) : 0.0f;
    out[1] = ms > 0.0 ? (float)sqrt(ms) : 0.0f;
  }
}

// x0[v] = (r_c * inv_rms, eps_c, 0 x 6) in BF16; zeros in the padding.
template <typename T>
__global__ void k_pack(Dims d, const T* __restrict__ r, const double* __restrict__ eps, const float* scal,
                       __nv_bfloat16* __restrict__ x0) {
  VOS_COUNT_EXEC();
  const long long n = (long long)d.nx * d.ny * d.nz;
  const float inv = scal[0];
  UNET_LOOP(v, n) {
    bool in;
    const long long c = phys_index(d, v, in);
    const float a = in ? (float)r[c] * inv : 0.0f;
    const float e = in ? (float)eps[c] : 0.0f;
    __align__(16) __nv_bfloat162 h[4];
    h[0] = __floats2bfloat162_rn(a, e);
    h[1] = h[2] = h[3] = __floats2bfloat162_rn(0.0f, 0.0f);
    *(uint4*)(x0 + v * 8) = *(const uint4*)h;
  }
}

// 2x2x2 average pooling, C a multiple of 8; coarse box (cx, cy, cz).
__global__ void k_pool(int cx, int cy, int cz, int C, const __nv_bfloat16* __restrict__ f,
                       __nv_bfloat16* __restrict__ c) {
  VOS_COUNT_EXEC();
  const int cg = C >> 3;
  const long long n = (long long)cx * cy * cz * cg;
  const int fx = 2 * cx, fy = 2 * cy;
  UNET_LOOP(t, n) {
    const int g = (int)(t % cg);
    const long long q = t / cg;
    const int i = (int)(q % cx), j = (int)((q / cx) % cy), k = (int)(q / ((long long)cx * cy));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const long long fv = (2 * i + dx) + (long long)fx * ((2 * j + dy) + (long long)fy * (2 * k + dz));
          const uint4 u = *(const uint4*)(f + fv * C + g * 8);
          const __nv_bfloat162* h = (const __nv_bfloat162*)&u;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 p = __bfloat1622float2(h[e]);
            acc[2 * e] += p.x;
            acc[2 * e + 1] += p.y;
          }
        }
    __align__(16) __nv_bfloat162 o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = __floats2bfloat162_rn(acc[2 * e] * 0.125f, acc[2 * e + 1] * 0.125f);
    *(uint4*)(c + q * C + g * 8) = *(const uint4*)o;
  }
}

// out[v] = [coarse[parent(v)] (Cu channels), skip[v] (Cs channels)].
__global__ void k_up_concat(int fx, int fy, int fz, int Cu, int Cs, const __nv_bfloat16* __restrict__ coarse,
                            const __nv_bfloat16* __restrict__ skip, __nv_bfloat16* __restrict__ out) {
  VOS_COUNT_EXEC();
  const int C = Cu + Cs, cg = C >> 3, ug = Cu >> 3;
  const long long n = (long long)fx * fy * fz * cg;
  const int cx = fx / 2, cy = fy / 2;
  UNET_LOOP(t, n) {
    const int g = (int)(t % cg);
    const long long v = t / cg;
    uint4 u;
    if (g < ug) {
      const int i = (int)(v % fx), j = (int)((v / fx) % fy), k = (int)(v / ((long long)fx * fy));
      const long long p = (i / 2) + (long long)cx * ((j / 2) + (long long)cy * (k / 2));
      u = *(const uint4*)(coarse + p * Cu + g * 8);
    } else {
      u = *(const uint4*)(skip + v * Cs + (g - ug) * 8);
    }
    *(uint4*)(out + v * C + g * 8) = u;
  }
}

// z_c = (sum_k w_k d1[v][k] + b) * scale for the physical voxels.
template <typename T>
__global__ void k_head(Dims d, const __nv_bfloat16* __restrict__ d1, const float* __restrict__ head,
                       const float* scal, int use_scale, T* __restrict__ z) {
  VOS_COUNT_EXEC();
  const long long n = (long long)d.px * d.py * d.pz;
  const float sc = use_scale ? scal[1] : 1.0f;
  UNET_LOOP(c, n) {
    const int i = (int)(c % d.px), j = (int)((c / d.px) % d.py), k = (int)(c / ((long long)d.px * d.py));
    const long long v = i + (long long)d.nx * (j + (long long)d.ny * k);
    const uint4* src = (const uint4*)(d1 + v * 16);
    float acc = head[16];
    for (int h2 = 0; h2 < 2; ++h2) {
      const uint4 u = src[h2];
      const __nv_bfloat162* h = (const __nv_bfloat162*)&u;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 p = __bfloat1622float2(h[e]);
        acc += head[h2 * 8 + 2 * e] * p.x + head[h2 * 8 + 2 * e + 1] * p.y;
      }
    }
    z[c] = (T)(acc * sc);
  }
}

// Head backward: g_d1[v][k] = dz_v w_k; grid sums of dz_v d1[v][k] and dz_v.
__global__ void __launch_bounds__(kThreads) k_head_bwd(Dims d, const float* __restrict__ dz,
                                                      const __nv_bfloat16* __restrict__ d1,
                                                      const float* __restrict__ head, float* __restrict__ g,
                                                      float* __restrict__ ghead, RedScratch rs) {
  VOS_COUNT_EXEC();
  const long long n = (long long)d.nx * d.ny * d.nz;
  double acc[17];
#pragma unroll
  for (int q = 0; q < 17; ++q) acc[q] = 0.0;
  UNET_LOOP(v, n) {
    bool in;
    const long long c = phys_index(d, v, in);
    const float dzv = in ? dz[c] : 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float x = __bfloat162float(d1[v * 16 + k]);
      g[v * 16 + k] = dzv * head[k];
      acc[k] += (double)(dzv * x);
    }
    acc[16] += (double)dzv;
  }
  if (grid_sum<17>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
#pragma unroll
    for (int q = 0; q < 17; ++q) ghead[q] = (float)acc[q];
  }
}

// g_pre = g * (out > 0) (FP32) and its BF16 copy.
__global__ void k_relu_bwd(long long n, const float* __restrict__ g, const __nv_bfloat16* __restrict__ out,
                           float* __restrict__ gp, __nv_bfloat16* __restrict__ gp16) {
  VOS_COUNT_EXEC();
  UNET_LOOP(t, n) {
    const float y = __bfloat162float(out[t]);
    const float v = y > 0.0f ? g[t] : 0.0f;
    gp[t] = v;
    gp16[t] = __float2bfloat16_rn(v);
  }
}

// Weight gradient on the tensor cores.  For the rows (j, k) of one chunk and
// the taps t, partial[chunk][t][o][i] = sum_v x[v + t][i] g[v][o] is a GEMM
// D[m][n] = sum_k A[m][k] B[n][k] with rows m = (tap, input channel) stacked
// 128 per MMA tile (27 * cin rows in ceil(27 cin / 128) tiles), n = output
// channel and k = voxel: K = 16 voxels per MMA, BF16 operands (x and the
// BF16 copy of g that the data-gradient convolution also reads), FP32
// accumulators in tensor memory, one N = cout column block per tile.  Both
// operands are MN-major: a core matrix is 8 voxels (rows along K) x 8
// channels (16 bytes along M or N), i.e. 8 channels-last vectors as they lie
// in memory.  So each operand group (tap, 8 input channels) of a stage is one
// TMA box of 8 channels x w voxels along x of the tap's neighbour row,
// with zeros outside the grid from the TMA's own fill: no thread copies
// anything.  A stage is w (16..64) voxels of one row; its groups sit w x 16 B
// apart (the descriptors' M / N stride), the two K halves of an MMA 128 B
// apart, consecutive MMAs of the stage 256 B apart.  One thread drives the
// pipeline (two stage buffers with full / empty mbarriers, as the forward
// convolution); blockIdx.y selects the tiles a CTA accumulates (at most four
// tiles and 256 tensor-memory columns), blockIdx.x its rows.
constexpr int kDwTiles = 4;  // A tiles per CTA at most
struct DwArgs {
  float* partial;  // [nchunk][27][cout][cin]
  int nx, ny, nz, cin, cout;
  int w, segs;     // voxels per stage (box x extent); stages per row
  int rows;        // rows (j, k) per CTA
  int tiles, tpc;  // A tiles in all; tiles per CTA
};
__host__ __device__ inline int dw_tiles(int cin) { return (27 * cin + 127) / 128; }
__host__ __device__ inline int dw_tpc(int cin, int cout) {
  const int t = dw_tiles(cin), cap = 256 / cout < kDwTiles ? 256 / cout : kDwTiles;
  return t < cap ? t : cap;
}
__host__ __device__ inline int dw_width(int nx) { return nx >= 64 ? 64 : (nx >= 32 ? 32 : 16); }
inline size_t dw_stage_bytes(int cin, int cout, int w) {
  return ((size_t)dw_tpc(cin, cout) * 16 + (size_t)(cout / 8)) * (size_t)w * 16;
}
inline size_t dw_smem_bytes(int cin, int cout, int w) { return 2 * dw_stage_bytes(cin, cout, w) + 128; }

// TMA descriptor of a channels-last BF16 tensor [nz][ny][nx][C] with boxes of
// 8 channels x w voxels of one row.
static cudaError_t make_row_map(CUtensorMap* m, const __nv_bfloat16* p, int C, int nx, int ny, int nz, int w) {
  if (!g_encode_tiled) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&g_encode_tiled, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !g_encode_tiled) {
      g_encode_tiled = nullptr;
      return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
  }
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * nx, (cuuint64_t)C * 2 * nx * ny};
  const cuuint32_t box[4] = {8, (cuuint32_t)w, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)p, dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

__global__ void __launch_bounds__(kTM) k_dw_tc(const __grid_constant__ CUtensorMap tmx,
                                              const __grid_constant__ CUtensorMap tmg, DwArgs a) {
  VOS_COUNT_EXEC();
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int T0 = blockIdx.y * a.tpc;
  const int nt = min(a.tpc, a.tiles - T0);
  const int ngA = nt * 16, ngB = a.cout >> 3;
  const int gbytes = a.w * 16;                 // one group's box
  const int sbytes = (a.tpc * 16 + ngB) * gbytes;  // one stage buffer
  unsigned char* buf = smem;
  uint64_t* full = (uint64_t*)(smem + 2 * sbytes);
  uint64_t* empty = full + 2;
  uint32_t* slot = (uint32_t*)(empty + 2);
  int* s_ok = (int*)(slot + 1);
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(nt * a.cout)) ncols <<= 1;
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  // rows of the last tile past 27 taps: zero in both buffers, never loaded
  int nvalid = 0;
  for (int g = 0; g < ngA; ++g)
    if ((T0 * 16 + g) * 8 / a.cin < 27) ++nvalid;
  for (int b = 0; b < 2; ++b)
    for (int g = nvalid; g < ngA; ++g)
      for (int e = tid; e < gbytes / 16; e += kTM)
        reinterpret_cast<uint4*>(buf + b * sbytes + g * gbytes)[e] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async_smem();
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(tc::smem_addr(&full[i]), 1);
      tc::mbar_init(tc::smem_addr(&empty[i]), 1);
    }
    tc::fence_mbar_init();
    *s_ok = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const int nrow = a.ny * a.nz;
  const int r0 = blockIdx.x * a.rows, r1 = min(r0 + a.rows, nrow);
  const int nst = (r1 - r0) * a.segs;  // stages of this CTA
  if (warp == 0) {  // the pipeline: lane 0 waits, issues the MMAs and commits; all lanes issue the TMAs
    const int lane = tid & 31;
    bool ok = true;
    uint32_t fph[2] = {0u, 0u}, eph[2] = {0u, 0u};
    const uint32_t idesc = tc::idesc_bf16_f32_mn(128, a.cout);
    auto issue = [&](int q) {
      const int s = q & 1;
      const int row = r0 + q / a.segs, i0 = (q % a.segs) * a.w;
      const int j = row % a.ny, k = row / a.ny;
      const uint32_t fb = tc::smem_addr(&full[s]);
      if (lane == 0) tc::mbar_arrive_expect_tx(fb, (uint32_t)((nvalid + ngB) * gbytes));
      __syncwarp();
      const uint32_t base = tc::smem_addr(buf + s * sbytes);
      for (int g = lane; g < nvalid; g += 32) {
        const int m = (T0 * 16 + g) * 8, tap = m / a.cin, c0 = m - tap * a.cin;
        tc::tma_load_4d(base + (uint32_t)(g * gbytes), &tmx, c0, i0 + tap % 3 - 1, j + (tap / 3) % 3 - 1,
                        k + tap / 9 - 1, fb);
      }
      const uint32_t bbase = base + (uint32_t)(a.tpc * 16 * gbytes);
      for (int og = lane; og < ngB; og += 32)
        tc::tma_load_4d(bbase + (uint32_t)(og * gbytes), &tmg, og * 8, i0, j, k, fb);
    };
    if (nst > 0) issue(0);
    if (nst > 1) issue(1);
    for (int q = 0; q < nst && ok; ++q) {
      const int s = q & 1;
      if (lane == 0) {
        ok = tc::mbar_wait(tc::smem_addr(&full[s]), fph[s], kWaitNs);
        if (ok) {
          tc::fence_after_sync();
          const uint32_t base = tc::smem_addr(buf + s * sbytes);
          const uint32_t bbase = base + (uint32_t)(a.tpc * 16 * gbytes);
          for (int kk = 0; kk < a.w / 16; ++kk) {  // MMAs of 16 voxels
            const uint64_t bd = tc::desc_mnmajor(bbase + (uint32_t)(kk * 256), (uint32_t)gbytes, 128);
            for (int t = 0; t < nt; ++t) {
              const uint64_t ad =
                  tc::desc_mnmajor(base + (uint32_t)(t * 16 * gbytes + kk * 256), (uint32_t)gbytes, 128);
              tc::mma_bf16(tmem + (uint32_t)(t * a.cout), ad, bd, idesc, (q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::commit(tc::smem_addr(&empty[s]));
          if (q + 2 < nst) {  // the buffer is refilled once the MMAs just issued have read it
            ok = tc::mbar_wait(tc::smem_addr(&empty[s]), eph[s], kWaitNs);
            eph[s] ^= 1u;
          }
        }
      }
      fph[s] ^= 1u;
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (ok && q + 2 < nst) issue(q + 2);
    }
    if (lane == 0) {
      // the last commit of each buffer: every MMA done, no arrival pending
      for (int q = (nst >= 2 ? nst - 2 : 0); q < nst && ok; ++q) {
        const int s = q & 1;
        ok = tc::mbar_wait(tc::smem_addr(&empty[s]), eph[s], kWaitNs);
        eph[s] ^= 1u;
      }
      *s_ok = ok ? 1 : 0;
      if (!ok) atomicExch(&g_tc_timeout, 1);
    }
  }
  __syncthreads();
  float* part = a.partial + (long long)blockIdx.x * 27 * a.cout * a.cin;
  if (*s_ok && nst > 0) {
    tc::fence_after_sync();
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int t = 0; t < nt; ++t) {
      const int m = (T0 + t) * 128 + tid;  // TMEM lane = row of tile t
      const int tap = m / a.cin, ci = m - tap * a.cin;
      for (int n0 = 0; n0 < a.cout; n0 += 16) {
        uint32_t r[16];
        tc::tmem_ld16(trow + (uint32_t)(t * a.cout + n0), r);
        if (tap < 27) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            part[((long long)tap * a.cout + n0 + q) * a.cin + ci] = __uint_as_float(r[q]);
        }
      }
    }
  } else if (nst == 0) {  // a CTA without rows contributes zeros
    for (int t = 0; t < nt; ++t) {
      const int m = (T0 + t) * 128 + tid, tap = m / a.cin, ci = m - tap * a.cin;
      if (tap < 27)
        for (int n = 0; n < a.cout; ++n) part[((long long)tap * a.cout + n) * a.cin + ci] = 0.0f;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// dW[o][tap][i] = sum over chunks of partial[chunk][tap][o][i] (fixed order).
__global__ void k_dw_reduce(int nchunk, int Cin, int Cout, const float* __restrict__ partial, float* __restrict__ dW) {
  VOS_COUNT_EXEC();
  const long long n = 27LL * Cout * Cin;
  UNET_LOOP(e, n) {
    const int i = (int)(e % Cin), o = (int)((e / Cin) % Cout), tap = (int)(e / ((long long)Cin * Cout));
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += partial[((long long)c * 27 + tap) * Cout * Cin + (long long)o * Cin + i];
    dW[((long long)o * 27 + tap) * Cin + i] = s;
  }
}

// db[o] = sum_v g[v][o]: per-block partial sums, then a fixed-order total.
__global__ void __launch_bounds__(kThreads) k_db(long long V, int C, const float* __restrict__ g,
                                                float* __restrict__ partial) {
  VOS_COUNT_EXEC();
  __shared__ float sh[kThreads];
  const int per = kThreads / C;  // voxels handled side by side (C divides 256)
  const int c = threadIdx.x % C, lane = threadIdx.x / C;
  float acc = 0.0f;
  for (long long v = (long long)blockIdx.x * per + lane; v < V; v += (long long)gridDim.x * per)
    acc += g[v * C + c];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < C) {
    float s = 0.0f;
    for (int l = 0; l < per; ++l) s += sh[l * C + threadIdx.x];
    partial[(long long)blockIdx.x * C + threadIdx.x] = s;
  }
}
__global__ void k_db_reduce(int nb, int C, const float* __restrict__ partial, float* __restrict__ db) {
  VOS_COUNT_EXEC();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.0f;
  for (int b = 0; b < nb; ++b) s += partial[(long long)b * C + c];
  db[c] = s;
}

// gf[v][c] += gc[parent(v)][c] / 8   (pool backward, added into gf)
__global__ void k_pool_bwd_add(int fx, int fy, int fz, int C, const float* __restrict__ gc, float* __restrict__ gf) {
  VOS_COUNT_EXEC();
  const long long n = (long long)fx * fy * fz * C;
  const int cx = fx / 2, cy = fy / 2;
  UNET_LOOP(t, n) {
    const int c = (int)(t % C);
    const long long v = t / C;
    const int i = (int)(v % fx), j = (int)((v / fx) % fy), k = (int)(v / ((long long)fx * fy));
    const long long p = (i / 2) + (long long)cx * ((j / 2) + (long long)cy * (k / 2));
    gf[t] += 0.125f * gc[p * C + c];
  }
}

// Up-concat backward: gcoarse[p][c] = sum over the 8 children of
// gcat[child][c] (c < Cu); gskip[v][c] = gcat[v][Cu + c].
__global__ void k_up_bwd(int cx, int cy, int cz, int Cu, int Ctot, const float* __restrict__ gcat,
                         float* __restrict__ gcoarse) {
  VOS_COUNT_EXEC();
  const long long n = (long long)cx * cy * cz * Cu;
  const int fx = 2 * cx, fy = 2 * cy;
  UNET_LOOP(t, n) {
    const int c = (int)(t % Cu);
    const long long p = t / Cu;
    const int i = (int)(p % cx), j = (int)((p / cx) % cy), k = (int)(p / ((long long)cx * cy));
    float s = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const long long fv = (2 * i + dx) + (long long)fx * ((2 * j + dy) + (long long)fy * (2 * k + dz));
          s += gcat[fv * Ctot + c];
        }
    gcoarse[t] = s;
  }
}
__global__ void k_split_skip(long long V, int Cu, int Cs, const float* __restrict__ gcat, float* __restrict__ gskip) {
  VOS_COUNT_EXEC();
  const long long n = V * Cs;
  UNET_LOOP(t, n) {
    const long long v = t / Cs;
    gskip[t] = gcat[v * (Cu + Cs) + Cu + (t % Cs)];
  }
}

// Adam (bias-corrected moments) on a flat parameter range.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  VOS_COUNT_EXEC();
  UNET_LOOP(e, n) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// out = A z for the symmetric FP64 pressure operator (FP64 sums, FP32 out).
__global__ void k_apply_op(Op<double> A, const float* __restrict__ z, float* __restrict__ out) {
  VOS_COUNT_EXEC();
  const Box b = A.box;
  const long long n = box_cells(b), sy = b.mx, sz = (long long)b.mx * b.my;
  UNET_LOOP(c, n) {
    const int i = (int)(c % b.mx), j = (int)((c / b.mx) % b.my), k = (int)(c / sz);
    double y = A.diag[c] * (double)z[c];
    if (i + 1 < b.mx) y += A.xp[c] * (double)z[c + 1];
    if (i > 0) y += A.xp[c - 1] * (double)z[c - 1];
    if (j + 1 < b.my) y += A.yp[c] * (double)z[c + sy];
    if (j > 0) y += A.yp[c - sy] * (double)z[c - sy];
    if (b.mz > 1) {
      if (k + 1 < b.mz) y += A.zp[c] * (double)z[c + sz];
      if (k > 0) y += A.zp[c - sz] * (double)z[c - sz];
    }
    out[c] = (float)y;
  }
}

// res = A z - r inv_rms; sums of res^2 and (r inv_rms)^2.
__global__ void __launch_bounds__(kThreads) k_loss_res(long long n, const float* __restrict__ Az,
                                                      const float* __restrict__ r, const float* scal,
                                                      float* __restrict__ res, double* out, RedScratch rs) {
  VOS_COUNT_EXEC();
  const float inv = scal[0];
  double acc[2] = {0.0, 0.0};
  UNET_LOOP(c, n) {
    const float rh = r[c] * inv;
    const float e = Az[c] - rh;
    res[c] = e;
    acc[0] += (double)e * e;
    acc[1] += (double)rh * rh;
  }
  if (grid_sum<2>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}
// dz = (2 / |r_hat|^2) A res  (A res already in dz)
__global__ void k_scale_dz(long long n, const double* sums, float* __restrict__ dz) {
  VOS_COUNT_EXEC();
  const float f = sums[1] > 0.0 ? (float)(2.0 / sums[1]) : 0.0f;
  UNET_LOOP(c, n) dz[c] *= f;
}

__global__ void __launch_bounds__(kThreads) k_sumsq(long long n, const float* __restrict__ r, double* out,
                                                   RedScratch rs) {
  VOS_COUNT_EXEC();
  double acc[1] = {0.0};
  UNET_LOOP(c, n) acc[0] += (double)r[c] * r[c];
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) out[0] = acc[0];
}

}  // namespace unet
}  // namespace vos

// ---------------------------------------------------------------------------
// The network object: weights, Adam state, activations and gradients for
// one box.
// ---------------------------------------------------------------------------
namespace vos {
namespace unet {

struct LayerSpec {
  int cin, cout, lev;
};
// enc1a enc1b enc2a enc2b enc3a enc3b dec2a dec2b dec1a dec1b
constexpr LayerSpec kSpec[10] = {{2, 16, 0},  {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                                 {64, 64, 2}, {96, 32, 1}, {32, 32, 1}, {48, 16, 0}, {16, 16, 0}};
enum { ENC1A, ENC1B, ENC2A, ENC2B, ENC3A, ENC3B, DEC2A, DEC2B, DEC1A, DEC1B };

struct Layer {
  int li, cin, cing, cout, lev;
  float *W, *b, *gW, *gb, *mW, *vW, *mb, *vb;  // W: [cout][27][cing]
  __nv_bfloat16 *img, *imgT, *out;             // weight images (forward, data gradient); out: [V_lev][cout]
};

long long num_params() {
  long long n = 17;
  for (const auto& l : kSpec) n += (long long)l.cout * 27 * l.cin + l.cout;
  return n;
}

}  // namespace unet
}  // namespace vos

struct vos_unet {
  vos::unet::Dims d;
  int lx[3], ly[3], lz[3];
  long long V[3];
  vos::unet::Layer L[10];
  float *head, *ghead, *mhead, *vhead;  // 17 = w[16], b
  __nv_bfloat16 *x0, *p1, *p2, *cat2, *cat1;
  float* scal;    // [inv_rms, rms]
  double* dscal;  // [|r|^2, |res|^2, |r_hat|^2]
  float* z;       // [physical cells] network output of the last forward
  vos::RedScratch rs;
  bool train;
  float *gA, *gB, *ge1, *ge2, *gpre;
  __nv_bfloat16* gpre16;
  float *part_dw, *part_db;
  long long chunk[3];
  int nchunk[3], ndb;
  float *az, *res, *dz;
  const double* eps;  // fluid fraction of the attached handle (device)
  int adam_t;
  cudaStream_t st;
  std::vector<void*> blocks;
};

namespace vos {
namespace unet {

static void* ualloc(vos_unet* u, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, (bytes + 255) & ~(size_t)255) != cudaSuccess) return nullptr;
  u->blocks.push_back(p);
  return p;
}

static void destroy_net(vos_unet* u) {
  if (!u) return;
  cudaStreamSynchronize(u->st);
  for (void* p : u->blocks) cudaFree(p);
  delete u;
}

static ConvArgs conv_args(const vos_unet* u, int lev, const __nv_bfloat16* x, int cin, const __nv_bfloat16* w,
                          const float* bias, int cout, int relu, float* yf, __nv_bfloat16* yb) {
  ConvArgs a;
  a.x = x;
  a.img = w;
  a.bias = bias;
  a.yf = yf;
  a.yb = yb;
  a.nx = u->lx[lev];
  a.ny = u->ly[lev];
  a.nz = u->lz[lev];
  a.cin = cin;
  a.cout = cout;
  a.relu = relu;
  a.V = u->V[lev];
  return a;
}

static void prep_weights(vos_unet* u) {
  for (auto& l : u->L) {
    const long long n = 27LL * l.cout * l.cing;
    (void)n;
    conv_image(l.cout, l.cing, 0, l.W, l.img, u->st);
    if (l.li > 0) conv_image(l.cout, l.cing, 1, l.W, l.imgT, u->st);
  }
}

// Forward pass: x0 from (r, eps), ten convs, head -> z (T, physical cells).
// rr: device |r|^2; use_scale multiplies the output by rms(r).
template <typename T>
static cudaError_t forward(vos_unet* u, const T* r, const double* eps, const double* rr, int use_scale, T* zout) {
  cudaStream_t st = u->st;
  const Dims d = u->d;
  const double nphys = (double)d.px * d.py * d.pz;
  vlaunch("unet_rms", 0.0, k_rms, 1, 32, st, rr, nphys, u->scal);
  vlaunch("unet_pack", 0.0, k_pack<T>, ugrid(u->V[0]), kThreads, st, d, r, eps, (const float*)u->scal, u->x0);
  Layer* L = u->L;
  auto conv = [&](int li, const __nv_bfloat16* x) -> cudaError_t {
    Layer& l = L[li];
    return conv3d(conv_args(u, l.lev, x, l.cing, l.img, l.b, l.cout, 1, nullptr, l.out), st);
  };
  VOS_CUDA_TRY(conv(ENC1A, u->x0));
  VOS_CUDA_TRY(conv(ENC1B, L[ENC1A].out));
  vlaunch("unet_pool", 0.0, k_pool, ugrid(u->V[1] * 2), kThreads, st, u->lx[1], u->ly[1], u->lz[1], 16,
          (const __nv_bfloat16*)L[ENC1B].out, u->p1);
  VOS_CUDA_TRY(conv(ENC2A, u->p1));
  VOS_CUDA_TRY(conv(ENC2B, L[ENC2A].out));
  vlaunch("unet_pool", 0.0, k_pool, ugrid(u->V[2] * 4), kThreads, st, u->lx[2], u->ly[2], u->lz[2], 32,
          (const __nv_bfloat16*)L[ENC2B].out, u->p2);
  VOS_CUDA_TRY(conv(ENC3A, u->p2));
  VOS_CUDA_TRY(conv(ENC3B, L[ENC3A].out));
  vlaunch("unet_up", 0.0, k_up_concat, ugrid(u->V[1] * 12), kThreads, st, u->lx[1], u->ly[1], u->lz[1], 64, 32,
          (const __nv_bfloat16*)L[ENC3B].out, (const __nv_bfloat16*)L[ENC2B].out, u->cat2);
  VOS_CUDA_TRY(conv(DEC2A, u->cat2));
  VOS_CUDA_TRY(conv(DEC2B, L[DEC2A].out));
  vlaunch("unet_up", 0.0, k_up_concat, ugrid(u->V[0] * 6), kThreads, st, u->lx[0], u->ly[0], u->lz[0], 32, 16,
          (const __nv_bfloat16*)L[DEC2B].out, (const __nv_bfloat16*)L[ENC1B].out, u->cat1);
  VOS_CUDA_TRY(conv(DEC1A, u->cat1));
  VOS_CUDA_TRY(conv(DEC1B, L[DEC1A].out));
  vlaunch("unet_head", 0.0, k_head<T>, ugrid((long long)nphys), kThreads, st, d, (const __nv_bfloat16*)L[DEC1B].out,
          (const float*)u->head, (const float*)u->scal, use_scale, zout);
  return cudaGetLastError();
}

// Backward of one conv layer: g_out (FP32 [V][cout]) -> gW, gb and, when
// g_in is given, the data gradient g_in (FP32 [V][cing]).
static cudaError_t layer_backward(vos_unet* u, int li, const __nv_bfloat16* xin, const float* g_out, float* g_in) {
  cudaStream_t st = u->st;
  Layer& l = u->L[li];
  const long long V = u->V[l.lev];
  vlaunch("unet_relu_bwd", 0.0, k_relu_bwd, ugrid(V * l.cout), kThreads, st, V * l.cout, g_out,
          (const __nv_bfloat16*)l.out, u->gpre, u->gpre16);
  const int nch = u->nchunk[l.lev];
  static bool dw_attr = false;
  if (!dw_attr) {
    // the widest stage: 64-voxel boxes (any level at least 64 cells along x)
    // and the layer with the most A tiles per CTA and output channels
    size_t mx = 0;
    for (const auto& s : kSpec) mx = std::max(mx, dw_smem_bytes(s.cin < 8 ? 8 : s.cin, s.cout, 64));
    VOS_CUDA_TRY(cudaFuncSetAttribute(k_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    dw_attr = true;
  }
  const int lx = u->lx[l.lev], ly = u->ly[l.lev], lz = u->lz[l.lev], w = dw_width(lx);
  alignas(64) CUtensorMap tmx, tmg;
  VOS_CUDA_TRY(make_row_map(&tmx, xin, l.cing, lx, ly, lz, w));
  VOS_CUDA_TRY(make_row_map(&tmg, u->gpre16, l.cout, lx, ly, lz, w));
  const DwArgs da{u->part_dw, lx, ly, lz, l.cing, l.cout, w, (lx + w - 1) / w, (int)u->chunk[l.lev],
                  dw_tiles(l.cing), dw_tpc(l.cing, l.cout)};
  const dim3 gdw((unsigned)nch, (unsigned)((da.tiles + da.tpc - 1) / da.tpc));
  vlaunch_smem("unet_dw_tc", 2.0 * 27.0 * l.cing * l.cout * (double)V, k_dw_tc, gdw, dim3(kTM),
               dw_smem_bytes(l.cing, l.cout, w), st, tmx, tmg, da);
  vlaunch("unet_dw_reduce", 0.0, k_dw_reduce, ugrid(27LL * l.cout * l.cing), kThreads, st, nch, l.cing, l.cout,
          (const float*)u->part_dw, l.gW);
  vlaunch("unet_db", 0.0, k_db, u->ndb, kThreads, st, V, l.cout, (const float*)u->gpre, u->part_db);
  vlaunch("unet_db_reduce", 0.0, k_db_reduce, 1, 64, st, u->ndb, l.cout, (const float*)u->part_db, l.gb);
  if (g_in) VOS_CUDA_TRY(conv3d(conv_args(u, l.lev, u->gpre16, l.cout, l.imgT, nullptr, l.cing, 0, g_in, nullptr), st));
  return cudaGetLastError();
}

// Gradients of sum(dz * z) for the last forward (dz: FP32 physical cells).
static cudaError_t backward(vos_unet* u, const float* dz) {
  cudaStream_t st = u->st;
  Layer* L = u->L;
  vlaunch("unet_head_bwd", 0.0, k_head_bwd, ugrid(u->V[0]), kThreads, st, u->d, dz,
          (const __nv_bfloat16*)L[DEC1B].out, (const float*)u->head, u->gA, u->ghead, u->rs);
  VOS_CUDA_TRY(layer_backward(u, DEC1B, L[DEC1A].out, u->gA, u->gB));
  VOS_CUDA_TRY(layer_backward(u, DEC1A, u->cat1, u->gB, u->gA));  // gA = g_cat1 [V0][48]
  vlaunch("unet_up_bwd", 0.0, k_up_bwd, ugrid(u->V[1] * 32), kThreads, st, u->lx[1], u->ly[1], u->lz[1], 32, 48,
          (const float*)u->gA, u->gB);
  vlaunch("unet_split", 0.0, k_split_skip, ugrid(u->V[0] * 16), kThreads, st, u->V[0], 32, 16, (const float*)u->gA,
          u->ge1);
  VOS_CUDA_TRY(layer_backward(u, DEC2B, L[DEC2A].out, u->gB, u->gA));
  VOS_CUDA_TRY(layer_backward(u, DEC2A, u->cat2, u->gA, u->gB));  // gB = g_cat2 [V1][96]
  vlaunch("unet_up_bwd", 0.0, k_up_bwd, ugrid(u->V[2] * 64), kThreads, st, u->lx[2], u->ly[2], u->lz[2], 64, 96,
          (const float*)u->gB, u->gA);
  vlaunch("unet_split", 0.0, k_split_skip, ugrid(u->V[1] * 32), kThreads, st, u->V[1], 64, 32, (const float*)u->gB,
          u->ge2);
  VOS_CUDA_TRY(layer_backward(u, ENC3B, L[ENC3A].out, u->gA, u->gB));
  VOS_CUDA_TRY(layer_backward(u, ENC3A, u->p2, u->gB, u->gA));  // gA = g_p2 [V2][32]
  vlaunch("unet_pool_bwd", 0.0, k_pool_bwd_add, ugrid(u->V[1] * 32), kThreads, st, u->lx[1], u->ly[1], u->lz[1], 32,
          (const float*)u->gA, u->ge2);
  VOS_CUDA_TRY(layer_backward(u, ENC2B, L[ENC2A].out, u->ge2, u->gA));
  VOS_CUDA_TRY(layer_backward(u, ENC2A, u->p1, u->gA, u->gB));  // gB = g_p1 [V1][16]
  vlaunch("unet_pool_bwd", 0.0, k_pool_bwd_add, ugrid(u->V[0] * 16), kThreads, st, u->lx[0], u->ly[0], u->lz[0], 16,
          (const float*)u->gB, u->ge1);
  VOS_CUDA_TRY(layer_backward(u, ENC1B, L[ENC1A].out, u->ge1, u->gA));
  VOS_CUDA_TRY(layer_backward(u, ENC1A, u->x0, u->gA, nullptr));
  return cudaGetLastError();
}

static void adam_step(vos_unet* u, float lr) {
  u->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f, e = 1e-8f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)u->adam_t)), c2 = 1.0f / (1.0f - powf(b2, (float)u->adam_t));
  for (auto& l : u->L) {
    const long long nw = 27LL * l.cout * l.cing;
    vlaunch("unet_adam", 0.0, k_adam, ugrid(nw), kThreads, u->st, nw, l.W, (const float*)l.gW, l.mW, l.vW, lr, b1, b2,
            e, c1, c2);
    vlaunch("unet_adam", 0.0, k_adam, 1, kThreads, u->st, (long long)l.cout, l.b, (const float*)l.gb, l.mb, l.vb, lr,
            b1, b2, e, c1, c2);
  }
  vlaunch("unet_adam", 0.0, k_adam, 1, kThreads, u->st, 17LL, u->head, (const float*)u->ghead, u->mhead, u->vhead,
          lr, b1, b2, e, c1, c2);
  prep_weights(u);
}

// Host flat vector (oracle layout: per layer W[cout][3][3][3][cin] then b,
// then head w[16], b) <-> device tensors (padded input channels).
static cudaError_t params_io(vos_unet* u, float* host, bool to_device, bool grads) {
  long long off = 0;
  std::vector<float> buf;
  for (auto& l : u->L) {
    const long long nw = 27LL * l.cout * l.cing;
    buf.assign((size_t)nw, 0.0f);
    float* dW = grads ? l.gW : l.W;
    float* db = grads ? l.gb : l.b;
    if (to_device) {
      for (int o = 0; o < l.cout; ++o)
        for (int t = 0; t < 27; ++t)
          for (int i = 0; i < l.cin; ++i)
            buf[((size_t)o * 27 + t) * l.cing + i] = host[off + ((long long)o * 27 + t) * l.cin + i];
      VOS_CUDA_TRY(cudaMemcpy(dW, buf.data(), nw * sizeof(float), cudaMemcpyHostToDevice));
      VOS_CUDA_TRY(cudaMemcpy(db, host + off + 27LL * l.cout * l.cin, l.cout * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      VOS_CUDA_TRY(cudaMemcpy(buf.data(), dW, nw * sizeof(float), cudaMemcpyDeviceToHost));
      for (int o = 0; o < l.cout; ++o)
        for (int t = 0; t < 27; ++t)
          for (int i = 0; i < l.cin; ++i)
            host[off + ((long long)o * 27 + t) * l.cin + i] = buf[((size_t)o * 27 + t) * l.cing + i];
      VOS_CUDA_TRY(cudaMemcpy(host + off + 27LL * l.cout * l.cin, db, l.cout * sizeof(float), cudaMemcpyDeviceToHost));
    }
    off += 27LL * l.cout * l.cin + l.cout;
  }
  float* dh = grads ? u->ghead : u->head;
  if (to_device)
    VOS_CUDA_TRY(cudaMemcpy(dh, host + off, 17 * sizeof(float), cudaMemcpyHostToDevice));
  else
    VOS_CUDA_TRY(cudaMemcpy(host + off, dh, 17 * sizeof(float), cudaMemcpyDeviceToHost));
  if (to_device && !grads) {
    // a new parameter set restarts the optimiser
    for (auto& l : u->L) {
      const long long nw = 27LL * l.cout * l.cing;
      cudaMemset(l.mW, 0, nw * 4);
      cudaMemset(l.vW, 0, nw * 4);
      cudaMemset(l.mb, 0, l.cout * 4);
      cudaMemset(l.vb, 0, l.cout * 4);
    }
    cudaMemset(u->mhead, 0, 17 * 4);
    cudaMemset(u->vhead, 0, 17 * 4);
    u->adam_t = 0;
    prep_weights(u);
  }
  return cudaStreamSynchronize(u->st);
}

static vos_unet* create_net(int px, int py, int pz, bool train, cudaStream_t st) {
  vos_unet* u = new vos_unet();
  u->st = st;
  u->train = train;
  u->adam_t = 0;
  u->eps = nullptr;
  auto up4 = [](int n) { return (n + 3) & ~3; };
  u->d = Dims{up4(px), up4(py), up4(pz), px, py, pz};
  for (int l = 0; l < 3; ++l) {
    u->lx[l] = u->d.nx >> l;
    u->ly[l] = u->d.ny >> l;
    u->lz[l] = u->d.nz >> l;
    u->V[l] = (long long)u->lx[l] * u->ly[l] * u->lz[l];
  }
  bool ok = true;
  auto A = [&](size_t bytes) -> void* {
    void* p = ualloc(u, bytes);
    if (!p) ok = false;
    return p;
  };
  const long long V0 = u->V[0], V1 = u->V[1], V2 = u->V[2];
  const long long nphys = (long long)px * py * pz;
  for (int i = 0; i < 10; ++i) {
    Layer& l = u->L[i];
    l.cin = kSpec[i].cin;
    l.cing = kSpec[i].cin < 8 ? 8 : kSpec[i].cin;
    l.cout = kSpec[i].cout;
    l.lev = kSpec[i].lev;
    const long long nw = 27LL * l.cout * l.cing;
    l.W = (float*)A(nw * 4);
    l.b = (float*)A(l.cout * 4);
    l.li = i;
    l.img = (__nv_bfloat16*)A(conv_image_elems(l.cing, l.cout) * 2);
    l.imgT = (__nv_bfloat16*)A(conv_image_elems(l.cout, l.cing) * 2);
    l.out = (__nv_bfloat16*)A((size_t)u->V[l.lev] * l.cout * 2);
    l.gW = (float*)A(nw * 4);
    l.gb = (float*)A(l.cout * 4);
    l.mW = (float*)A(nw * 4);
    l.vW = (float*)A(nw * 4);
    l.mb = (float*)A(l.cout * 4);
    l.vb = (float*)A(l.cout * 4);
  }
  u->head = (float*)A(17 * 4);
  u->ghead = (float*)A(17 * 4);
  u->mhead = (float*)A(17 * 4);
  u->vhead = (float*)A(17 * 4);
  u->x0 = (__nv_bfloat16*)A((size_t)V0 * 8 * 2);
  u->p1 = (__nv_bfloat16*)A((size_t)V1 * 16 * 2);
  u->p2 = (__nv_bfloat16*)A((size_t)V2 * 32 * 2);
  u->cat2 = (__nv_bfloat16*)A((size_t)V1 * 96 * 2);
  u->cat1 = (__nv_bfloat16*)A((size_t)V0 * 48 * 2);
  u->scal = (float*)A(16);
  u->dscal = (double*)A(64);
  u->z = (float*)A((size_t)nphys * 4);
  u->rs.partials = (double*)A(32 * kMaxRedBlocks * sizeof(double));
  u->rs.counter = (unsigned int*)A(256);
  if (train) {
    const long long gmax = std::max(std::max(V0 * 48, V1 * 96), V2 * 64);
    u->gA = (float*)A(gmax * 4);
    u->gB = (float*)A(gmax * 4);
    u->ge1 = (float*)A(V0 * 16 * 4);
    u->ge2 = (float*)A(V1 * 32 * 4);
    const long long pmax = std::max(std::max(V0 * 16, V1 * 32), V2 * 64);
    u->gpre = (float*)A(pmax * 4);
    u->gpre16 = (__nv_bfloat16*)A(pmax * 2);
    long long pdw = 0;
    for (int l = 0; l < 3; ++l) {  // weight-gradient chunks: rows (j, k) per CTA, about two CTAs per SM
      const long long rows = (long long)u->ly[l] * u->lz[l], target = 2LL * g_num_sms;
      long long ch = (rows + target - 1) / target;
      const long long minrows = (256 + u->lx[l] - 1) / u->lx[l];  // 256 voxels per CTA at least
      if (ch < minrows) ch = minrows;
      u->chunk[l] = ch;
      u->nchunk[l] = (int)((rows + ch - 1) / ch);
    }
    for (auto& l : u->L) pdw = std::max(pdw, (long long)u->nchunk[l.lev] * 27 * l.cout * l.cing);
    u->part_dw = (float*)A(pdw * 4);
    u->ndb = 2 * g_num_sms;
    u->part_db = (float*)A((size_t)u->ndb * 64 * 4);
    u->az = (float*)A(nphys * 4);
    u->res = (float*)A(nphys * 4);
    u->dz = (float*)A(nphys * 4);
  } else {
    u->gA = u->gB = u->ge1 = u->ge2 = u->gpre = nullptr;
    u->gpre16 = nullptr;
    u->part_dw = u->part_db = nullptr;
    u->az = u->res = u->dz = nullptr;
  }
  if (!ok) {
    destroy_net(u);
    return nullptr;
  }
  cudaMemsetAsync(u->rs.counter, 0, 256, st);
  return u;
}

// Solver hook: z = UNet(r / rms(r), eps) * rms(r), rr = |r|^2 on the device.
template <typename T>
void precond_apply(vos_unet* u, const T* r, T* z, const double* rr, cudaStream_t st) {
  cudaStream_t keep = u->st;
  u->st = st;
  forward<T>(u, r, u->eps, rr, 1, z);
  u->st = keep;
}

}  // namespace unet

void unet_box(const vos_unet* net, int* px, int* py, int* pz) {
  *px = net->d.px;
  *py = net->d.py;
  *pz = net->d.pz;
}
void unet_attach_eps(vos_unet* net, const double* eps) { net->eps = eps; }

template <typename T>
void unet_precond(vos_unet* net, const T* r, T* z, const double* rr, cudaStream_t st) {
  unet::precond_apply<T>(net, r, z, rr, st);
}
template void unet_precond<float>(vos_unet*, const float*, float*, const double*, cudaStream_t);
template void unet_precond<double>(vos_unet*, const double*, double*, const double*, cudaStream_t);

}  // namespace vos

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace vos;

extern "C" {

int vos_conv3d_bf16(const uint16_t* x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const uint16_t* w,
                    const float* bias, int32_t cout, int32_t relu, float* y_f32, uint16_t* y_bf16, void* stream) {
  if (!x || !w || (!y_f32 && !y_bf16) || nx < 1 || ny < 1 || nz < 1 || !unet::conv_shape_ok(cin, cout)) {
    set_global_error("vos_conv3d_bf16: bad argument (cin a multiple of 8, cout a multiple of 16 in [16, 96])");
    return VOS_EINVAL;
  }
  // the kernel reads the weights in its shared-memory image layout: build
  // that in a temporary buffer
  __nv_bfloat16* img = nullptr;
  const long long nimg = unet::conv_image_elems(cin, cout);
  if (cudaMalloc((void**)&img, (size_t)nimg * 2) != cudaSuccess) {
    cudaGetLastError();
    set_global_error("vos_conv3d_bf16: device allocation failed");
    return VOS_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  {
    long long b = (nimg + kThreads - 1) / kThreads;
    if (b > 4096) b = 4096;
    vlaunch("unet_image", 0.0, unet::k_image_bf16, (int)b, kThreads, st, (int)cout, (int)cin,
            (const __nv_bfloat16*)w, img);
  }
  unet::ConvArgs a;
  a.x = (const __nv_bfloat16*)x;
  a.img = img;
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
  cudaError_t e = unet::conv3d(a, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(img);
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

int vos_unet_create(int32_t nx, int32_t ny, int32_t nz, int32_t train, void* stream, vos_unet** out) {
  if (!out || nx < 4 || ny < 4 || nz < 4) {
    set_global_error("vos_unet_create: need out and a box of at least 4 x 4 x 4");
    return VOS_EINVAL;
  }
  *out = nullptr;
  if ((double)nx * ny * nz > 4.0e8) {
    set_global_error("vos_unet_create: box too large");
    return VOS_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) g_num_sms = sms;
  vos_unet* u = unet::create_net(nx, ny, nz, train != 0, (cudaStream_t)stream);
  if (!u) {
    set_global_error("vos_unet_create: device allocation failed");
    return VOS_ENOMEM;
  }
  *out = u;
  return VOS_OK;
}

int64_t vos_unet_num_params(void) { return unet::num_params(); }

static int unet_io(vos_unet* u, float* host, int64_t n, bool to_dev, bool grads, const char* what) {
  if (!u || !host || n != unet::num_params()) {
    set_global_error(what);
    return VOS_EINVAL;
  }
  if (grads && !u->train) {
    set_global_error("vos_unet_get_grads: the network was created without training buffers");
    return VOS_EINVAL;
  }
  cudaError_t e = unet::params_io(u, host, to_dev, grads);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  return VOS_OK;
}

int vos_unet_set_params(vos_unet* u, const float* host, int64_t n) {
  return unet_io(u, const_cast<float*>(host), n, true, false, "vos_unet_set_params: bad argument");
}
int vos_unet_get_params(vos_unet* u, float* host, int64_t n) {
  return unet_io(u, host, n, false, false, "vos_unet_get_params: bad argument");
}
int vos_unet_get_grads(vos_unet* u, float* host, int64_t n) {
  return unet_io(u, host, n, false, true, "vos_unet_get_grads: bad argument");
}

static int unet_finish(vos_unet* u, const char* what) {
  cudaError_t e = cudaStreamSynchronize(u->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  if (unet::take_timeout_flag()) {
    set_global_error(what);
    return VOS_ETIMEOUT;
  }
  return VOS_OK;
}

int vos_unet_forward(vos_unet* u, const float* r, const double* eps, float* z) {
  if (!u || !r || !eps || !z) {
    set_global_error("vos_unet_forward: NULL argument");
    return VOS_EINVAL;
  }
  const long long n = (long long)u->d.px * u->d.py * u->d.pz;
  vlaunch("unet_sumsq", 0.0, unet::k_sumsq, unet::ugrid(n), kThreads, u->st, n, r, u->dscal, u->rs);
  cudaError_t e = unet::forward<float>(u, r, eps, u->dscal, 0, u->z);
  if (e == cudaSuccess) e = cudaMemcpyAsync(z, u->z, n * sizeof(float), cudaMemcpyDeviceToDevice, u->st);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  return unet_finish(u, "vos_unet_forward: a tensor-core wait ran out of time");
}

int vos_unet_backward(vos_unet* u, const float* dz) {
  if (!u || !dz || !u->train) {
    set_global_error("vos_unet_backward: NULL argument or no training buffers");
    return VOS_EINVAL;
  }
  cudaError_t e = unet::backward(u, dz);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  return unet_finish(u, "vos_unet_backward: a tensor-core wait ran out of time");
}

// Loss of the network on one residual r of h's pressure operator; with
// lr > 0 also one Adam step.
static int unet_loss_step(vos_unet* u, vos_handle* h, const float* r, float lr, bool update, float* loss) {
  if (!u || !h || !r || !loss || !u->train) {
    set_global_error("vos_unet_train_step: NULL argument or no training buffers");
    return VOS_EINVAL;
  }
  const Op<double>* A = handle_pressure_op(h);
  const double* eps = handle_eps(h);
  if (!A || !A->diag || A->box.mx != u->d.px || A->box.my != u->d.py || A->box.mz != u->d.pz) {
    set_global_error("vos_unet_train_step: the network box differs from the handle's grid");
    return VOS_EINVAL;
  }
  cudaStream_t st = u->st;
  const long long n = (long long)u->d.px * u->d.py * u->d.pz;
  const int g = unet::ugrid(n);
  vlaunch("unet_sumsq", 0.0, unet::k_sumsq, g, kThreads, st, n, r, u->dscal, u->rs);
  cudaError_t e = unet::forward<float>(u, r, eps, u->dscal, 0, u->z);
  if (e == cudaSuccess) {
    vlaunch("unet_apply_op", 0.0, unet::k_apply_op, g, kThreads, st, *A, (const float*)u->z, u->az);
    vlaunch("unet_loss", 0.0, unet::k_loss_res, g, kThreads, st, n, (const float*)u->az, r, (const float*)u->scal,
            u->res, u->dscal + 1, u->rs);
    if (update) {
      vlaunch("unet_apply_op", 0.0, unet::k_apply_op, g, kThreads, st, *A, (const float*)u->res, u->dz);
      vlaunch("unet_scale_dz", 0.0, unet::k_scale_dz, g, kThreads, st, n, (const double*)(u->dscal + 1), u->dz);
      e = unet::backward(u, u->dz);
      if (e == cudaSuccess) unet::adam_step(u, lr);
    }
  }
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return VOS_ECUDA;
  }
  double sums[2] = {0.0, 0.0};
  cudaMemcpyAsync(sums, u->dscal + 1, sizeof(sums), cudaMemcpyDeviceToHost, st);
  int rc = unet_finish(u, "vos_unet_train_step: a tensor-core wait ran out of time");
  if (rc != VOS_OK) return rc;
  *loss = sums[1] > 0.0 ? (float)(sums[0] / sums[1]) : 0.0f;
  return VOS_OK;
}

int vos_unet_train_step(vos_unet* u, vos_handle* h, const float* r, float lr, float* loss) {
  if (!(lr > 0.0f) || !std::isfinite(lr)) {
    set_global_error("vos_unet_train_step: lr must be > 0");
    return VOS_EINVAL;
  }
  return unet_loss_step(u, h, r, lr, true, loss);
}
int vos_unet_eval_loss(vos_unet* u, vos_handle* h, const float* r, float* loss) {
  return unet_loss_step(u, h, r, 0.0f, false, loss);
}

void vos_unet_destroy(vos_unet* u) { unet::destroy_net(u); }

}  // extern "C"
