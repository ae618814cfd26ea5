// Allocation-free variant of the time-step limit (vos_suggest_dt_noalloc).
//
// Some callers cannot let a library allocate device memory: hosts that keep
// every byte of the GPU in their own pool (a framework's caching allocator,
// a plugin inside another application), and time-critical loops that must
// not pay the implicit device-wide synchronisation a cudaMalloc/cudaFree can
// cause.  This entry point computes the same limit as vos_suggest_dt from
// fields the caller already holds on the device, and keeps its scratch -- one
// pair of partial maxima per 256-cell tile, a completion counter and the two
// results -- in a file-scope device array that every GPU loading the library
// holds until the process exits.
#include <cmath>
#include <mutex>

#include "../../include/vos.h"
#include "vos_internal.cuh"

namespace vos {
void set_global_error(const char* msg);
}

namespace {

constexpr int kTile = 256;                 // cells per block (one block per tile)
constexpr int kMaxTiles = 65536;           // tiles the scratch can hold
constexpr long long kMaxCells = (long long)kTile * kMaxTiles;  // 16,777,216 cells
constexpr int kCounterSlot = 2 * kMaxTiles;                    // counter lives here
constexpr int kResultSlot = 2 * kMaxTiles + 8;                 // results [umax, rmax]
constexpr int kScratchDoubles = 2 * kMaxTiles + 16;            // 1 MiB + 128 B

// The scratch.  In host code this name is only a stand-in: its device
// address comes from cudaGetSymbolAddress (once per device, below).
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_ready[kMaxDevices] = {};
double* g_addr[kMaxDevices] = {};

struct Grid {
  int dim, nx, ny, nz;
  int hasv;  // 0: no v array (ny == 1, every v face is a wall face with zero velocity)
  double Vm;
};

__device__ __forceinline__ long long cix(const Grid& g, int i, int j, int k) {
  return i + (long long)g.nx * (j + (long long)g.ny * k);
}
__device__ __forceinline__ long long fix(const Grid& g, int a, int i, int j, int k) {
  const int fx = g.nx + (a == 0), fy = g.ny + (a == 1);
  return i + (long long)fx * (j + (long long)fy * k);
}

// NaN compares false with everything, so fmax would drop it: a NaN speed or
// rate is taken as +inf instead (the limit then becomes dt = 0).
__device__ __forceinline__ double nan_to_inf(double x) { return (x == x) ? x : INFINITY; }

// One block per 256-cell tile: per cell, |u_f| / eps_f over its minus faces
// (and its plus face at the last cell along an axis) and |Vm R|; block
// maxima to scratch[2 tile], scratch[2 tile + 1]; the last block reduces
// the tiles in order and writes the two results.  Axis y is skipped when
// there is no v array (g.hasv == 0, only allowed for ny == 1).
__global__ void k_dt_limits_tiles(Grid g, const double* __restrict__ eps, const double* __restrict__ u0,
                                  const double* __restrict__ u1, const double* __restrict__ u2,
                                  const double* __restrict__ R, double* scratch) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long c = (long long)blockIdx.x * kTile + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (c < N) {
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const int n3[3] = {g.nx, g.ny, g.nz};
    const double* us[3] = {u0, u1, u2};
    const double e = eps[c];
    const int nb = (g.dim == 2) ? 2 : 3;
    for (int d = 0; d < nb; ++d) {
      if (d == 1 && !g.hasv) continue;
      int lo[3] = {i, j, k};
      lo[d] -= 1;
      const double ef = (lo[d] >= 0) ? 0.5 * (e + eps[cix(g, lo[0], lo[1], lo[2])]) : e;
      v[0] = fmax(v[0], nan_to_inf(fabs(us[d][fix(g, d, i, j, k)]) / ef));
      int f[3] = {i, j, k};
      if (f[d] == n3[d] - 1) {
        f[d] += 1;
        v[0] = fmax(v[0], nan_to_inf(fabs(us[d][fix(g, d, f[0], f[1], f[2])]) / e));
      }
    }
    v[1] = nan_to_inf(fabs(g.Vm * R[c]));
  }
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounterSlot);
  __shared__ double sh[2][kTile / 32];
  __shared__ bool last;
  for (int q = 0; q < 2; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0, m1 = 0.0;
    for (int w = 0; w < kTile / 32; ++w) {
      m0 = fmax(m0, sh[0][w]);
      m1 = fmax(m1, sh[1][w]);
    }
    scratch[2 * blockIdx.x] = m0;
    scratch[2 * blockIdx.x + 1] = m1;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double m[2] = {0.0, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kTile) {
    m[0] = fmax(m[0], __ldcg(scratch + 2 * b));
    m[1] = fmax(m[1], __ldcg(scratch + 2 * b + 1));
  }
  __syncthreads();
  for (int q = 0; q < 2; ++q) {
    double x = m[q];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0, m1 = 0.0;
    for (int w = 0; w < kTile / 32; ++w) {
      m0 = fmax(m0, sh[0][w]);
      m1 = fmax(m1, sh[1][w]);
    }
    scratch[kResultSlot] = m0;
    scratch[kResultSlot + 1] = m1;
    *counter = 0u;
  }
}

int fail(int code, const char* msg) {
  vos::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int vos_suggest_dt_noalloc(const vos_params* prm, const double* eps, const double* u, const double* v,
                                      const double* w, const double* R, double cfl, double deps_max, void* stream,
                                      double* dt) {
  if (!prm || !eps || !u || !R || !dt) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: NULL argument");
  if (prm->dim != 2 && prm->dim != 3) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: dim must be 2 or 3");
  if (prm->nx < 2 || prm->ny < 1 || prm->nz < 1 || (prm->dim == 2 && prm->nz != 1))
    return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: need nx >= 2, ny >= 1, nz >= 1 (nz == 1 in 2D)");
  if (!(prm->dx > 0.0) || !std::isfinite(prm->dx) || !std::isfinite(prm->Vm))
    return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: dx must be finite and > 0, Vm finite");
  if (prm->ny > 1 && !v) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: v is NULL");
  if (prm->dim == 3 && !w) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: w is NULL for a 3D grid");
  if (!(cfl > 0.0) || !(deps_max > 0.0)) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: cfl and deps_max must be > 0");
  const long long N = (long long)prm->nx * prm->ny * prm->nz;
  if (N > kMaxCells)
    return fail(VOS_EINVAL,
                "vos_suggest_dt_noalloc: grid has more than 16777216 cells, the most its fixed scratch holds; "
                "use vos_suggest_dt");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(VOS_ECUDA, "vos_suggest_dt_noalloc: no usable current device");
  cudaStream_t st = (cudaStream_t)stream;
  if (st != nullptr) {
    // the scratch address below is the current device's: the stream must
    // belong to that device
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: stream is not a valid CUDA stream");
    }
    if (sdev != dev) return fail(VOS_EINVAL, "vos_suggest_dt_noalloc: stream belongs to another device than the current one");
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      // Once per device, with that device current: the device address of
      // the scratch (the host-side name is not a device address).
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || p == nullptr) return fail(VOS_ECUDA, "vos_suggest_dt_noalloc: cudaGetSymbolAddress failed");
      g_addr[dev] = static_cast<double*>(p);
      g_ready[dev] = true;
    }
    scratch = g_addr[dev];
  }
  // The counter must start at zero (the array keeps the last call's contents).
  cudaError_t e = cudaMemsetAsync(scratch + kCounterSlot, 0, sizeof(double), st);
  if (e != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(e));
  Grid g{prm->dim, prm->nx, prm->ny, prm->nz, v != nullptr, prm->Vm};
  const unsigned tiles = (unsigned)((N + kTile - 1) / kTile);
  // v and w are never read when absent (hasv == 0; w only in 3D): u stands
  // in for the unused pointer arguments
  k_dt_limits_tiles<<<tiles, kTile, 0, st>>>(g, eps, u, v ? v : u, w ? w : u, R, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(e));
  double res[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(res, scratch + kResultSlot, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(e));
  const double d1 = res[0] > 0.0 ? cfl * prm->dx / res[0] : INFINITY;
  const double d2 = res[1] > 0.0 ? deps_max / res[1] : INFINITY;
  *dt = d1 < d2 ? d1 : d2;
  return VOS_OK;
}
