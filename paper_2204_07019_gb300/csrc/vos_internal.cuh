// Internal declarations of the VoS CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

struct vos_unet;
struct vos_handle;

namespace vos {

// ---------------------------------------------------------------------------
// Launch accounting: every kernel launch of the library goes through
// vlaunch(), which counts it and, when per-kernel timing is enabled for a
// matching name (vos_prof_enable), brackets it with CUDA events on the same
// stream and records its algorithmic bytes.
// ---------------------------------------------------------------------------
extern std::atomic<unsigned long long> g_launch_count;
unsigned long long exec_count_sum();  // sum of the per-file device counters
extern bool g_prof_any;
int prof_before(const char* name, double bytes, cudaStream_t st);
void prof_after(int slot, cudaStream_t st);

// Kernel executions counted on the device (one atomic per execution, by
// block 0 thread 0), so launches replayed inside CUDA graphs are counted.
#define VOS_COUNT_EXEC()                                                        \
  do {                                                                          \
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && \
        threadIdx.y == 0 && threadIdx.z == 0)                                   \
      atomicAdd(&vos_exec_count, 1ull);                                         \
  } while (0)

template <typename... KArgs, typename... Args>
inline void vlaunch(const char* name, double bytes, void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                    Args&&... args) {
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  int slot = g_prof_any ? prof_before(name, bytes, st) : -1;
  k<<<grid, block, 0, st>>>(std::forward<Args>(args)...);
  if (slot >= 0) prof_after(slot, st);
}

template <typename... KArgs, typename... Args>
inline void vlaunch_smem(const char* name, double bytes, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args&&... args) {
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  int slot = g_prof_any ? prof_before(name, bytes, st) : -1;
  k<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
  if (slot >= 0) prof_after(slot, st);
}

constexpr int kThreads = 256;             // threads per block of every grid kernel
constexpr int kWarps = kThreads / 32;     // warps per block
constexpr int kMaxRedBlocks = 8192;       // upper bound of blocks in reduction kernels
constexpr int kMaxRedValues = 8;          // values reduced per reduction kernel

// A box of unknowns, x fastest: index i + mx*(j + my*k).
struct Box {
  int mx, my, mz;
};
__host__ __device__ inline long long box_cells(Box b) { return (long long)b.mx * b.my * b.mz; }
__host__ inline Box coarse_box(Box b) {
  return Box{b.mx > 1 ? (b.mx + 1) / 2 : 1, b.my > 1 ? (b.my + 1) / 2 : 1, b.mz > 1 ? (b.mz + 1) / 2 : 1};
}

// Strided view of a box inside a larger array (e.g. the unknown faces of
// a velocity component inside its face array): element (i,j,k) at
// base[i + sy*j + sz*k].
template <typename T>
struct View {
  T* base;
  int sy, sz;
};

// 5/7-point stencil operator on a box:
//   (A x)_c = diag_c x_c + sum over existing neighbours n of a_{c->n} x_n.
// Symmetric operators store only the "plus" links (xp, yp, zp); the link
// to the minus neighbour is the plus link of that neighbour.  Non-symmetric
// operators also store xm, ym, zm.  dinv = omega / diag (Jacobi smoother).
template <typename T>
struct Op {
  Box box;
  int sym;
  T *diag, *dinv, *xp, *yp, *zp, *xm, *ym, *zm;
  // Matrix-free form of the pressure operator (FP32 fine level only): when
  // mfe is set, stencil sweeps compute the links from the fluid fraction,
  // a_cn = 0.5 (e_c + e_n) mfs, diag = sum of the links + 2 e_c mfs on the
  // outlet column (i = mx - 1), instead of reading diag/xp/yp/zp.
  const float* mfe;
  float mfs;
  // Constant-link form (FP32 momentum fine levels): when mfc != 0 every link
  // between two unknowns of the box is mfc (-nu / dx^2) and sweeps read only
  // diag, not xp/yp/zp.
  float mfc;
};

// Rows of the assembled stencil operators are formed with explicit rounding
// in every kernel that applies them (separate sweeps, fused passes, the
// cluster-resident cycle, the coarsest-level solve): A x = d x_c, then one
// FMA per link in the order x+, x-, y+, y-, z+, z-; a Jacobi update is one
// FMA, x + w (b - A x); the prolongation x + wc x_c[parent] one FMA.  So
// their results agree bit for bit whatever the compiler would contract.
// FP64 -> FP32 rounded to nearest (ties to even) by integer operations on the
// bit pattern: the conversion instruction executes on the FP64 pipe of this
// part, which bounds the kernels that convert.  Results in the normal FP32
// range (including the rounding up to infinity above the largest float) are
// those of the IEEE conversion; other magnitudes, NaN and infinity take the
// instruction.
__device__ __forceinline__ float f32_rn(double v) {
  const unsigned h = (unsigned)__double2hiint(v), l = (unsigned)__double2loint(v);
  const unsigned e = (h >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return __double2float_rn(v);
  unsigned bits = ((e - 896u) << 23) | ((h & 0xfffffu) << 3) | (l >> 29);
  const unsigned rem = l & 0x1fffffffu;  // the 29 bits dropped
  if (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) ++bits;  // a carry moves into the exponent
  return __uint_as_float((h & 0x80000000u) | bits);
}
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

// Work split: a warp handles one 32-cell row segment along x; blocks stride
// over segments.  Grid size is fixed per box so reductions are deterministic.
struct Seg {
  int spr;        // segments per row
  long long nseg; // total segments
};
__host__ __device__ inline Seg make_seg(Box b) {
  Seg s;
  s.spr = (b.mx + 31) / 32;
  s.nseg = (long long)s.spr * b.my * b.mz;
  return s;
}
__host__ int grid_for(Box b, int max_blocks);

// Decode segment q -> (i, row) for this lane.
__device__ __forceinline__ void seg_decode(const Seg& s, const Box& b, long long q, int& i, int& j,
                                           int& k) {
  long long row = q / s.spr;
  i = (int)(q - row * s.spr) * 32 + (int)(threadIdx.x & 31);
  j = (int)(row % b.my);
  k = (int)(row / b.my);
}

#define VOS_SEG_LOOP(seg, q)                                                          \
  for (long long q = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); q < (seg).nseg; \
       q += (long long)gridDim.x * kWarps)

// ---------------------------------------------------------------------------
// Deterministic block / grid reductions (fixed order, FP64).  Blocks of
// kThreads threads in any shape; grids in any shape.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lin_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ unsigned lin_bid() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ unsigned n_blocks() { return gridDim.x * gridDim.y * gridDim.z; }

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kWarps];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[q] = x;
  }
  const int t = lin_tid(), w = t >> 5, l = t & 31;
  __syncthreads();
  if (l == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][w] = v[q];
  }
  __syncthreads();
  if (t < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = (l < kWarps) ? sh[q][l] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[q] = x;
    }
  }
}

template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV]) {
  __shared__ double sh[NV][kWarps];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    v[q] = x;
  }
  const int t = lin_tid(), w = t >> 5, l = t & 31;
  __syncthreads();
  if (l == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][w] = v[q];
  }
  __syncthreads();
  if (t < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = (l < kWarps) ? sh[q][l] : -1e308;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
      v[q] = x;
    }
  }
}

// Grid-wide sum: each block publishes its partial sums; the last block to
// arrive adds the partials in block order and returns true in every thread
// of that block, with the totals in thread 0's v[].  Scratch: partials has
// room for NV * gridDim.x doubles; counter is 0 on entry and reset on exit.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* counter) {
  __shared__ bool last;
  block_sum<NV>(v);
  const unsigned nb = n_blocks();
  const int t = lin_tid();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * nb + lin_bid()] = v[q];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    s[q] = 0.0;
    for (int b = t; b < (int)nb; b += kThreads) s[q] += __ldcg(partials + q * nb + b);
  }
  block_sum<NV>(s);
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = s[q];
    *counter = 0u;
  }
  return true;
}

template <int NV>
__device__ bool grid_max(double (&v)[NV], double* partials, unsigned int* counter) {
  __shared__ bool last;
  block_max<NV>(v);
  const unsigned nb = n_blocks();
  const int t = lin_tid();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * nb + lin_bid()] = v[q];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    s[q] = -1e308;
    for (int b = t; b < (int)nb; b += kThreads) s[q] = fmax(s[q], __ldcg(partials + q * nb + b));
  }
  block_max<NV>(s);
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = s[q];
    *counter = 0u;
  }
  return true;
}

// Grid-wide NS sums and NM maxima in one pass (same protocol as grid_sum:
// partials of value q at partials[q * nb + block], the last block to arrive
// combines them in block order, thread 0 of that block holds the totals in
// s[] and m[]; NS + NM <= kMaxRedValues).
template <int NS, int NM>
__device__ bool grid_sum_max(double (&s)[NS], double (&m)[NM], double* partials, unsigned int* counter) {
  __shared__ bool last;
  block_sum<NS>(s);
  block_max<NM>(m);
  const unsigned nb = n_blocks();
  const int t = lin_tid();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NS; ++q) partials[q * nb + lin_bid()] = s[q];
#pragma unroll
    for (int q = 0; q < NM; ++q) partials[(NS + q) * nb + lin_bid()] = m[q];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double ts[NS], tm[NM];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    ts[q] = 0.0;
    for (int b = t; b < (int)nb; b += kThreads) ts[q] += __ldcg(partials + q * nb + b);
  }
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    tm[q] = -1e308;
    for (int b = t; b < (int)nb; b += kThreads) tm[q] = fmax(tm[q], __ldcg(partials + (NS + q) * nb + b));
  }
  block_sum<NS>(ts);
  block_max<NM>(tm);
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NS; ++q) s[q] = ts[q];
#pragma unroll
    for (int q = 0; q < NM; ++q) m[q] = tm[q];
    *counter = 0u;
  }
  return true;
}

// Reduction scratch shared by all kernels of one handle (one stream, so
// kernels never overlap).
struct RedScratch {
  double* partials;       // kMaxRedValues * kMaxRedBlocks
  unsigned int* counter;  // 1
};

// ---------------------------------------------------------------------------
// Linear solver (vos_solver.cu)
// ---------------------------------------------------------------------------

// Device scalars of one Krylov solve (FP64).
struct KScal {
  double bb, rr, rz, rz_old, pq, alpha, beta, omega, rho, rhv, tol2;
  double tol2s;  // diagonally preconditioned CG: stop when z.z <= tol2s (scaled norm)
  double ss, ts, tt;
  double rz_part;  // r.z of the fine sweep before the deflation's share (fused PCG)
  int done, iters, max_iters, breakdown;
};

struct MGParams {
  double omega;   // Jacobi damping
  double wc;      // coarse-correction weight
  int nu;         // pre/post sweeps
  int coarse_sweeps;
};

template <typename T>
struct Level {
  Op<T> op;
  T *x, *t, *b;  // solution, ping-pong, right-hand side
};

// Deflation of floating pore clusters (vos_deflate.cu).  A cluster is a
// connected set of cells joined by strong faces (face porosity >= a
// threshold) that reaches no Dirichlet cell: in the pressure operator it is
// tied to the rest of the domain only through solid-solid links, which are
// eps_min / 1 times weaker, so its mean value is a near-null mode that the
// smoother and the aggregation hierarchy hardly reduce.  The preconditioner
// adds the exact correction of those modes, M^-1 = V + W E^-1 W^T, with W the
// 0/1 indicator of each cluster and E = W^T A W (diagonal: distinct clusters
// are never joined by a link of A when every cluster boundary is weak, and
// the off-diagonal part is dropped when they are).
// ent[q] = cell | mask << kDeflMaskShift, mask bit d set when the neighbour in
// direction d (x-, x+, y-, y+, z-, z+) belongs to the same cluster; the
// entries of cluster k are ent[ptr[k] .. ptr[k+1]), cells ascending.
constexpr int kDeflMaskShift = 58;
constexpr unsigned long long kDeflCellMask = (1ull << kDeflMaskShift) - 1ull;
struct Defl {
  int K;                           // number of clusters (0: no deflation)
  const int* ptr;                  // K + 1
  const unsigned long long* ent;   // ptr[K]
  double* Einv;                    // K: 1 / E_kk (0 when E_kk <= 0)
};

// Multigrid hierarchy + Krylov vectors for one linear system.
template <typename T>
struct Hier {
  int nlev;
  Level<T> lev[16];
  MGParams mg;
  Defl defl;     // floating-cluster deflation (pressure only)
  vos_unet* net; // learned preconditioner (pressure only; eager solves)
  int tail;      // first level of the cluster-resident coarse cycle (nlev: none)
};

// Cluster-resident coarse cycle (vos_mgtail.cu): levels tail..nlev-1 of a
// V-cycle in one launch of one thread-block cluster, from lev[tail].b to
// lev[tail].x, bit-identical to the separate launches.  tail_plan picks the
// first level (nlev: none; g_tail_enabled = false disables it for
// hierarchies set up afterwards); tail_supported checks that the device can
// run the cluster with that much shared memory.
extern bool g_tail_enabled;
// Matrix-free FP32 pressure sweeps with four cells per thread and 16-byte
// accesses when the row length is a multiple of 4 (vos_solver.cu).
extern bool g_mf4;
extern int g_fused_pcg;  // fused Krylov forms, bit mask (vos_set_fused_pcg)
template <typename T>
int tail_plan(const Hier<T>& h);
template <typename T>
size_t tail_smem(const Hier<T>& h, int ls);
template <typename T, bool SYM>
bool tail_supported(size_t smem);
template <typename T, bool SYM>
void tail_launch(Hier<T>& h, int ls, const KScal* sc, cudaStream_t st);

// Host: label the floating clusters of the pressure operator built from the
// fluid fraction eps (nx*ny*nz, x fastest).  Faces with 0.5 (eps_a + eps_b)
// >= theta are strong; clusters of >= 2 cells that contain no outlet cell
// (i = nx - 1, the Dirichlet row of the pressure operator) are kept.  Fills
// ptr/ent (layout of Defl) and, when label is not NULL, label[c] = cluster
// id or -1.  Returns the number of clusters.
int floating_clusters(const double* eps, int nx, int ny, int nz, double theta, std::vector<int>& ptr,
                      std::vector<unsigned long long>& ent, int32_t* label);
constexpr double kDeflTheta = 0.01;

// E_kk = sum over the cluster's cells of (A 1_k)_c from the FP64 symmetric
// operator; stores 1 / E_kk in D.Einv.
void launch_defl_energy(const Defl& D, const Op<double>& A, cudaStream_t st);
// z += W E^-1 W^T r (skipped when the solve is done).
template <typename T>
void launch_defl_apply(const Defl& D, const T* r, T* z, const KScal* sc, cudaStream_t st);
// The same for PCG with r.z fused into the fine sweep: adds the correction's
// share of r.z to sc->rz_part and finalises beta (D.K >= 1, D.K <= the
// reduction scratch's kMaxRedValues * kMaxRedBlocks partials).
template <typename T>
void launch_defl_apply_rz(const Defl& D, const T* r, T* z, KScal* sc, const RedScratch& rs, cudaStream_t st);

// PCG: beta = r.z / r.z_prev (0 on a pass's first iteration), keep r.z;
// a non-positive or non-finite r.z ends the pass as a breakdown.
__device__ __forceinline__ void fin_pcg_beta(KScal* sc, double rz) {
  sc->beta = (sc->iters == 0) ? 0.0 : rz / sc->rz;
  sc->rz = rz;
  if (!(rz > 0.0) || !isfinite(rz)) {
    sc->breakdown = 1;
    sc->done = 1;
  }
}

// Device-side record of one solve when the loops run inside a CUDA graph.
struct SolveStats {
  double relres;  // last scaled relative residual
  int iters;      // inner Krylov iterations (summed over passes)
  int outer;      // refinement passes
  int converged;
  int zero;       // right-hand side was zero: x set to 0
  int started;    // an inner pass has been initialised
  int pad;
};

struct SolveResult {
  int iters;      // total inner Krylov iterations
  int outer;      // refinement passes
  double relres;  // final true scaled residual ||D^-1 (b - A x)|| / ||D^-1 b||
  int converged;
  int net_iters;  // of which flexible-CG iterations with the learned preconditioner
  int fallback;   // 1 if the learned preconditioner stagnated and MG-PCG finished
};

// Host-side driver: outer FP64 refinement around an inner solve in T.
// op64: fine operator in FP64 (for the true residual); h: hierarchy in T
// (level 0 is the same operator in T); b: right-hand side (box layout);
// x: solution view (initial guess on entry).  sym selects PCG or BiCGStab;
// use_mg selects the multigrid V-cycle (else the diagonal) preconditioner
// for PCG (BiCGStab always uses multigrid).
// Double-FP32 copies of a symmetric system for the refinement residual of
// the mixed path (each value v as float hi + lo, see df_split): the
// operator's diagonal and plus links in the z view, the right-hand side and
// the current solution, in the solve box's flat layout.
struct DFBuf {
  float2 *dg, *xp, *yp, *zp, *b, *x;
};
struct SolverWork;  // opaque: Krylov vectors + scalars
template <typename T>
SolveResult solve(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, double rtol,
                  int max_iter, SolverWork* w, const RedScratch& rs, cudaStream_t st, bool use_mg);

template <typename T>
void build_coarse_levels(Hier<T>& h, cudaStream_t st);

// MG-PCG residual snapshots of A e = b (training data of the learned
// preconditioner); see vos_pressure_snapshots.
template <typename T>
int residual_snapshots(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, SolverWork* w,
                       const RedScratch& rs, cudaStream_t st, int count, const int* iters, float* out);

// Layout helpers for allocation.
template <typename T>
size_t hier_bytes(Box fine, int sym, bool share_level0);
size_t op64_bytes(Box b, int sym);
void op64_carve(Op<double>& A, Box b, int sym, char*& cursor);
extern int g_num_sms;
template <typename T>
void hier_carve(Hier<T>& h, Box fine, int sym, char*& cursor, const MGParams& mg, bool share_level0,
                const Op<double>* op64);

// Enqueue a whole solve on a stream that is being captured into a CUDA
// graph: the refinement loop and the Krylov loop become conditional WHILE
// nodes driven by device-side controller kernels (no host round trip).
// Bodies are captured on s1 (outer) and s2 (inner).  Results in *ss.
template <typename T>
cudaError_t solve_capture(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, double rtol,
                          int max_iter, SolverWork* w, const RedScratch& rs, cudaStream_t st, bool use_mg,
                          SolveStats* ss, cudaStream_t s1, cudaStream_t s2);

// Tile autotuner: time the Jacobi sweep of every level of h with at least
// 2^16 cells over a fixed set of tile shapes / z chunks and keep the fastest
// per (box, operand type, symmetry) for all later stencil launches of the
// process.  Uses the Krylov vectors of w as scratch; synchronises st.
template <typename T>
void autotune_hier(const Hier<T>& h, SolverWork* w, cudaStream_t st);
// The tuned tile of a box, if any: returns 1 and fills (tx, ty, zc).
int tuned_config(int mx, int my, int mz, int tsize, int sym, int* tx, int* ty, int* zc);
// The sweep shape of a box the autotuner did not measure.
void default_sweep_config(int mx, int my, int mz, int* tx, int* ty, int* zc);

// Learned preconditioner (vos_unet.cu): z = UNet(r / rms(r), eps) rms(r),
// rr = |r|^2 on the device.
template <typename T>
void unet_precond(vos_unet* net, const T* r, T* z, const double* rr, cudaStream_t st);
// Accessors of a handle (vos_capi.cu): the FP64 pressure operator of the
// last step and the fluid fraction.
const Op<double>* handle_pressure_op(vos_handle* h);
const double* handle_eps(vos_handle* h);

size_t solver_work_bytes(long long max_cells);
SolverWork* solver_work_carve(char*& cursor, long long max_cells);
void solver_work_free(SolverWork* w);

// Error check helper
#define VOS_CUDA_TRY(expr)                       \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return _e;            \
  } while (0)

}  // namespace vos
