// Cluster-resident coarse part of the multigrid V-cycle.
//
// On the coarse levels of a hierarchy (here: every level from the first one
// with at most kTailMaxCells cells down to the coarsest) each smoothing
// sweep, residual, restriction and prolongation touches a few thousand to a
// few tens of thousands of cells: as separate kernel launches they are
// bound by launch latency and by the latency of their loads, not by
// bandwidth (about 22 launches per V-cycle on a 256^3 grid).  Here all of
// them run in ONE launch of one thread-block cluster of kTailCTAs CTAs:
//   * every tail level's operator (diag, omega/diag, links) and its three
//     vectors (b, x, t) live in distributed shared memory: CTA r holds the
//     cells [r * chunk, (r + 1) * chunk) of the level in x-fastest order
//     (the coarsest level, at most kThreads cells, sits in CTA 0);
//   * a stencil reads a neighbour held by another CTA of the cluster through
//     its mapped shared-memory address (DSMEM);
//   * the phases (first sweep, sweeps, residual, restriction, coarse solve,
//     prolongation, sweeps) are separated by cluster barriers, which are
//     hardware barriers: no CTA of the cluster can be missing, since the
//     cluster is co-scheduled and every thread passes every barrier (the
//     only early exit, a finished solve, is taken by all threads before the
//     first barrier).
// Each cell is updated with the same arithmetic, in the same order, as the
// separate sweep (k_stencil, k_jac0), restriction (k_restrict_sum),
// prolongation (k_prolong_add) and coarsest-level (k_coarse_solve) kernels,
// so the cycle's result is bit-identical to the multi-launch one.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "vos_internal.cuh"

namespace cg = cooperative_groups;

namespace vos {

static __device__ unsigned long long vos_exec_count = 0;
unsigned long long exec_count_mgtail() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}

namespace {

constexpr int kTailCTAs = 8;         // CTAs per cluster (the portable maximum)
constexpr int kTailThreads = 1024;   // threads per CTA
constexpr int kTailMaxLev = 8;
constexpr long long kTailMaxCells = 32768;  // largest level in the tail (32^3)
constexpr int kTailSmemMax = 200 * 1024;    // shared memory per CTA (of 227 KB)
constexpr int kNoArr = -1;
enum TArr { TA_DIAG = 0, TA_DINV, TA_XP, TA_YP, TA_ZP, TA_XM, TA_YM, TA_ZM, TA_B, TA_X, TA_T, TA_COUNT };

template <typename T>
struct TailLev {
  int mx, my, mz;
  int n;      // cells
  int chunk;  // cells per CTA (the coarsest level: n, all in CTA 0)
  int off[TA_COUNT];  // byte offset of each array in shared memory (kNoArr: absent)
  const T* g[TA_ZM + 1];  // the level's operator in global memory
};

template <typename T>
struct TailArgs {
  int nlev;  // tail levels, the last one the coarsest (>= 2)
  int nu, coarse_sweeps;
  T omega, wc;
  const T* b0;  // right-hand side of the first tail level (global)
  T* x0;        // result of the first tail level (global)
  const KScal* sc;
  TailLev<T> lev[kTailMaxLev];
};

// Access to one tail level's arrays in the cluster: a cell this CTA holds is
// read from its own shared memory (a compare and a shared load); any other
// cell from the holding CTA's shared memory through its mapped address.
template <typename T>
struct Acc {
  const TailLev<T>* L;
  char* smem;
  char* const* peer;  // shared-memory base of every CTA (generic addresses)
  int c0;             // first cell held by this CTA
  __device__ __forceinline__ T get(int arr, int c) const {
    const unsigned o = (unsigned)(c - c0);
    if (o < (unsigned)L->chunk) return reinterpret_cast<const T*>(smem + L->off[arr])[o];
    const int r = c / L->chunk;
    return reinterpret_cast<const T*>(peer[r] + L->off[arr])[c - r * L->chunk];
  }
  __device__ __forceinline__ T* loc(int arr) const { return reinterpret_cast<T*>(smem + L->off[arr]); }
};

template <typename T>
__device__ __forceinline__ T jac_weight(T omega, T d, T dinv) {
  if constexpr (sizeof(T) == 4)
    return __fdividef(omega, d);  // as k_stencil / k_jac0 in FP32
  else
    return dinv;
}

// (A v)_c at cell c = (i, j, k) of the level, v given by vf(c, i, j, k)
// (same term order as k_stencil; an absent z link adds nothing).
template <typename T, bool SYM, class VF>
__device__ __forceinline__ T tail_ax(const Acc<T>& A, int c, int i, int j, int k, T vc, T d, VF vf) {
  const TailLev<T>& L = *A.L;
  const int sy = L.mx, sz = L.mx * L.my;
  T ax = rn_mul(d, vc);
  if (i + 1 < L.mx) ax = fma(A.get(TA_XP, c), vf(c + 1, i + 1, j, k), ax);
  if (i > 0) ax = fma((SYM ? A.get(TA_XP, c - 1) : A.get(TA_XM, c)), vf(c - 1, i - 1, j, k), ax);
  if (j + 1 < L.my) ax = fma(A.get(TA_YP, c), vf(c + sy, i, j + 1, k), ax);
  if (j > 0) ax = fma((SYM ? A.get(TA_YP, c - sy) : A.get(TA_YM, c)), vf(c - sy, i, j - 1, k), ax);
  if (L.mz > 1) {
    if (k + 1 < L.mz) ax = fma(A.get(TA_ZP, c), vf(c + sz, i, j, k + 1), ax);
    if (k > 0) ax = fma((SYM ? A.get(TA_ZP, c - sz) : A.get(TA_ZM, c)), vf(c - sz, i, j, k - 1), ax);
  }
  return ax;
}

template <typename T>
__device__ __forceinline__ void cell_ijk(const TailLev<T>& L, int c, int& i, int& j, int& k) {
  const int q = c / L.mx;
  i = c - q * L.mx;
  k = q / L.my;
  j = q - k * L.my;
}

template <typename T, bool SYM>
__global__ void __launch_bounds__(kTailThreads) k_mg_tail(TailArgs<T> a) {
  VOS_COUNT_EXEC();
  if (a.sc != nullptr && a.sc->done) return;  // uniform: every thread of every CTA leaves here
  extern __shared__ __align__(16) char smem[];
  __shared__ char* s_peer[kTailCTAs];
  __shared__ int pre[kTailMaxLev];  // buffer (TA_X / TA_T) holding level l's pre-smoothed iterate
  __shared__ int fin[kTailMaxLev];  // buffer holding level l's result
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  if (tid < kTailCTAs) s_peer[tid] = cl.map_shared_rank(smem, tid);
  auto acc = [&](int l) {
    const TailLev<T>& L = a.lev[l];
    return Acc<T>{&L, smem, s_peer, rank * L.chunk};
  };
  auto own_end = [&](const TailLev<T>& L) { return min(rank * L.chunk + L.chunk, L.n); };

  // load the operators of every tail level and the first level's b
  for (int l = 0; l < a.nlev; ++l) {
    const TailLev<T>& L = a.lev[l];
    const int c0 = rank * L.chunk, c1 = own_end(L);
    for (int arr = TA_DIAG; arr <= TA_ZM; ++arr) {
      if (L.off[arr] == kNoArr) continue;
      T* dst = reinterpret_cast<T*>(smem + L.off[arr]);
      const T* src = L.g[arr];
      for (int c = c0 + tid; c < c1; c += kTailThreads) dst[c - c0] = __ldg(src + c);
    }
    if (l == 0) {
      T* dst = reinterpret_cast<T*>(smem + L.off[TA_B]);
      for (int c = c0 + tid; c < c1; c += kTailThreads) dst[c - c0] = __ldcg(a.b0 + c);
    }
  }
  cl.sync();

  const int nu = a.nu < 1 ? 1 : a.nu;
  const T om = a.omega, wc = a.wc;
  // one damped Jacobi sweep of level l from buffer `cur` into buffer `out`
  auto sweep = [&](int l, int cur, int out) {
    const Acc<T> A = acc(l);
    const TailLev<T>& L = a.lev[l];
    const int c0 = A.c0, c1 = own_end(L);
    T* o = A.loc(out);
    const T *bl = A.loc(TA_B), *dg = A.loc(TA_DIAG), *dv = A.loc(TA_DINV), *v = A.loc(cur);
    auto vf = [&](int c, int, int, int) { return A.get(cur, c); };
    for (int c = c0 + tid; c < c1; c += kTailThreads) {
      int i, j, k;
      cell_ijk(L, c, i, j, k);
      const T d = dg[c - c0], vc = v[c - c0];
      const T ax = tail_ax<T, SYM>(A, c, i, j, k, vc, d, vf);
      o[c - c0] = fma(jac_weight(om, d, dv[c - c0]), bl[c - c0] - ax, vc);
    }
  };
  // ---- down: pre-smoothing, residual and restriction
  for (int l = 0; l + 1 < a.nlev; ++l) {
    const Acc<T> A = acc(l);
    const TailLev<T>& L = a.lev[l];
    const int c0 = A.c0, c1 = own_end(L);
    const T *bl = A.loc(TA_B), *dg = A.loc(TA_DIAG), *dv = A.loc(TA_DINV);
    int cur;
    if (nu >= 2) {
      // the first two sweeps in one phase: the first (from zero, x = w b)
      // is evaluated wherever the second reads it
      T* o = A.loc(TA_X);
      auto x0 = [&](int c, int, int, int) {
        return jac_weight(om, A.get(TA_DIAG, c), A.get(TA_DINV, c)) * A.get(TA_B, c);
      };
      for (int c = c0 + tid; c < c1; c += kTailThreads) {
        int i, j, k;
        cell_ijk(L, c, i, j, k);
        const T d = dg[c - c0];
        const T w = jac_weight(om, d, dv[c - c0]);
        const T vc = w * bl[c - c0];
        const T ax = tail_ax<T, SYM>(A, c, i, j, k, vc, d, x0);
        o[c - c0] = fma(w, bl[c - c0] - ax, vc);
      }
      cur = TA_X;
      cl.sync();
      for (int s = 2; s < nu; ++s) {
        const int out = (cur == TA_X) ? TA_T : TA_X;
        sweep(l, cur, out);
        cl.sync();
        cur = out;
      }
    } else {
      T* o = A.loc(TA_T);
      for (int c = c0 + tid; c < c1; c += kTailThreads) o[c - c0] = jac_weight(om, dg[c - c0], dv[c - c0]) * bl[c - c0];
      cur = TA_T;
      cl.sync();
    }
    if (tid == 0) pre[l] = cur;  // read after later barriers
    {  // residual b - A x of the children, summed into the next level's b
      const TailLev<T>& C = a.lev[l + 1];
      const Acc<T> AC = acc(l + 1);
      const int k0 = AC.c0, k1 = own_end(C);
      T* bc = AC.loc(TA_B);
      auto xv = [&](int c, int, int, int) { return A.get(cur, c); };
      const int ni = L.mx > 1 ? 2 : 1, nj = L.my > 1 ? 2 : 1, nk = L.mz > 1 ? 2 : 1;
      for (int q = k0 + tid; q < k1; q += kTailThreads) {
        int I, J, K;
        cell_ijk(C, q, I, J, K);
        T sum = 0;
        for (int dk = 0; dk < nk; ++dk) {
          const int k = (L.mz > 1) ? 2 * K + dk : 0;
          if (k >= L.mz) continue;
          for (int dj = 0; dj < nj; ++dj) {
            const int j = (L.my > 1) ? 2 * J + dj : 0;
            if (j >= L.my) continue;
            const int row = L.mx * (j + L.my * k);
            for (int di = 0; di < ni; ++di) {
              const int i = (L.mx > 1) ? 2 * I + di : 0;
              if (i >= L.mx) continue;
              const int c = row + i;
              const T ax = tail_ax<T, SYM>(A, c, i, j, k, A.get(cur, c), A.get(TA_DIAG, c), xv);
              sum += A.get(TA_B, c) - ax;
            }
          }
        }
        bc[q - k0] = sum;
      }
    }
    cl.sync();
  }
  // ---- coarsest level: damped Jacobi sweeps from zero in CTA 0 (as k_coarse_solve)
  {
    const int lc = a.nlev - 1;
    const TailLev<T>& L = a.lev[lc];
    const Acc<T> A = acc(lc);
    const int ns = a.coarse_sweeps;
    if (rank == 0) {
      T* bufs[2] = {A.loc(TA_X), A.loc(TA_T)};
      const int c = tid;
      const bool in = c < L.n;
      int i = 0, j = 0, k = 0;
      if (in) cell_ijk(L, c, i, j, k);
      const T bc = in ? A.loc(TA_B)[c] : T(0);
      const T w = in ? A.loc(TA_DINV)[c] : T(0);
      const T dd = in ? A.loc(TA_DIAG)[c] : T(0);
      if (in) bufs[0][c] = w * bc;
      __syncthreads();
      int cb = 0;
      for (int it = 1; it < ns; ++it) {
        if (in) {
          const T* v = bufs[cb];
          auto vf = [&](int cc, int, int, int) { return v[cc]; };
          const T ax = tail_ax<T, SYM>(A, c, i, j, k, v[c], dd, vf);
          bufs[cb ^ 1][c] = fma(w, bc - ax, v[c]);
        }
        __syncthreads();
        cb ^= 1;
      }
    }
    // every CTA needs to know the buffer: the sweep count fixes it
    if (tid == 0) fin[lc] = (((ns > 1 ? ns - 1 : 0) % 2) == 0) ? TA_X : TA_T;
  }
  cl.sync();
  // ---- up: prolongation and post-smoothing
  for (int l = a.nlev - 2; l >= 0; --l) {
    const Acc<T> A = acc(l);
    const Acc<T> AC = acc(l + 1);
    const TailLev<T>& L = a.lev[l];
    const TailLev<T>& C = a.lev[l + 1];
    const int c0 = A.c0, c1 = own_end(L);
    const int cur = pre[l];
    const int oth = (cur == TA_X) ? TA_T : TA_X;
    const int ec = fin[l + 1];
    {  // coarse correction x += wc e(parent) evaluated wherever the first post-sweep reads x
      auto xp = [&](int c, int i, int j, int k) {
        const int pc = (i >> 1) + C.mx * ((j >> 1) + C.my * (k >> 1));
        return fma(wc, AC.get(ec, pc), A.get(cur, c));
      };
      T* o = A.loc(oth);
      const T *bl = A.loc(TA_B), *dg = A.loc(TA_DIAG), *dv = A.loc(TA_DINV);
      for (int c = c0 + tid; c < c1; c += kTailThreads) {
        int i, j, k;
        cell_ijk(L, c, i, j, k);
        const T d = dg[c - c0];
        const T vc = xp(c, i, j, k);
        const T ax = tail_ax<T, SYM>(A, c, i, j, k, vc, d, xp);
        o[c - c0] = fma(jac_weight(om, d, dv[c - c0]), bl[c - c0] - ax, vc);
      }
    }
    cl.sync();
    int r = oth;
    for (int s = 1; s < nu; ++s) {
      const int out = (r == TA_X) ? TA_T : TA_X;
      sweep(l, r, out);
      cl.sync();
      r = out;
    }
    if (tid == 0) fin[l] = r;
    __syncthreads();
  }
  {  // the first tail level's result to global memory (own cells; no remote
     // access follows the last barrier)
    const TailLev<T>& L = a.lev[0];
    const int c0 = rank * L.chunk, c1 = own_end(L);
    const T* v = reinterpret_cast<const T*>(smem + L.off[fin[0]]);
    for (int c = c0 + tid; c < c1; c += kTailThreads) a.x0[c] = v[c - c0];
  }
}

}  // namespace

namespace {
std::mutex g_attr_mu;
bool g_attr_done[2][2] = {};

template <typename T, bool SYM>
bool ensure_attr(size_t smem) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  bool& done = g_attr_done[sizeof(T) == 8][SYM];
  if (!done) {
    if (cudaFuncSetAttribute(k_mg_tail<T, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemMax) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    done = true;
  }
  return smem <= (size_t)kTailSmemMax;
}

}  // namespace

// Off by default: measured on the 256^3 rock (mixed path, graph replay) the
// cluster launch takes about 94 us per V-cycle against about 50 us for the
// 22 graph-replayed launches it replaces (step 114.0 vs 110.1 ms).  Timing
// every phase inside the kernel showed why: a phase with almost no work still
// costs about 2 us (the cluster barrier across 8 SMs), as much as a kernel
// node of a graph, and 8 SMs have too little issue bandwidth for the 32^3
// level (7-9 us per phase there).
bool g_tail_enabled = false;

// Shared-memory layout of the tail starting at level ls: per level, its
// operator arrays and b, x, t, each `chunk` values rounded up to 16 bytes.
template <typename T>
static size_t tail_layout(const Hier<T>& h, int ls, TailArgs<T>* a) {
  size_t off = 0;
  auto take = [&](int n) {
    size_t o = off;
    off += ((size_t)n * sizeof(T) + 15) & ~(size_t)15;
    return (int)o;
  };
  for (int l = ls; l < h.nlev; ++l) {
    const Op<T>& A = h.lev[l].op;
    TailLev<T> L;
    L.mx = A.box.mx;
    L.my = A.box.my;
    L.mz = A.box.mz;
    L.n = (int)box_cells(A.box);
    L.chunk = (l == h.nlev - 1) ? L.n : (L.n + kTailCTAs - 1) / kTailCTAs;
    const T* src[TA_ZM + 1] = {A.diag, A.dinv, A.xp, A.yp, A.zp, A.xm, A.ym, A.zm};
    for (int arr = 0; arr < TA_COUNT; ++arr) L.off[arr] = kNoArr;
    for (int arr = TA_DIAG; arr <= TA_ZM; ++arr) {
      L.g[arr] = src[arr];
      if (src[arr]) L.off[arr] = take(L.chunk);
    }
    L.off[TA_B] = take(L.chunk);
    L.off[TA_X] = take(L.chunk);
    L.off[TA_T] = take(L.chunk);
    if (a) a->lev[l - ls] = L;
  }
  return off;
}

// First level of h run by the cluster-resident tail (h.nlev: none).  The
// tail starts at the largest level l >= 1 with at most kTailMaxCells cells
// whose levels l..nlev-1 fit the shared memory of the cluster, and it needs
// at least one level above the coarsest.
template <typename T>
int tail_plan(const Hier<T>& h) {
  if (!g_tail_enabled || h.nlev < 3) return h.nlev;
  if (box_cells(h.lev[h.nlev - 1].op.box) > kThreads) return h.nlev;
  for (int l = 1; l + 1 < h.nlev; ++l) {
    if (h.nlev - l > kTailMaxLev) continue;
    if (box_cells(h.lev[l].op.box) > kTailMaxCells) continue;
    if (tail_layout<T>(h, l, nullptr) <= (size_t)kTailSmemMax) return l;
  }
  return h.nlev;
}
template int tail_plan<double>(const Hier<double>&);
template int tail_plan<float>(const Hier<float>&);

// One launch: levels ls..nlev-1 of the V-cycle, from lev[ls].b to lev[ls].x.
template <typename T, bool SYM>
void tail_launch(Hier<T>& h, int ls, const KScal* sc, cudaStream_t st) {
  TailArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.nlev = h.nlev - ls;
  a.nu = h.mg.nu;
  a.coarse_sweeps = h.mg.coarse_sweeps;
  a.omega = (T)h.mg.omega;
  a.wc = (T)h.mg.wc;
  a.b0 = h.lev[ls].b;
  a.x0 = h.lev[ls].x;
  a.sc = sc;
  const size_t smem = tail_layout<T>(h, ls, &a);
  ensure_attr<T, SYM>(smem);
  double words = 0.0;  // operator and b in, x out, per tail level
  for (int l = ls; l < h.nlev; ++l) {
    const Op<T>& A = h.lev[l].op;
    const double nop = 2.0 + (A.box.mz > 1 ? 3.0 : 2.0) * (SYM ? 1.0 : 2.0);
    words += (nop + (l == ls ? 2.0 : 0.0)) * (double)box_cells(A.box);
  }
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(kTailCTAs, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTailCTAs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  const char* name = sizeof(T) == 4 ? "mg_tail_f32_Lc" : "mg_tail_f64_Lc";
  int slot = g_prof_any ? prof_before(name, words * sizeof(T), st) : -1;
  cudaLaunchKernelEx(&cfg, k_mg_tail<T, SYM>, a);
  if (slot >= 0) prof_after(slot, st);
}
template void tail_launch<float, true>(Hier<float>&, int, const KScal*, cudaStream_t);
template void tail_launch<float, false>(Hier<float>&, int, const KScal*, cudaStream_t);
template void tail_launch<double, true>(Hier<double>&, int, const KScal*, cudaStream_t);
template void tail_launch<double, false>(Hier<double>&, int, const KScal*, cudaStream_t);

// Can a cluster of kTailCTAs CTAs with `smem` bytes each run on this device
// (checked once per process and size class; false disables the tail).
template <typename T, bool SYM>
bool tail_supported(size_t smem) {
  if (!ensure_attr<T, SYM>(smem)) return false;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(kTailCTAs, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTailCTAs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_tail<T, SYM>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters > 0;
}
template bool tail_supported<float, true>(size_t);
template bool tail_supported<float, false>(size_t);
template bool tail_supported<double, true>(size_t);
template bool tail_supported<double, false>(size_t);

template <typename T>
size_t tail_smem(const Hier<T>& h, int ls) {
  return tail_layout<T>(h, ls, nullptr);
}
template size_t tail_smem<double>(const Hier<double>&, int);
template size_t tail_smem<float>(const Hier<float>&, int);

}  // namespace vos
