// Deflation of floating pore clusters for the pressure correction (a solver
// aid, not part of the paper's method).
//
// In the pressure operator div(eps_f grad) with eps_f the arithmetic face
// mean, a pore pocket that touches the connected pore network only through
// solid (eps = eps_min) has links of order eps_min to the outside and of
// order 1 inside.  Its mean pressure is then a near-null mode of the
// operator: Jacobi smoothing leaves it alone and the 2x2x2 aggregation
// hierarchy, whose aggregates straddle the pocket wall, sees it only weakly,
// so each such pocket costs Krylov iterations.  The preconditioner adds the
// exact coarse correction of those modes (see Defl in vos_internal.cuh):
//   z = V(r) + W E^-1 W^T r,   E_kk = 1_k^T A 1_k.
// Labels are computed on the host when the geometry is set (create,
// set_fields with eps); E is recomputed on the device from the assembled
// FP64 operator every step, so the correction stays exact for the current
// operator while the solid dissolves.  A stale label set (a pocket that has
// since opened) still gives an SPD preconditioner.
#include <cstdint>
#include <cstring>
#include <vector>

#include "vos_internal.cuh"

namespace vos {

static __device__ unsigned long long vos_exec_count = 0;
unsigned long long exec_count_deflate() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}

// ---------------------------------------------------------------------------
// Host labeling (union-find over strong faces)
// ---------------------------------------------------------------------------
namespace {

struct DisjointSets {
  std::vector<int32_t> parent;
  explicit DisjointSets(long long n) : parent((size_t)n) {
    for (long long i = 0; i < n; ++i) parent[(size_t)i] = (int32_t)i;
  }
  int32_t find(int32_t a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];  // path halving
      a = parent[a];
    }
    return a;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b)  // smaller index becomes the root: labels independent of visit order
      parent[b] = a;
    else
      parent[a] = b;
  }
};

}  // namespace

int floating_clusters(const double* eps, int nx, int ny, int nz, double theta, std::vector<int>& ptr,
                      std::vector<unsigned long long>& ent, int32_t* label) {
  const long long N = (long long)nx * ny * nz;
  const long long sy = nx, sz = (long long)nx * ny;
  DisjointSets ds(N);
  auto strong = [&](long long a, long long b) { return 0.5 * (eps[a] + eps[b]) >= theta; };
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long long c = i + sy * j + sz * k;
        if (i + 1 < nx && strong(c, c + 1)) ds.unite((int32_t)c, (int32_t)(c + 1));
        if (j + 1 < ny && strong(c, c + sy)) ds.unite((int32_t)c, (int32_t)(c + sy));
        if (k + 1 < nz && strong(c, c + sz)) ds.unite((int32_t)c, (int32_t)(c + sz));
      }
  // root of each cell; component sizes and outlet contact per root
  std::vector<int32_t> root((size_t)N);
  std::vector<int32_t> size((size_t)N, 0);
  std::vector<uint8_t> anchored((size_t)N, 0);
  for (long long c = 0; c < N; ++c) {
    const int32_t r = ds.find((int32_t)c);
    root[(size_t)c] = r;
    size[(size_t)r] += 1;
    if ((int)(c % nx) == nx - 1) anchored[(size_t)r] = 1;
  }
  // cluster ids in order of their first (smallest) cell
  std::vector<int32_t> id((size_t)N, -1);
  int K = 0;
  for (long long c = 0; c < N; ++c) {
    const int32_t r = root[(size_t)c];
    if (r == (int32_t)c && size[(size_t)r] >= 2 && !anchored[(size_t)r]) id[(size_t)r] = K++;
  }
  ptr.assign((size_t)K + 1, 0);
  for (long long c = 0; c < N; ++c) {
    const int32_t q = id[(size_t)root[(size_t)c]];
    if (q >= 0) ptr[(size_t)q + 1] += 1;
  }
  for (int q = 0; q < K; ++q) ptr[(size_t)q + 1] += ptr[(size_t)q];
  ent.assign((size_t)ptr[(size_t)K], 0ull);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long long c = i + sy * j + sz * k;
        const int32_t r = root[(size_t)c];
        const int32_t q = id[(size_t)r];
        if (label) label[c] = q;
        if (q < 0) continue;
        unsigned long long m = 0;
        if (i > 0 && root[(size_t)(c - 1)] == r) m |= 1ull;
        if (i + 1 < nx && root[(size_t)(c + 1)] == r) m |= 2ull;
        if (j > 0 && root[(size_t)(c - sy)] == r) m |= 4ull;
        if (j + 1 < ny && root[(size_t)(c + sy)] == r) m |= 8ull;
        if (k > 0 && root[(size_t)(c - sz)] == r) m |= 16ull;
        if (k + 1 < nz && root[(size_t)(c + sz)] == r) m |= 32ull;
        ent[(size_t)fill[(size_t)q]++] = (unsigned long long)c | (m << kDeflMaskShift);
      }
  return K;
}

// ---------------------------------------------------------------------------
// Device kernels: one block per cluster, fixed summation order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_defl_energy(Defl D, Op<double> A) {
  VOS_COUNT_EXEC();
  const int q = blockIdx.x;
  const long long sy = A.box.mx, sz = (long long)A.box.mx * A.box.my;
  double v[1] = {0.0};
  for (int e = D.ptr[q] + threadIdx.x; e < D.ptr[q + 1]; e += kThreads) {
    const unsigned long long w = D.ent[e];
    const long long c = (long long)(w & kDeflCellMask);
    const unsigned m = (unsigned)(w >> kDeflMaskShift);
    // row sum of A over the cluster's columns: diag + links to member cells
    double s = A.diag[c];
    if (m & 1u) s += A.xp[c - 1];
    if (m & 2u) s += A.xp[c];
    if (m & 4u) s += A.yp[c - sy];
    if (m & 8u) s += A.yp[c];
    if (m & 16u) s += A.zp[c - sz];
    if (m & 32u) s += A.zp[c];
    v[0] += s;
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) D.Einv[q] = (v[0] > 0.0) ? 1.0 / v[0] : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_defl_apply(Defl D, const T* __restrict__ r, T* __restrict__ z,
                                                        const KScal* sc) {
  VOS_COUNT_EXEC();
  if (sc != nullptr && sc->done) return;
  const int q = blockIdx.x;
  const int b = D.ptr[q], e = D.ptr[q + 1];
  double v[1] = {0.0};
  for (int t = b + threadIdx.x; t < e; t += kThreads) v[0] += (double)r[D.ent[t] & kDeflCellMask];
  block_sum<1>(v);
  __shared__ double s_add;
  if (threadIdx.x == 0) s_add = v[0] * D.Einv[q];
  __syncthreads();
  const T add = (T)s_add;
  for (int t = b + threadIdx.x; t < e; t += kThreads) z[D.ent[t] & kDeflCellMask] += add;
}

// The same, also completing r.z for PCG: the fine sweep that produced z
// stored sum r.z_mg in sc->rz_part; cluster q adds add_q (sum over its cells
// of r), the change of r.z its correction makes, into partials[q], and the
// last block to finish adds those in cluster order and finalises beta.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_defl_apply_rz(Defl D, const T* __restrict__ r, T* __restrict__ z,
                                                           KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  if (sc->done) return;  // the same for every block of the launch
  const int q = blockIdx.x;
  const int b = D.ptr[q], e = D.ptr[q + 1];
  double v[1] = {0.0};
  for (int t = b + threadIdx.x; t < e; t += kThreads) v[0] += (double)r[D.ent[t] & kDeflCellMask];
  block_sum<1>(v);
  __shared__ double s_add;
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_add = v[0] * D.Einv[q];
  __syncthreads();
  const T add = (T)s_add;
  for (int t = b + threadIdx.x; t < e; t += kThreads) z[D.ent[t] & kDeflCellMask] += add;
  if (threadIdx.x == 0) {
    rs.partials[q] = (double)add * v[0];
    __threadfence();
    s_last = atomicAdd(rs.counter, 1u) == (unsigned)D.K - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double c[1] = {0.0};
  for (int t = threadIdx.x; t < D.K; t += kThreads) c[0] += __ldcg(rs.partials + t);
  block_sum<1>(c);
  if (threadIdx.x == 0) {
    *rs.counter = 0u;
    fin_pcg_beta(sc, sc->rz_part + c[0]);
  }
}

template <typename T>
void launch_defl_apply_rz(const Defl& D, const T* r, T* z, KScal* sc, const RedScratch& rs, cudaStream_t st) {
  vlaunch("defl_apply", 0.0, k_defl_apply_rz<T>, D.K, kThreads, st, D, r, z, sc, rs);
}
template void launch_defl_apply_rz<float>(const Defl&, const float*, float*, KScal*, const RedScratch&, cudaStream_t);

void launch_defl_energy(const Defl& D, const Op<double>& A, cudaStream_t st) {
  if (D.K <= 0) return;
  vlaunch("defl_energy", 0.0, k_defl_energy, D.K, kThreads, st, D, A);
}

template <typename T>
void launch_defl_apply(const Defl& D, const T* r, T* z, const KScal* sc, cudaStream_t st) {
  if (D.K <= 0) return;
  vlaunch("defl_apply", 0.0, k_defl_apply<T>, D.K, kThreads, st, D, r, z, sc);
}
template void launch_defl_apply<float>(const Defl&, const float*, float*, const KScal*, cudaStream_t);
template void launch_defl_apply<double>(const Defl&, const double*, double*, const KScal*, cudaStream_t);

}  // namespace vos
