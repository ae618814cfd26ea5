// Linear solvers of the VoS step: geometric multigrid (Jacobi smoothing,
// Galerkin coarse operators with piecewise-constant transfer) as the
// preconditioner of CG (symmetric systems: momentum, pressure, VoS-psi
// transport) or BiCGStab (iVoS transport), inside an FP64 refinement loop
// that recomputes the true residual b - A x in FP64.  The inner solve runs
// in T = double (FP64 path) or T = float (mixed path); dot products and
// norms are always accumulated in FP64 with deterministic reductions.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "vos_internal.cuh"

namespace vos {

// Kernel executions of this file (see VOS_COUNT_EXEC).
static __device__ unsigned long long vos_exec_count = 0;
unsigned long long exec_count_solver() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}


int g_num_sms = 152;
constexpr double kDiagFloor32 = 2e-5;

__host__ int grid_for(Box b, int max_blocks) {
  Seg s = make_seg(b);
  long long need = (s.nseg + kWarps - 1) / kWarps;
  long long cap = (long long)g_num_sms * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;  // reduction scratch holds kMaxRedBlocks partials
  if (max_blocks > 0 && cap > max_blocks) cap = max_blocks;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

struct SolverWork {
  long long cap;
  void *r, *z, *p, *p2, *q, *e, *rh, *v, *s, *t, *ph, *sh;
  DFBuf df;         // double-FP32 copies for the refinement residual (mixed path)
  int* dfbad;       // device: 1 once a value did not fit the double-FP32 form
  KScal* sc;        // device
  KScal* sc_host;   // pinned
  double* outer;    // device [|D^-1 r|^2, |D^-1 b|^2, |r|^2]
  double* outer_host;
};

// ---------------------------------------------------------------------------
// Stencil application
// ---------------------------------------------------------------------------
template <typename T, bool SYM, typename F>
__device__ __forceinline__ T stencil(const Op<T>& A, int i, int j, int k, long long c, F xat) {
  const Box b = A.box;
  T y = rn_mul(A.diag[c], xat(c, i, j, k));
  if (i + 1 < b.mx) y = fma(A.xp[c], xat(c + 1, i + 1, j, k), y);
  if (i > 0) y = fma((SYM ? A.xp[c - 1] : A.xm[c]), xat(c - 1, i - 1, j, k), y);
  const long long sy = b.mx;
  if (j + 1 < b.my) y = fma(A.yp[c], xat(c + sy, i, j + 1, k), y);
  if (j > 0) y = fma((SYM ? A.yp[c - sy] : A.ym[c]), xat(c - sy, i, j - 1, k), y);
  if (b.mz > 1) {
    const long long sz = (long long)b.mx * b.my;
    if (k + 1 < b.mz) y = fma(A.zp[c], xat(c + sz, i, j, k + 1), y);
    if (k > 0) y = fma((SYM ? A.zp[c - sz] : A.zm[c]), xat(c - sz, i, j, k - 1), y);
  }
  return y;
}

// Per-thread partial sums of dot products.  The FP32 inner solver
// accumulates in compensated (Kahan) FP32 and converts once per thread:
// FP64 arithmetic runs at ~1/60 of FP32 here, and a conversion plus an FP64
// FMA per element would cap the streaming kernels near 2 TB/s.  Block and
// grid reductions stay FP64 with a fixed order.
template <typename T>
struct PSum;
template <>
struct PSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct PSum<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float y = __fmul_rn(a, b) - c;
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

#define DONE_RETURN(sc) \
  if ((sc) != nullptr && (sc)->done) return;

// Names and algorithmic bytes of launches (per-kernel timing/roofline).
#define KN(base, fine) \
  ((fine) ? (sizeof(T) == 4 ? base "_f32_L0" : base "_f64_L0") : (sizeof(T) == 4 ? base "_f32_Lc" : base "_f64_Lc"))
template <typename T>
static inline double n_offs(const Op<T>& A) {
  return (A.box.mz > 1 ? 3.0 : 2.0) * (A.sym ? 1.0 : 2.0);
}
template <typename T>
static inline double ncell(const Op<T>& A) {
  return (double)box_cells(A.box);
}

// FIN codes for the fused dot of the last level-0 smoothing sweep.
enum Fin { FIN_NONE = 0, FIN_PCG_BETA = 1 };


// ---------------------------------------------------------------------------
// 2.5D stencil sweeps: a (blockDim.x x blockDim.y) tile of threads in the
// (x, y) plane marches along z over zc planes; the z-neighbours of the input
// vector and the z-link coefficient of the plane below stay in registers,
// x/y neighbours come through L1.  2D boxes are remapped to (mx, 1, my) so
// that y is the marched axis (see zview).
// val(c, i, j, k) gives the input vector at a cell (it may be computed, e.g.
// with a fused prolongation); emit(c, i, j, k, v_c, Av_c, diag_c) consumes
// the result.  Threads outside the box do nothing but stay for reductions.
// ---------------------------------------------------------------------------
template <typename T, bool SYM, class VAL, class EMIT>
__device__ __forceinline__ void zmarch(const Op<T>& A, int zc, VAL val, EMIT emit) {
  const Box bx = A.box;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  if (i >= bx.mx || j >= bx.my || k0 >= k1) return;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  // Coefficients are read-only for the kernel's lifetime (ld.global.nc), so
  // the compiler may move their loads across the stores of emit().
  const T* __restrict__ dg = A.diag;
  const T* __restrict__ xp = A.xp;
  const T* __restrict__ yp = A.yp;
  const T* __restrict__ zp = A.zp;
  long long c = i + sy * j + sz * k0;
  T v_lo = (k0 > 0) ? val(c - sz, i, j, k0 - 1) : T(0);
  T v_c = val(c, i, j, k0);
  T zl = (SYM && k0 > 0) ? __ldg(zp + c - sz) : T(0);
  for (int k = k0; k < k1; ++k, c += sz) {
    const bool up = (k + 1 < bx.mz);
    const T v_hi = up ? val(c + sz, i, j, k + 1) : T(0);
    const T d = __ldg(dg + c);
    T ax = rn_mul(d, v_c);
    if (i + 1 < bx.mx) ax = fma(__ldg(xp + c), val(c + 1, i + 1, j, k), ax);
    if (i > 0) ax = fma((SYM ? __ldg(xp + c - 1) : __ldg(A.xm + c)), val(c - 1, i - 1, j, k), ax);
    if (j + 1 < bx.my) ax = fma(__ldg(yp + c), val(c + sy, i, j + 1, k), ax);
    if (j > 0) ax = fma((SYM ? __ldg(yp + c - sy) : __ldg(A.ym + c)), val(c - sy, i, j - 1, k), ax);
    if (bx.mz > 1) {
      const T zu = up ? __ldg(zp + c) : T(0);
      ax = fma(zu, v_hi, ax);
      if (k > 0) ax = fma((SYM ? zl : __ldg(A.zm + c)), v_lo, ax);
      zl = zu;
    }
    emit(c, i, j, k, v_c, ax, d);
    v_lo = v_c;
    v_c = v_hi;
  }
}

// Pure 2.5D stencil kernels, written out explicitly (one input vector, one
// output, no epilogue): on this part a fused reduction or extra per-
// neighbour loads cost 30-60% of the bandwidth of the plain sweep, so dots,
// updates and grid transfers run as separate streaming kernels.
//   SK_JAC: out = x + (omega / diag) (b - A x)   (omega/diag in registers for
//           FP32, read from dinv for FP64)
//   SK_MV:  out = A x
//   SK_RES: out = b - A x
enum StencilKind { SK_JAC = 0, SK_MV = 1, SK_RES = 2, SK_JAC0 = 3 };

template <typename T, bool SYM, int KIND>
__global__ void __launch_bounds__(kThreads) k_stencil(Op<T> A, const T* __restrict__ b, const T* __restrict__ x,
                                                     T* __restrict__ out, T omega, int zc, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const Box bx = A.box;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  if (i >= bx.mx || j >= bx.my || k0 >= k1) return;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  const T* __restrict__ dg = A.diag;
  const T* __restrict__ xp = A.xp;
  const T* __restrict__ yp = A.yp;
  const T* __restrict__ zp = A.zp;
  const bool has_z = bx.mz > 1;
  long long c = i + sy * j + sz * k0;
  T vlo = (k0 > 0) ? __ldg(x + c - sz) : T(0);
  T vc = __ldg(x + c);
  T zl = (SYM && k0 > 0) ? __ldg(zp + c - sz) : T(0);
  for (int k = k0; k < k1; ++k, c += sz) {
    const bool up = (k + 1 < bx.mz);
    const T vhi = up ? __ldg(x + c + sz) : T(0);
    const T d = __ldg(dg + c);
    T ax = rn_mul(d, vc);
    if (i + 1 < bx.mx) ax = fma(__ldg(xp + c), __ldg(x + c + 1), ax);
    if (i > 0) ax = fma((SYM ? __ldg(xp + c - 1) : __ldg(A.xm + c)), __ldg(x + c - 1), ax);
    if (j + 1 < bx.my) ax = fma(__ldg(yp + c), __ldg(x + c + sy), ax);
    if (j > 0) ax = fma((SYM ? __ldg(yp + c - sy) : __ldg(A.ym + c)), __ldg(x + c - sy), ax);
    if (has_z) {
      const T zu = up ? __ldg(zp + c) : T(0);
      ax = fma(zu, vhi, ax);
      if (k > 0) ax = fma((SYM ? zl : __ldg(A.zm + c)), vlo, ax);
      zl = zu;
    }
    if (KIND == SK_JAC) {
      T w;
      if constexpr (sizeof(T) == 4)
        w = __fdividef(omega, d);
      else
        w = __ldg(A.dinv + c);
      out[c] = fma(w, __ldg(b + c) - ax, vc);
    } else if (KIND == SK_MV) {
      out[c] = ax;
    } else {
      out[c] = __ldg(b + c) - ax;
    }
    vlo = vc;
    vc = vhi;
  }
}

// Row arithmetic of the matrix-free FP32 pressure operator, shared by every
// kernel that applies it (one or four cells per thread, fused passes): the
// link to a neighbour n is a_cn = (e_c + e_n) s / 2, the diagonal the sum of
// the links present (plus 2 e_c s on the outlet face of the last column),
// the links taken in the order x+, x-, y+, y-, z+, z-; explicit rounding,
// so that all these kernels give identical values.
__device__ __forceinline__ float mf_outlet(float ec, float s, bool outlet) {
  return outlet ? __fmul_rn(__fmul_rn(2.0f, ec), s) : 0.0f;
}
// adds the link to a neighbour (fluid fraction en, value vn) to d and off
__device__ __forceinline__ void mf_link(float ec, float en, float vn, float hs, bool has_x, float& d, float& off) {
  const float a = __fmul_rn(__fadd_rn(ec, en), hs);
  d = __fadd_rn(d, a);
  if (has_x) off = __fmaf_rn(a, vn, off);
}
// SK_JAC0: (omega / d) b; SK_JAC: x + (omega / d)(b - A x); SK_MV: A x;
// SK_RES: b - A x (A x = d x_c - off)
template <int KIND>
__device__ __forceinline__ float mf_result(float d, float off, float vc, float bc, float omega) {
  if (KIND == SK_JAC0) return __fmul_rn(__fdividef(omega, d), bc);
  const float ax = __fmaf_rn(d, vc, -off);
  if (KIND == SK_JAC) return __fmaf_rn(__fdividef(omega, d), __fsub_rn(bc, ax), vc);
  if (KIND == SK_MV) return ax;
  return __fsub_rn(bc, ax);
}

// First Jacobi sweep from zero: x = (omega / diag) b.
// Matrix-free FP32 sweeps of the pressure operator (Op::mfe): the same z
// march as k_stencil, but the links and the diagonal are formed from the
// fluid fraction e in registers, a_cn = 0.5 (e_c + e_n) s, so a sweep reads
// one coefficient word per cell instead of four.  KIND as in k_stencil, plus
// SK_JAC0: out = (omega / diag) b (the first sweep from zero).
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_stencil_mf(Box bx, const float* __restrict__ e, float s,
                                                        const float* __restrict__ b, const float* __restrict__ x,
                                                        float* __restrict__ out, float omega, int zc, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  if (i >= bx.mx || j >= bx.my || k0 >= k1) return;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  const float hs = 0.5f * s;
  const bool has_x = KIND != SK_JAC0;
  // Registers hold planes k-1, k, k+1 of e and x; the loads of plane k+2
  // (and of b at k+1) are issued before plane k is computed, so each thread
  // keeps two planes of DRAM loads in flight.
  long long c = i + sy * j + sz * k0;
  float elo = (k0 > 0) ? __ldg(e + c - sz) : 0.0f;
  float ec = __ldg(e + c);
  float ehi = (k0 + 1 < bx.mz) ? __ldg(e + c + sz) : 0.0f;
  float vlo = (has_x && k0 > 0) ? __ldg(x + c - sz) : 0.0f;
  float vc = has_x ? __ldg(x + c) : 0.0f;
  float vhi = (has_x && k0 + 1 < bx.mz) ? __ldg(x + c + sz) : 0.0f;
  float bc = (KIND != SK_MV) ? __ldg(b + c) : 0.0f;
  for (int k = k0; k < k1; ++k, c += sz) {
    const bool up = (k + 1 < bx.mz);
    const bool up2 = (k + 2 < bx.mz) && (k + 1 < k1);
    const float e2 = up2 ? __ldg(e + c + 2 * sz) : 0.0f;
    const float v2 = (has_x && up2) ? __ldg(x + c + 2 * sz) : 0.0f;
    const float bn = (KIND != SK_MV && k + 1 < k1) ? __ldg(b + c + sz) : 0.0f;
    float d = mf_outlet(ec, s, i == bx.mx - 1);  // outlet: phi = 0 on the face
    float off = 0.0f;                              // sum over links of a_cn x_n
    if (i + 1 < bx.mx) mf_link(ec, __ldg(e + c + 1), has_x ? __ldg(x + c + 1) : 0.0f, hs, has_x, d, off);
    if (i > 0) mf_link(ec, __ldg(e + c - 1), has_x ? __ldg(x + c - 1) : 0.0f, hs, has_x, d, off);
    if (j + 1 < bx.my) mf_link(ec, __ldg(e + c + sy), has_x ? __ldg(x + c + sy) : 0.0f, hs, has_x, d, off);
    if (j > 0) mf_link(ec, __ldg(e + c - sy), has_x ? __ldg(x + c - sy) : 0.0f, hs, has_x, d, off);
    if (up) mf_link(ec, ehi, vhi, hs, has_x, d, off);
    if (k > 0) mf_link(ec, elo, vlo, hs, has_x, d, off);
    out[c] = mf_result<KIND>(d, off, vc, bc, omega);
    elo = ec;
    ec = ehi;
    ehi = e2;
    vlo = vc;
    vc = vhi;
    vhi = v2;
    bc = bn;
  }
}

// The matrix-free sweep with four consecutive x cells per thread and
// 16-byte accesses: the own, y-1 and y+1 rows of e, x and b come as float4
// (rows start on 16-byte boundaries: mx % 4 == 0 and 256-byte aligned
// arrays), the x neighbours beyond the four cells as two scalar loads, the
// z neighbours from the register march.  Four times fewer load instructions
// for the same bytes, more bytes in flight per thread.  Each cell is
// computed with the arithmetic of k_stencil_mf, term by term in the same
// order, so the two kernels give identical results.
__device__ __forceinline__ float f4get(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}
// Register march of the four-cells-per-thread sweep, shared by the sweep,
// matrix-vector and fused residual-restriction kernels so that all compute
// each cell with the same arithmetic.  XS says where the iterate x comes from:
//   XS_PLAIN: x itself;
//   XS_PRO:   the prolongated iterate x + wc * xc[parent] (the coarse
//             correction of the V-cycle, added on the fly with the FMA of
//             k_prolong_add), so the first post-smoothing sweep needs no
//             separate prolongation pass.
enum XSrc { XS_PLAIN = 0, XS_PRO = 1 };
template <int KIND, int XS>
struct Mf4March {
  static constexpr bool has_x = KIND != SK_JAC0;
  Box bx;
  const float* __restrict__ e;
  const float* __restrict__ b;
  const float* __restrict__ x;
  float s, hs, omega;
  Box cb;                        // XS_PRO: coarse box (z view)
  const float* __restrict__ xc;  // XS_PRO: coarse correction
  float wc;                      // XS_PRO: coarse weight
  int i0, j;
  long long sy, sz;
  bool hxm, hxp, hym, hyp;
  float4 elo, ec, ehi, vlo, vc, vhi, bc;

  __device__ __forceinline__ static float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  __device__ __forceinline__ long long parent(int ii, int jj, int kk) const {
    return (ii >> 1) + (long long)cb.mx * ((jj >> 1) + (long long)cb.my * (kk >> 1));
  }
  // x of cells i0..i0+3 of row (jj, kk), flat index c of cell i0 (i0 % 4 == 0:
  // parents i0/2 and i0/2 + 1)
  __device__ __forceinline__ float4 x4(long long c, int jj, int kk) const {
    float4 v = ld4(x + c);
    if (XS == XS_PRO) {
      const long long p = parent(i0, jj, kk);
      const float ca = __ldg(xc + p), cq = __ldg(xc + p + 1);
      v = make_float4(__fmaf_rn(wc, ca, v.x), __fmaf_rn(wc, ca, v.y), __fmaf_rn(wc, cq, v.z), __fmaf_rn(wc, cq, v.w));
    }
    return v;
  }
  __device__ __forceinline__ float x1(long long c, int ii, int jj, int kk) const {
    const float v = __ldg(x + c);
    if (XS == XS_PRO) return __fmaf_rn(wc, __ldg(xc + parent(ii, jj, kk)), v);
    return v;
  }
  __device__ __forceinline__ void init(int k0) {
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    sy = bx.mx;
    sz = (long long)bx.mx * bx.my;
    hs = 0.5f * s;
    hxm = i0 > 0;
    hxp = i0 + 4 < bx.mx;
    hym = j > 0;
    hyp = j + 1 < bx.my;
    const long long c = i0 + sy * j + sz * k0;
    elo = (k0 > 0) ? ld4(e + c - sz) : z4;
    ec = ld4(e + c);
    ehi = (k0 + 1 < bx.mz) ? ld4(e + c + sz) : z4;
    vlo = (has_x && k0 > 0) ? x4(c - sz, j, k0 - 1) : z4;
    vc = has_x ? x4(c, j, k0) : z4;
    vhi = (has_x && k0 + 1 < bx.mz) ? x4(c + sz, j, k0 + 1) : z4;
    bc = (KIND != SK_MV) ? ld4(b + c) : z4;
  }
  // Results of the four cells of plane k (flat index c of cell i0; k1: end of
  // the block's planes), then the march advances one plane.  Registers hold
  // planes k-1, k, k+1 of e and x; the loads of plane k+2 (and of b at k+1)
  // are issued before plane k is computed.
  __device__ __forceinline__ void plane(int k, int k1, long long c, float r[4]) {
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const bool up = (k + 1 < bx.mz);
    const bool up2 = (k + 2 < bx.mz) && (k + 1 < k1);
    const float4 e2 = up2 ? ld4(e + c + 2 * sz) : z4;
    const float4 v2 = (has_x && up2) ? x4(c + 2 * sz, j, k + 2) : z4;
    const float4 bn = (KIND != SK_MV && k + 1 < k1) ? ld4(b + c + sz) : z4;
    const float exm = hxm ? __ldg(e + c - 1) : 0.0f, exp_ = hxp ? __ldg(e + c + 4) : 0.0f;
    const float vxm = (has_x && hxm) ? x1(c - 1, i0 - 1, j, k) : 0.0f;
    const float vxp = (has_x && hxp) ? x1(c + 4, i0 + 4, j, k) : 0.0f;
    const float4 eym = hym ? ld4(e + c - sy) : z4, eyp = hyp ? ld4(e + c + sy) : z4;
    const float4 vym = (has_x && hym) ? x4(c - sy, j - 1, k) : z4, vyp = (has_x && hyp) ? x4(c + sy, j + 1, k) : z4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q;
      const float ecq = f4get(ec, q);
      float d = mf_outlet(ecq, s, i == bx.mx - 1);  // outlet: phi = 0 on the face
      float off = 0.0f;
      if (i + 1 < bx.mx)
        mf_link(ecq, q < 3 ? f4get(ec, q + 1) : exp_, q < 3 ? f4get(vc, q + 1) : vxp, hs, has_x, d, off);
      if (i > 0) mf_link(ecq, q > 0 ? f4get(ec, q - 1) : exm, q > 0 ? f4get(vc, q - 1) : vxm, hs, has_x, d, off);
      if (hyp) mf_link(ecq, f4get(eyp, q), f4get(vyp, q), hs, has_x, d, off);
      if (hym) mf_link(ecq, f4get(eym, q), f4get(vym, q), hs, has_x, d, off);
      if (up) mf_link(ecq, f4get(ehi, q), f4get(vhi, q), hs, has_x, d, off);
      if (k > 0) mf_link(ecq, f4get(elo, q), f4get(vlo, q), hs, has_x, d, off);
      r[q] = mf_result<KIND>(d, off, f4get(vc, q), f4get(bc, q), omega);
    }
    elo = ec;
    ec = ehi;
    ehi = e2;
    vlo = vc;
    vc = vhi;
    vhi = v2;
    bc = bn;
  }
};

template <int KIND, int XS>
__global__ void __launch_bounds__(kThreads, (KIND == SK_JAC0) ? 4 : 3) k_stencil_mf4(Box bx, const float* __restrict__ e, float s,
                                                         const float* __restrict__ b, const float* __restrict__ x,
                                                         float* __restrict__ out, float omega, int zc,
                                                         const KScal* sc, Box cb, const float* __restrict__ xc,
                                                         float wc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  Mf4March<KIND, XS> m;
  m.i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  m.j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  if (m.i0 >= bx.mx || m.j >= bx.my || k0 >= k1) return;
  m.bx = bx;
  m.e = e;
  m.b = b;
  m.x = x;
  m.s = s;
  m.omega = omega;
  m.cb = cb;
  m.xc = xc;
  m.wc = wc;
  m.init(k0);
  long long c = m.i0 + m.sy * m.j + m.sz * k0;
  for (int k = k0; k < k1; ++k, c += m.sz) {
    float r[4];
    m.plane(k, k1, c, r);
    *reinterpret_cast<float4*>(out + c) = make_float4(r[0], r[1], r[2], r[3]);
  }
}

// Residual of the matrix-free fine level fused with its restriction: the
// residual b - A x of each cell (the row arithmetic of the sweeps) goes
// straight into the coarse right-hand side bc[I] = sum of its children, added
// in the order of k_restrict_sum (z pair, then y pair, then x pair), so the
// result is bit-identical to the two separate passes while the fine residual
// never reaches memory.  Each thread owns 2 x 2 cells of a plane (x pair, y
// pair: one aggregate) and marches an even number of planes from an even
// plane (z pairs).
__global__ void __launch_bounds__(kThreads, 3) k_resid_restrict_mf22(Box bx, const float* __restrict__ e, float s,
                                                                 const float* __restrict__ b,
                                                                 const float* __restrict__ x, Box cb,
                                                                 float* __restrict__ bcoarse, int zc,
                                                                 const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j0 = 2 * (blockIdx.y * blockDim.y + threadIdx.y);
  const int k0 = blockIdx.z * zc;  // zc even
  const int k1 = min(k0 + zc, bx.mz);
  if (i0 >= bx.mx || j0 >= bx.my || k0 >= k1) return;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  const float hs = 0.5f * s;
  const bool row1 = j0 + 1 < bx.my;          // the pair's second row exists
  const bool hxm = i0 > 0, hxp = i0 + 2 < bx.mx;  // i0 + 1 < mx: mx is even
  const bool hym = j0 > 0, hyp = j0 + 2 < bx.my;
  const float2 z2 = make_float2(0.0f, 0.0f);
  auto ld2 = [](const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); };
  auto g2 = [](const float2& v, int q) { return q == 0 ? v.x : v.y; };
  float2 elo[2], ec[2], ehi[2], vlo[2], vc[2], vhi[2], bc[2];
  long long c = i0 + sy * j0 + sz * k0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const bool on = (r == 0) || row1;
    const long long cr = c + r * sy;
    elo[r] = (on && k0 > 0) ? ld2(e + cr - sz) : z2;
    ec[r] = on ? ld2(e + cr) : z2;
    ehi[r] = (on && k0 + 1 < bx.mz) ? ld2(e + cr + sz) : z2;
    vlo[r] = (on && k0 > 0) ? ld2(x + cr - sz) : z2;
    vc[r] = on ? ld2(x + cr) : z2;
    vhi[r] = (on && k0 + 1 < bx.mz) ? ld2(x + cr + sz) : z2;
    bc[r] = on ? ld2(b + cr) : z2;
  }
  float acc = 0.0f;
  for (int k = k0; k < k1; ++k, c += sz) {
    const bool up = (k + 1 < bx.mz);
    const bool up2 = (k + 2 < bx.mz) && (k + 1 < k1);
    float2 e2[2], v2[2], bn[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const bool on = (r == 0) || row1;
      const long long cr = c + r * sy;
      e2[r] = (on && up2) ? ld2(e + cr + 2 * sz) : z2;
      v2[r] = (on && up2) ? ld2(x + cr + 2 * sz) : z2;
      bn[r] = (on && k + 1 < k1) ? ld2(b + cr + sz) : z2;
    }
    const float2 eym = hym ? ld2(e + c - sy) : z2, vym = hym ? ld2(x + c - sy) : z2;
    const float2 eyp = (row1 && hyp) ? ld2(e + c + 2 * sy) : z2, vyp = (row1 && hyp) ? ld2(x + c + 2 * sy) : z2;
    if ((k & 1) == 0) acc = 0.0f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r == 1 && !row1) break;
      const int j = j0 + r;
      const long long cr = c + r * sy;
      const float exm = hxm ? __ldg(e + cr - 1) : 0.0f, exp_ = hxp ? __ldg(e + cr + 2) : 0.0f;
      const float vxm = hxm ? __ldg(x + cr - 1) : 0.0f, vxp = hxp ? __ldg(x + cr + 2) : 0.0f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = i0 + q;
        const float ecq = g2(ec[r], q);
        float d = mf_outlet(ecq, s, i == bx.mx - 1);
        float off = 0.0f;
        if (i + 1 < bx.mx) mf_link(ecq, q == 0 ? ec[r].y : exp_, q == 0 ? vc[r].y : vxp, hs, true, d, off);
        if (i > 0) mf_link(ecq, q == 1 ? ec[r].x : exm, q == 1 ? vc[r].x : vxm, hs, true, d, off);
        if (j + 1 < bx.my) mf_link(ecq, r == 0 ? g2(ec[1], q) : g2(eyp, q), r == 0 ? g2(vc[1], q) : g2(vyp, q), hs,
                                   true, d, off);
        if (j > 0) mf_link(ecq, r == 0 ? g2(eym, q) : g2(ec[0], q), r == 0 ? g2(vym, q) : g2(vc[0], q), hs, true, d,
                           off);
        if (up) mf_link(ecq, g2(ehi[r], q), g2(vhi[r], q), hs, true, d, off);
        if (k > 0) mf_link(ecq, g2(elo[r], q), g2(vlo[r], q), hs, true, d, off);
        acc += mf_result<SK_RES>(d, off, g2(vc[r], q), g2(bc[r], q), 0.0f);
      }
    }
    if ((k & 1) == 1 || k + 1 == bx.mz)
      bcoarse[(i0 >> 1) + (long long)cb.mx * ((j0 >> 1) + (long long)cb.my * (k >> 1))] = acc;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      elo[r] = ec[r];
      ec[r] = ehi[r];
      ehi[r] = e2[r];
      vlo[r] = vc[r];
      vc[r] = vhi[r];
      vhi[r] = v2[r];
      bc[r] = bn[r];
    }
  }
}

// The same on boxes of one row per plane (the z view of a 2D grid): four x
// cells per thread, aggregates of an x pair and a z pair.
__global__ void __launch_bounds__(kThreads) k_resid_restrict_mf4row(Box bx, const float* __restrict__ e, float s,
                                                                   const float* __restrict__ b,
                                                                   const float* __restrict__ x, Box cb,
                                                                   float* __restrict__ bcoarse, int zc,
                                                                   const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  Mf4March<SK_RES, XS_PLAIN> m;
  m.i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  m.j = 0;
  const int k0 = blockIdx.z * zc;  // zc even
  const int k1 = min(k0 + zc, bx.mz);
  if (m.i0 >= bx.mx || bx.my != 1 || k0 >= k1) return;
  m.bx = bx;
  m.e = e;
  m.b = b;
  m.x = x;
  m.s = s;
  m.omega = 0.0f;
  m.cb = cb;
  m.xc = nullptr;
  m.wc = 0.0f;
  m.init(k0);
  float sa = 0.0f, sb = 0.0f;  // aggregates i0/2 and i0/2 + 1
  long long c = m.i0 + m.sz * k0;
  for (int k = k0; k < k1; ++k, c += m.sz) {
    float r[4];
    m.plane(k, k1, c, r);
    if ((k & 1) == 0) {
      sa = 0.0f;
      sb = 0.0f;
    }
    sa += r[0];
    sa += r[1];
    sb += r[2];
    sb += r[3];
    if ((k & 1) == 1 || k + 1 == bx.mz) {
      const long long pc = (m.i0 >> 1) + (long long)cb.mx * (k >> 1);
      bcoarse[pc] = sa;
      bcoarse[pc + 1] = sb;
    }
  }
}

// MG-PCG on the matrix-free pressure level, fused with the V-cycle's first
// and last fine sweeps (four cells per thread, float):
//   k_xr_jac0_mf4: e += alpha p, r -= alpha q (the FMAs of k_pcg_xr), |r|^2
//     and the pass's stop test, and the V-cycle's first sweep from zero on
//     the new residual, x1 = (omega / diag) r, written to the V-cycle's
//     scratch vector;
//   k_jac_mf4_rz: the last post-smoothing sweep (z = its output, r = its
//     right-hand side) with sum r.z, finalising beta, or -- when the
//     floating-cluster deflation follows -- leaving the partial in
//     sc->rz_part for k_defl_apply_rz.
// The cell values are those of the separate kernels; the sums run in the
// sweep's thread order instead of the flat kernels', so the iterates agree
// to rounding, not bit for bit.
__global__ void __launch_bounds__(kThreads, 3) k_xr_jac0_mf4(Box bx, const float* __restrict__ e, float s,
                                                            const float* __restrict__ p, const float* __restrict__ q,
                                                            float* __restrict__ ex, float* __restrict__ r,
                                                            float* __restrict__ x1, float omega, int zc, KScal* sc,
                                                            RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const float alpha = (float)sc->alpha;
  Mf4March<SK_JAC0, XS_PLAIN> m;
  m.i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  m.j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (m.i0 < bx.mx && m.j < bx.my && k0 < k1) {
    m.bx = bx;
    m.e = e;
    m.b = q;  // the march's right-hand-side loads are dummies: each plane's b is the new r below
    m.x = nullptr;
    m.s = s;
    m.omega = omega;
    m.cb = bx;
    m.xc = nullptr;
    m.wc = 0.0f;
    m.init(k0);
    long long c = m.i0 + m.sy * m.j + m.sz * k0;
    for (int k = k0; k < k1; ++k, c += m.sz) {
      const float4 pv = Mf4March<SK_JAC0, XS_PLAIN>::ld4(p + c), qv = Mf4March<SK_JAC0, XS_PLAIN>::ld4(q + c);
      float4 ev = *reinterpret_cast<const float4*>(ex + c), rv = *reinterpret_cast<const float4*>(r + c);
      ev = make_float4(fmaf(alpha, pv.x, ev.x), fmaf(alpha, pv.y, ev.y), fmaf(alpha, pv.z, ev.z),
                       fmaf(alpha, pv.w, ev.w));
      rv = make_float4(fmaf(-alpha, qv.x, rv.x), fmaf(-alpha, qv.y, rv.y), fmaf(-alpha, qv.z, rv.z),
                       fmaf(-alpha, qv.w, rv.w));
      *reinterpret_cast<float4*>(ex + c) = ev;
      *reinterpret_cast<float4*>(r + c) = rv;
      ps.add(rv.x, rv.x);
      ps.add(rv.y, rv.y);
      ps.add(rv.z, rv.z);
      ps.add(rv.w, rv.w);
      m.bc = rv;
      float o[4];
      m.plane(k, k1, c, o);
      *reinterpret_cast<float4*>(x1 + c) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    sc->rr = acc[0];
    sc->iters += 1;
    if (acc[0] <= sc->tol2 || sc->iters >= sc->max_iters || !isfinite(acc[0])) sc->done = 1;
  }
}

template <int XS>
__global__ void __launch_bounds__(kThreads, 3) k_jac_mf4_rz(Box bx, const float* __restrict__ e, float s,
                                                           const float* __restrict__ b, const float* __restrict__ x,
                                                           float* __restrict__ out, float omega, int zc, KScal* sc,
                                                           RedScratch rs, Box cb, const float* __restrict__ xc,
                                                           float wc, int defer) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  Mf4March<SK_JAC, XS> m;
  m.i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  m.j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (m.i0 < bx.mx && m.j < bx.my && k0 < k1) {
    m.bx = bx;
    m.e = e;
    m.b = b;
    m.x = x;
    m.s = s;
    m.omega = omega;
    m.cb = cb;
    m.xc = xc;
    m.wc = wc;
    m.init(k0);
    long long c = m.i0 + m.sy * m.j + m.sz * k0;
    for (int k = k0; k < k1; ++k, c += m.sz) {
      const float4 bq = m.bc;
      float o[4];
      m.plane(k, k1, c, o);
      *reinterpret_cast<float4*>(out + c) = make_float4(o[0], o[1], o[2], o[3]);
      ps.add(bq.x, o[0]);
      ps.add(bq.y, o[1]);
      ps.add(bq.z, o[2]);
      ps.add(bq.w, o[3]);
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    if (defer)
      sc->rz_part = acc[0];
    else
      fin_pcg_beta(sc, acc[0]);
  }
}

// Constant-link FP32 sweeps (Op::mfc): links to the neighbours inside the
// box are all `a`, so a sweep reads diag and x (and b), not xp/yp/zp.
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_stencil_mfc(Box bx, const float* __restrict__ dg, float a,
                                                         const float* __restrict__ b, const float* __restrict__ x,
                                                         float* __restrict__ out, float omega, int zc,
                                                         const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  if (i >= bx.mx || j >= bx.my || k0 >= k1) return;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  const bool has_x = KIND != SK_JAC0;
  long long c = i + sy * j + sz * k0;
  float vlo = (has_x && k0 > 0) ? __ldg(x + c - sz) : 0.0f;
  float vc = has_x ? __ldg(x + c) : 0.0f;
  float vhi = (has_x && k0 + 1 < bx.mz) ? __ldg(x + c + sz) : 0.0f;
  float dc = __ldg(dg + c);
  float bc = (KIND != SK_MV) ? __ldg(b + c) : 0.0f;
  for (int k = k0; k < k1; ++k, c += sz) {
    const bool nxt = k + 1 < k1;
    const float v2 = (has_x && nxt && k + 2 < bx.mz) ? __ldg(x + c + 2 * sz) : 0.0f;
    const float dn = nxt ? __ldg(dg + c + sz) : 0.0f;
    const float bn = (KIND != SK_MV && nxt) ? __ldg(b + c + sz) : 0.0f;
    if (KIND == SK_JAC0) {
      out[c] = __fdividef(omega, dc) * bc;
    } else {
      float sum = 0.0f;  // sum of the neighbours inside the box
      if (i + 1 < bx.mx) sum += __ldg(x + c + 1);
      if (i > 0) sum += __ldg(x + c - 1);
      if (j + 1 < bx.my) sum += __ldg(x + c + sy);
      if (j > 0) sum += __ldg(x + c - sy);
      if (k + 1 < bx.mz) sum += vhi;
      if (k > 0) sum += vlo;
      const float ax = __fmaf_rn(dc, vc, __fmul_rn(a, sum));  // explicit rounding: the same in every kernel
      if (KIND == SK_JAC)
        out[c] = vc + __fdividef(omega, dc) * (bc - ax);
      else if (KIND == SK_MV)
        out[c] = ax;
      else
        out[c] = bc - ax;
    }
    vlo = vc;
    vc = vhi;
    vhi = v2;
    dc = dn;
    bc = bn;
  }
}

template <typename T>
__global__ void k_jac0(long long n, const T* __restrict__ diag, const T* __restrict__ dinv, const T* __restrict__ b,
                       T* __restrict__ x, T omega, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    T w;
    if constexpr (sizeof(T) == 4)
      w = __fdividef(omega, __ldg(diag + c));
    else
      w = __ldg(dinv + c);
    x[c] = w * __ldg(b + c);
  }
}

// Coarse correction x += wc * ec[parent] (2.5D: one thread per fine column).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_add(Box fb, Box cb, T* __restrict__ x, const T* __restrict__ ec,
                                                         T wc, int zc, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, fb.mz);
  if (i >= fb.mx || j >= fb.my || k0 >= k1) return;
  const long long sz = (long long)fb.mx * fb.my, csz = (long long)cb.mx * cb.my;
  long long c = i + (long long)fb.mx * j + sz * k0;
  const long long pc0 = (i >> 1) + (long long)cb.mx * (j >> 1);
  for (int k = k0; k < k1; ++k, c += sz) x[c] = fma(wc, __ldg(ec + pc0 + csz * (k >> 1)), x[c]);
}

// Restriction of a fine residual: bc[I] = sum of its (up to 8) children.
template <typename T>
__global__ void k_restrict_sum(Box fb, Box cb, const T* __restrict__ r, T* __restrict__ bc, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const Seg s = make_seg(cb);
  const int ni = fb.mx > 1 ? 2 : 1, nj = fb.my > 1 ? 2 : 1, nk = fb.mz > 1 ? 2 : 1;
  VOS_SEG_LOOP(s, q) {
    int I, J, K;
    seg_decode(s, cb, q, I, J, K);
    if (I >= cb.mx) continue;
    T sum = 0;
    for (int dk = 0; dk < nk; ++dk) {
      const int k = (fb.mz > 1) ? 2 * K + dk : 0;
      if (k >= fb.mz) continue;
      for (int dj = 0; dj < nj; ++dj) {
        const int j = (fb.my > 1) ? 2 * J + dj : 0;
        if (j >= fb.my) continue;
        const long long row = (long long)fb.mx * (j + (long long)fb.my * k);
        for (int di = 0; di < ni; ++di) {
          const int i = (fb.mx > 1) ? 2 * I + di : 0;
          if (i < fb.mx) sum += __ldg(r + row + i);
        }
      }
    }
    bc[I + (long long)cb.mx * (J + (long long)cb.my * K)] = sum;
  }
}

// ---------------------------------------------------------------------------
// Fused passes on the assembled (coarse) levels, one thread per output cell
// in the z view: the residual with the restriction (k_resid_restrict_c: each
// coarse cell sums the residuals b - A x of its children, added in the order
// of k_restrict_sum) and the prolongation with the first post-smoothing
// sweep (k_prolong_jac_c: x + wc x_c[parent] formed at the cell and its
// neighbours with the FMA of k_prolong_add, then the Jacobi update of
// k_stencil).  row_ax repeats k_stencil's statements for one cell, so both
// give the separate launches' values bit for bit with one launch fewer each
// per level and V-cycle (the coarse levels are launch-latency bound).
// ---------------------------------------------------------------------------
template <typename T, bool SYM, class XV>
__device__ __forceinline__ T row_ax(const Op<T>& Z, long long c, int i, int j, int k, T vc, XV xv) {
  const Box bx = Z.box;
  const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
  const T d = __ldg(Z.diag + c);
  T ax = rn_mul(d, vc);
  if (i + 1 < bx.mx) ax = fma(__ldg(Z.xp + c), xv(c + 1, i + 1, j, k), ax);
  if (i > 0) ax = fma((SYM ? __ldg(Z.xp + c - 1) : __ldg(Z.xm + c)), xv(c - 1, i - 1, j, k), ax);
  if (j + 1 < bx.my) ax = fma(__ldg(Z.yp + c), xv(c + sy, i, j + 1, k), ax);
  if (j > 0) ax = fma((SYM ? __ldg(Z.yp + c - sy) : __ldg(Z.ym + c)), xv(c - sy, i, j - 1, k), ax);
  if (bx.mz > 1) {
    const bool up = (k + 1 < bx.mz);
    const T vhi = up ? xv(c + sz, i, j, k + 1) : T(0);
    const T zu = up ? __ldg(Z.zp + c) : T(0);
    ax = fma(zu, vhi, ax);
    if (k > 0) ax = fma((SYM ? __ldg(Z.zp + c - sz) : __ldg(Z.zm + c)), xv(c - sz, i, j, k - 1), ax);
  }
  return ax;
}

template <typename T, bool SYM>
__global__ void k_resid_restrict_c(Op<T> Z, const T* __restrict__ b, const T* __restrict__ x, Box cz,
                                   T* __restrict__ bc, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const Box fb = Z.box;
  const Seg s = make_seg(cz);
  const int ni = fb.mx > 1 ? 2 : 1, nj = fb.my > 1 ? 2 : 1, nk = fb.mz > 1 ? 2 : 1;
  auto xv = [&](long long n, int, int, int) { return __ldg(x + n); };
  VOS_SEG_LOOP(s, q) {
    int I, J, K;
    seg_decode(s, cz, q, I, J, K);
    if (I >= cz.mx) continue;
    T sum = 0;
    for (int dk = 0; dk < nk; ++dk) {
      const int k = (fb.mz > 1) ? 2 * K + dk : 0;
      if (k >= fb.mz) continue;
      for (int dj = 0; dj < nj; ++dj) {
        const int j = (fb.my > 1) ? 2 * J + dj : 0;
        if (j >= fb.my) continue;
        for (int di = 0; di < ni; ++di) {
          const int i = (fb.mx > 1) ? 2 * I + di : 0;
          if (i >= fb.mx) continue;
          const long long c = i + (long long)fb.mx * (j + (long long)fb.my * k);
          sum += __ldg(b + c) - row_ax<T, SYM>(Z, c, i, j, k, __ldg(x + c), xv);
        }
      }
    }
    bc[I + (long long)cz.mx * (J + (long long)cz.my * K)] = sum;
  }
}

template <typename T, bool SYM>
__global__ void k_prolong_jac_c(Op<T> Z, const T* __restrict__ b, const T* __restrict__ x, Box cz,
                                const T* __restrict__ ec, T wc, T omega, T* __restrict__ out, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const Box fb = Z.box;
  const Seg s = make_seg(fb);
  auto xv = [&](long long n, int i, int j, int k) {
    return fma(wc, __ldg(ec + (i >> 1) + (long long)cz.mx * ((j >> 1) + (long long)cz.my * (k >> 1))), __ldg(x + n));
  };
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, fb, q, i, j, k);
    if (i >= fb.mx) continue;
    const long long c = i + (long long)fb.mx * (j + (long long)fb.my * k);
    const T vc = xv(c, i, j, k);
    const T ax = row_ax<T, SYM>(Z, c, i, j, k, vc, xv);
    T w;
    if constexpr (sizeof(T) == 4)
      w = __fdividef(omega, __ldg(Z.diag + c));
    else
      w = __ldg(Z.dinv + c);
    out[c] = fma(w, __ldg(b + c) - ax, vc);
  }
}

// Dot products with a device-side finalisation (deterministic FP64 reduce).
enum DotFin { DF_PCG_BETA = 0, DF_PCG_ALPHA = 1, DF_BICG_ALPHA = 2, DF_BICG_OMEGA = 3, DF_FCG_BETA = 4 };


template <typename T, int NV, int FIN>
__global__ void k_dots(long long n, const T* __restrict__ a0, const T* __restrict__ b0, const T* __restrict__ a1,
                       const T* __restrict__ b1, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  PSum<T> p0, p1;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    p0.add(__ldg(a0 + c), __ldg(b0 + c));
    if (NV == 2) p1.add(__ldg(a1 + c), __ldg(b1 + c));
  }
  double acc[NV];
  acc[0] = p0.get();
  if (NV == 2) acc[NV - 1] = p1.get();
  if (grid_sum<NV>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    if (FIN == DF_PCG_BETA) {
      fin_pcg_beta(sc, acc[0]);
    } else if (FIN == DF_FCG_BETA) {
      // Flexible CG with one stored direction (the preconditioner may vary
      // between iterations): beta = -(z.q_prev) / (p_prev.q_prev) makes the
      // new direction A-orthogonal to the previous one; alpha = (r.z) / (p.q)
      // stays the exact line search because r is orthogonal to p_prev.
      const double rz = acc[0];
      sc->beta = (sc->iters == 0 || !(sc->pq > 0.0)) ? 0.0 : -acc[NV - 1] / sc->pq;
      sc->rz = rz;
      if (!isfinite(rz) || !isfinite(sc->beta) || rz == 0.0) {
        sc->breakdown = 1;
        sc->done = 1;
      }
    } else if (FIN == DF_PCG_ALPHA) {
      const double pq = acc[0];
      sc->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        sc->breakdown = 1;
        sc->done = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / pq;
      }
    } else if (FIN == DF_BICG_ALPHA) {
      const double rhv = acc[0];
      sc->rhv = rhv;
      if (rhv == 0.0 || !isfinite(rhv)) {
        sc->breakdown = 1;
        sc->done = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rho / rhv;
      }
    } else {
      sc->ts = acc[0];
      sc->tt = acc[NV - 1];
      sc->omega = (acc[NV - 1] > 0.0 && isfinite(acc[NV - 1])) ? acc[0] / acc[NV - 1] : 0.0;
    }
  }
}

// PCG: p = z + beta p (first iteration: p = z)
template <typename T>
__global__ void k_pcg_p(long long n, const T* __restrict__ z, T* __restrict__ p, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const bool first = (sc->iters == 0);
  const T beta = (T)sc->beta;
  long long c0 = 0;
  if constexpr (sizeof(T) == 4) {  // FP32: 16-byte accesses (vectors are 256-byte aligned)
    const long long n4 = n >> 2;
    const float4* z4 = (const float4*)z;
    float4* p4 = (float4*)p;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += (long long)gridDim.x * blockDim.x) {
      const float4 zv = __ldg(z4 + v);
      if (first) {
        p4[v] = zv;
      } else {
        const float4 pv = p4[v];
        p4[v] = make_float4(fmaf(beta, pv.x, zv.x), fmaf(beta, pv.y, zv.y), fmaf(beta, pv.z, zv.z),
                            fmaf(beta, pv.w, zv.w));
      }
    }
    c0 = n4 << 2;
  }
  for (long long c = c0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    p[c] = first ? __ldg(z + c) : fma(beta, p[c], __ldg(z + c));
}

// ---------------------------------------------------------------------------
// Double-FP32 ("double-float") form of FP64 values for the refinement
// residual of the mixed path.  FP64 arithmetic is the bottleneck of the FP64
// residual on this part, so after the first refinement pass of a solve the
// residual b - A x is evaluated from FP32 pairs on the FP32 pipes.
// df_split cuts a double into hi = its leading 24 significand bits (exact,
// truncated) and lo = the next 23 bits (exact), by integer operations on the
// bit pattern, so it costs no FP64 instruction: |v - hi - lo| < 2^-46 |v|.
// Magnitudes below 2^-80 keep hi only (below 2^-126, nothing); a magnitude of
// 2^127 or more does not fit and is reported through the return value.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool df_split(double v, float2& out) {
  const unsigned h = (unsigned)__double2hiint(v), l = (unsigned)__double2loint(v);
  const unsigned e = (h >> 20) & 0x7ffu, sgn = h & 0x80000000u;
  if (e > 1150u) {
    out = make_float2(0.0f, 0.0f);
    return false;
  }
  if (e < 897u) {
    out = make_float2(0.0f, 0.0f);
    return true;
  }
  const float hi = __uint_as_float(sgn | ((e - 896u) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
  float lo = 0.0f;
  if (e >= 943u) {
    const float unit = __uint_as_float(0x4b000000u | ((l & 0x1fffffffu) >> 6)) - 8388608.0f;  // bits 28..6, exactly
    lo = __uint_as_float(__float_as_uint(unit * __uint_as_float((e - 942u) << 23)) | sgn);
  }
  out = make_float2(hi, lo);
  return true;
}

// s - a * x in double-FP32: (s.x, s.y) is an unevaluated sum, a * x is
// formed from the exact product of the leading parts (FMA error term) and
// the two cross terms; the new leading part comes from an exact two-sum.
__device__ __forceinline__ void df_sub_prod(float2& s, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float pe = __fmaf_rn(a.x, x.x, -p);
  const float cr = __fmaf_rn(a.x, x.y, __fmul_rn(a.y, x.x));
  const float t = __fsub_rn(s.x, p);
  const float bp = __fsub_rn(t, s.x);
  const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bp)), __fsub_rn(-p, bp));
  s.x = t;
  s.y = __fsub_rn(__fadd_rn(s.y, err), __fadd_rn(pe, cr));
}

// FP64 true residual b - A x in the 2.5D form (device body shared by the
// kernels below).  outer[0] = |D^-1 r|^2 and outer[1] = |D^-1 b|^2 (the
// convergence test); outer[2] = |r|^2, the unscaled norm the inner Krylov
// loop measures.  b is fixed during a solve, so |D^-1 b|^2 is summed on its
// first pass only (need_bb) and kept in outer[1]: FP64 arithmetic, not
// memory, bounds this kernel on this part.  dfo (non-null): also write the
// double-FP32 copies of b, x and the operator's diagonal and plus links
// (dfbad = 1 if a value does not fit that form).
template <typename T, bool SYM>
__device__ __forceinline__ void resid64_body(const Op<double>& A, const double* __restrict__ b, View<double> x,
                                             T* __restrict__ rT, double* outer, bool need_bb, int zc,
                                             const RedScratch& rs, const DFBuf* dfo, int* dfbad) {
  double acc[3] = {0.0, 0.0, 0.0};
  auto val = [&](long long, int i, int j, int k) -> double {
    return __ldg(x.base + i + (long long)x.sy * j + (long long)x.sz * k);
  };
  auto emit = [&](long long c, int i, int j, int k, double vc, double ax, double d) {
    const double bc = __ldg(b + c);
    const double r = bc - ax;
    if constexpr (sizeof(T) == 4)
      rT[c] = f32_rn(r);
    else
      rT[c] = (T)r;
    const double di = A.dinv[c];  // omega / diag: the constant omega cancels in the ratio
    const double r1 = r * di;
    acc[0] += r1 * r1;
    if (need_bb) {
      const double b1 = bc * di;
      acc[1] += b1 * b1;
    }
    acc[2] += r * r;
    if (dfo) {
      bool ok = df_split(bc, dfo->b[c]);
      ok &= df_split(vc, dfo->x[c]);
      ok &= df_split(d, dfo->dg[c]);
      if (i + 1 < A.box.mx) ok &= df_split(__ldg(A.xp + c), dfo->xp[c]);
      if (j + 1 < A.box.my) ok &= df_split(__ldg(A.yp + c), dfo->yp[c]);
      if (k + 1 < A.box.mz) ok &= df_split(__ldg(A.zp + c), dfo->zp[c]);
      if (!ok) *dfbad = 1;
    }
  };
  zmarch<double, SYM>(A, zc, val, emit);
  if (grid_sum<3>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    outer[0] = acc[0];
    if (need_bb) outer[1] = acc[1];
    outer[2] = acc[2];
  }
}

// The FP64 residual.  pass: the solve's refinement pass counter (null: a
// first pass); only0: run on the first pass only (later passes use
// k_outer_residual_df); dfo.x non-null: write the double-FP32 copies.
template <typename T, bool SYM>
__global__ void __launch_bounds__(kThreads) k_outer_residual_z(Op<double> A, const double* __restrict__ b,
                                                              View<double> x, T* __restrict__ rT, double* outer,
                                                              const int* pass, int zc, RedScratch rs, DFBuf dfo,
                                                              int* dfbad, int only0) {
  VOS_COUNT_EXEC();
  const bool first = (pass == nullptr) || (*pass == 0);
  if (only0 && !first) return;  // the same for every thread of the launch
  resid64_body<T, SYM>(A, b, x, rT, outer, first, zc, rs, dfo.x ? &dfo : nullptr, dfbad);
}

// The refinement residual of passes after the first in double-FP32 (mixed
// path, symmetric systems solved to 1e-9 or looser): from the copies written
// by the first pass (operator, b) and by the outer updates (x), with the
// row's terms subtracted in the FP64 kernel's order, r = hi + lo rounded to
// FP32.  The norms are summed in compensated FP32 after scaling by powers of
// two taken from the previous pass's norms (so the squares stay in range)
// and rescaled exactly in FP64.  If a value did not fit the double-FP32 form
// (*dfbad), the FP64 body runs instead.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_outer_residual_df(DFBuf d, const float* __restrict__ dinv32,
                                                               Op<double> A, const double* __restrict__ b,
                                                               View<double> x, T* __restrict__ rT, double* outer,
                                                               const int* pass, const int* dfbad, int zc,
                                                               RedScratch rs) {
  VOS_COUNT_EXEC();
  if (pass != nullptr && *pass == 0) return;  // the same for every thread of the launch
  if (*dfbad) {
    resid64_body<T, true>(A, b, x, rT, outer, false, zc, rs, nullptr, nullptr);
    return;
  }
  const Box bx = A.box;
  auto scale_exp = [](double o) {  // k with o * 4^-k near 1, |k| <= 100
    int e = 0;
    if (o > 0.0) frexp(o, &e);
    e /= 2;
    return e > 100 ? 100 : (e < -100 ? -100 : e);
  };
  const int k0s = scale_exp(outer[0]), k2s = scale_exp(outer[2]);
  const float s0 = ldexpf(1.0f, -k0s), s2 = ldexpf(1.0f, -k2s);
  PSum<float> p0, p2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int kb = blockIdx.z * zc;
  const int ke = min(kb + zc, bx.mz);
  if (i < bx.mx && j < bx.my && kb < ke) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    const float2 z2 = make_float2(0.0f, 0.0f);
    // z march: x at k-1, k, k+1 and the plane's own words in registers; the
    // loads of plane k+1 (x at k+2) are issued before plane k is computed
    long long c = i + sy * j + sz * kb;
    float2 xlo = (kb > 0) ? __ldg(d.x + c - sz) : z2;
    float2 xc = __ldg(d.x + c);
    float2 xhi = (kb + 1 < bx.mz) ? __ldg(d.x + c + sz) : z2;
    float2 zl = (kb > 0) ? __ldg(d.zp + c - sz) : z2;
    float2 bc = __ldg(d.b + c), dgc = __ldg(d.dg + c);
    float2 zu = (kb + 1 < bx.mz) ? __ldg(d.zp + c) : z2;
    float dic = __ldg(dinv32 + c);
    for (int k = kb; k < ke; ++k, c += sz) {
      const bool up = (k + 1 < bx.mz);
      const bool nxt = (k + 1 < ke);
      const float2 x2 = (nxt && k + 2 < bx.mz) ? __ldg(d.x + c + 2 * sz) : z2;
      const float2 bn = nxt ? __ldg(d.b + c + sz) : z2, dgn = nxt ? __ldg(d.dg + c + sz) : z2;
      const float2 zun = (nxt && k + 2 < bx.mz) ? __ldg(d.zp + c + sz) : z2;
      const float din = nxt ? __ldg(dinv32 + c + sz) : 0.0f;
      float2 S = bc;
      df_sub_prod(S, dgc, xc);
      if (i + 1 < bx.mx) df_sub_prod(S, __ldg(d.xp + c), __ldg(d.x + c + 1));
      if (i > 0) df_sub_prod(S, __ldg(d.xp + c - 1), __ldg(d.x + c - 1));
      if (j + 1 < bx.my) df_sub_prod(S, __ldg(d.yp + c), __ldg(d.x + c + sy));
      if (j > 0) df_sub_prod(S, __ldg(d.yp + c - sy), __ldg(d.x + c - sy));
      if (bx.mz > 1) {
        if (up) df_sub_prod(S, zu, xhi);
        if (k > 0) df_sub_prod(S, zl, xlo);
      }
      const float r = __fadd_rn(S.x, S.y);
      rT[c] = (T)r;
      const float r1 = __fmul_rn(__fmul_rn(r, dic), s0), r2 = __fmul_rn(r, s2);
      p0.add(r1, r1);
      p2.add(r2, r2);
      xlo = xc;
      xc = xhi;
      xhi = x2;
      zl = zu;
      zu = zun;
      bc = bn;
      dgc = dgn;
      dic = din;
    }
  }
  double acc[2] = {p0.get(), p2.get()};
  if (grid_sum<2>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    outer[0] = ldexp(acc[0], 2 * k0s);
    outer[2] = ldexp(acc[1], 2 * k2s);
  }
}

// Host: remap 2D boxes (mz == 1) so that y is the marched axis.
template <typename T>
static Op<T> zview(const Op<T>& A) {
  if (A.box.mz > 1 || A.box.my == 1) return A;
  Op<T> B = A;
  B.box = Box{A.box.mx, 1, A.box.my};
  B.zp = A.yp;
  B.zm = A.ym;
  B.yp = nullptr;
  B.ym = nullptr;
  return B;
}
static Box zbox(Box b) { return (b.mz > 1 || b.my == 1) ? b : Box{b.mx, 1, b.my}; }
static View<double> zview_x(View<double> x, Box b) {
  if (b.mz > 1 || b.my == 1) return x;
  return View<double>{x.base, 0, x.sy};
}

struct ZCfg {
  dim3 grid, block;
  int zc;
};
// A tile of tx x (kThreads / tx) threads in (x, y) marching over zc planes,
// zc chosen so that the grid has about target blocks (at least zmin planes
// per block, at most kMaxRedBlocks blocks).
static ZCfg zcfg_tile(Box b, int tx, long long target, int zmin = 4) {
  ZCfg z;
  const int ty = kThreads / tx;
  const long long gx = (b.mx + tx - 1) / tx, gy = (b.my + ty - 1) / ty;
  const long long tiles = gx * gy;
  long long zc = (tiles * b.mz + target - 1) / target;
  if (zc < zmin) zc = zmin;
  if (zc > b.mz) zc = b.mz;
  while (tiles * ((b.mz + zc - 1) / zc) > kMaxRedBlocks) ++zc;
  z.block = dim3(tx, ty, 1);
  z.grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)((b.mz + zc - 1) / zc));
  z.zc = (int)zc;
  return z;
}
// Default: tile 32 x 8, or 256 x 1 when the box has one row per plane, and
// about 4096 blocks.  Kernels with grid reductions always use this shape, so
// their summation order does not depend on tuning.
static ZCfg zcfg(Box b) { return zcfg_tile(b, (b.my == 1) ? 256 : 32, 4096); }
// Kernels without reductions (stencil sweeps, prolongation): the same tile,
// but blocks may march as little as one plane.  On small coarse levels each
// plane step waits for its loads, so fewer planes per block and more blocks
// cut the sweep's latency (a 64^3 level has 256 blocks of 4 planes with the
// default, 1,024 of one plane here).
static ZCfg zcfg_sweep(Box b) { return zcfg_tile(b, (b.my == 1) ? 256 : 32, 4096, 1); }
// Four-cells-per-thread matrix-free sweeps: 32 x 8 threads cover 128 x 8
// cells (256 x 1 threads = 1024 cells of a row on 2D boxes), about 1024
// blocks of one or more planes for the kernels with a grid reduction (on the
// 256^3 rock the graph-replayed step measured 91.1-91.5 ms with about 4096
// blocks, 88.9 with 2048 and 88.7 with 1024: the reductions' last blocks
// have fewer partial sums to add); the sweeps without one keep about 4096
// blocks (zcfg_mf4s; 88.5 ms).
static ZCfg zcfg_mf4(Box b) {
  const Box q{(b.mx + 3) / 4, b.my, b.mz};
  return zcfg_tile(q, (b.my == 1) ? 256 : 32, 1024, 1);
}
// The same tile for the four-cell sweeps without a reduction: about 4096
// blocks of fewer planes.
static ZCfg zcfg_mf4s(Box b) {
  const Box q{(b.mx + 3) / 4, b.my, b.mz};
  return zcfg_tile(q, (b.my == 1) ? 256 : 32, 4096, 1);
}
// Process-wide switch of the four-cells-per-thread matrix-free sweeps
// (vos_set_vector_sweeps; results are identical either way).
bool g_mf4 = true;

// ---------------------------------------------------------------------------
// Tile autotuner for the stencil sweeps (Jacobi / matvec / residual): per box
// shape, operand type and symmetry, the tile shape and z chunk with the
// shortest measured Jacobi sweep among a fixed candidate set.  Each cell's
// result is computed by the same arithmetic whatever the tile, so the choice
// changes timings only, never values.  Results are cached per process.
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, int>;  // mx, my, mz, sizeof(T), SYM (2: matrix-free)
static std::map<TuneKey, ZCfg> g_tuned;
static std::mutex g_tuned_mu;
constexpr long long kTuneMinCells = 1 << 16;  // smaller boxes are launch-latency bound

static ZCfg zcfg_stencil(Box b, int tsize, int sym) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  auto it = g_tuned.find(TuneKey{b.mx, b.my, b.mz, tsize, sym});
  return it == g_tuned.end() ? zcfg_sweep(b) : it->second;
}

static int tune_candidates(Box b, ZCfg* out) {
  int n = 0;
  const long long targets[] = {1024, 2048, 4096, 8192};
  if (b.my == 1) {
    for (long long t : targets) out[n++] = zcfg_tile(b, 256, t, 1);
  } else {
    const int txs[] = {32, 64, 128};
    for (int tx : txs)
      for (long long t : targets) out[n++] = zcfg_tile(b, tx, t, 1);
  }
  return n;
}

// ---------------------------------------------------------------------------
// Smoothing kernels
// ---------------------------------------------------------------------------

// Diagonal preconditioner z = (omega / diag) r with the fused r.z for PCG
// (the constant omega does not change the CG iterates).
template <typename T>
__global__ void k_diag_prec(long long n, const T* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ z,
                            KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  PSum<T> ps, pz;
  long long c0 = 0;
  if constexpr (sizeof(T) == 4) {  // FP32: 16-byte accesses (256-byte aligned arrays)
    const long long n4 = n >> 2;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += (long long)gridDim.x * blockDim.x) {
      const float4 rv = __ldg((const float4*)r + v), dv = __ldg((const float4*)dinv + v);
      const float4 zv = make_float4(dv.x * rv.x, dv.y * rv.y, dv.z * rv.z, dv.w * rv.w);
      ((float4*)z)[v] = zv;
      ps.add(rv.x, zv.x);
      ps.add(rv.y, zv.y);
      ps.add(rv.z, zv.z);
      ps.add(rv.w, zv.w);
      pz.add(zv.x, zv.x);
      pz.add(zv.y, zv.y);
      pz.add(zv.z, zv.z);
      pz.add(zv.w, zv.w);
    }
    c0 = n4 << 2;
  }
  for (long long c = c0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const T rc = r[c];
    const T zc = dinv[c] * rc;
    z[c] = zc;
    ps.add(rc, zc);
    pz.add(zc, zc);
  }
  double acc[2] = {ps.get(), pz.get()};
  if (grid_sum<2>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    fin_pcg_beta(sc, acc[0]);
    // z = (omega / diag) r, so z.z is omega^2 |D^-1 r|^2: the same scaled norm
    // as the FP64 refinement test, which ends the pass here
    if (sc->iters > 0 && acc[1] <= sc->tol2s) sc->done = 1;
  }
}

// Coarsest level: nsweep damped-Jacobi sweeps from zero, one block, in
// shared memory (box of at most kThreads cells).
template <typename T, bool SYM>
__global__ void k_coarse_solve(Op<T> A, const T* __restrict__ b, T* __restrict__ x, int nsweep, const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  __shared__ T xs[2][kThreads];
  const Box bx = A.box;
  const int n = (int)box_cells(bx);
  const int c = threadIdx.x;
  int i = 0, j = 0, k = 0;
  if (c < n) {
    i = c % bx.mx;
    j = (c / bx.mx) % bx.my;
    k = c / (bx.mx * bx.my);
  }
  T bc = (c < n) ? b[c] : T(0);
  T dinv = (c < n) ? A.dinv[c] : T(0);
  xs[0][c] = dinv * bc;
  __syncthreads();
  int cur = 0;
  for (int it = 1; it < nsweep; ++it) {
    if (c < n) {
      auto xat = [&](long long cc, int, int, int) -> T { return xs[cur][cc]; };
      T ax = stencil<T, SYM>(A, i, j, k, c, xat);
      xs[cur ^ 1][c] = fma(dinv, bc - ax, xs[cur][c]);
    }
    __syncthreads();
    cur ^= 1;
  }
  if (c < n) x[c] = xs[cur][c];
}

// ---------------------------------------------------------------------------
// Galerkin coarse operator (piecewise-constant prolongation P, R = P^T)
// ---------------------------------------------------------------------------
template <typename T, bool SYM>
__global__ void k_galerkin(Op<T> F, Op<T> C, T omega) {
  VOS_COUNT_EXEC();
  const Box fb = F.box, cb = C.box;
  const Seg s = make_seg(cb);
  VOS_SEG_LOOP(s, q) {
    int I, J, K;
    seg_decode(s, cb, q, I, J, K);
    if (I >= cb.mx) continue;
    double d = 0, xp = 0, yp = 0, zp = 0, xm = 0, ym = 0, zm = 0;
    const int nk = (fb.mz > 1) ? 2 : 1, nj = (fb.my > 1) ? 2 : 1, ni = (fb.mx > 1) ? 2 : 1;
    for (int dk = 0; dk < nk; ++dk) {
      int k = (fb.mz > 1) ? 2 * K + dk : 0;
      if (k >= fb.mz) continue;
      for (int dj = 0; dj < nj; ++dj) {
        int j = (fb.my > 1) ? 2 * J + dj : 0;
        if (j >= fb.my) continue;
        for (int di = 0; di < ni; ++di) {
          int i = (fb.mx > 1) ? 2 * I + di : 0;
          if (i >= fb.mx) continue;
          long long c = i + (long long)fb.mx * (j + (long long)fb.my * k);
          d += (double)F.diag[c];
          // x links
          if (i + 1 < fb.mx) {
            double a = (double)F.xp[c];
            if (di == 0 && fb.mx > 1) {  // internal link to i+1 (same parent)
              d += a;
              if (SYM) d += a;
            } else {
              xp += a;
            }
          }
          if (i > 0) {
            if (!SYM) {
              double a = (double)F.xm[c];
              if (di == 1) d += a; else xm += a;
            }
          }
          if (j + 1 < fb.my) {
            double a = (double)F.yp[c];
            if (dj == 0 && fb.my > 1) {
              d += a;
              if (SYM) d += a;
            } else {
              yp += a;
            }
          }
          if (j > 0 && !SYM) {
            double a = (double)F.ym[c];
            if (dj == 1) d += a; else ym += a;
          }
          if (fb.mz > 1) {
            if (k + 1 < fb.mz) {
              double a = (double)F.zp[c];
              if (dk == 0) {
                d += a;
                if (SYM) d += a;
              } else {
                zp += a;
              }
            }
            if (k > 0 && !SYM) {
              double a = (double)F.zm[c];
              if (dk == 1) d += a; else zm += a;
            }
          }
        }
      }
    }
    long long cc = I + (long long)cb.mx * (J + (long long)cb.my * K);
    C.diag[cc] = (T)d;
    C.dinv[cc] = (T)((double)omega / d);
    C.xp[cc] = (T)xp;
    C.yp[cc] = (T)yp;
    if (cb.mz > 1) C.zp[cc] = (T)zp;
    if (!SYM) {
      C.xm[cc] = (T)xm;
      C.ym[cc] = (T)ym;
      if (cb.mz > 1) C.zm[cc] = (T)zm;
    }
  }
}

// ---------------------------------------------------------------------------
// Krylov vector kernels
// ---------------------------------------------------------------------------
// scaled != 0: the pass ends on the diagonally scaled norm (z.z in
// k_diag_prec, or |dscale r|^2 in k_pcg_xr) instead of the unscaled r.r
// (see scaled_test).
__global__ void k_kscal_init(KScal* sc, const double* outer, double rtol_inner, int max_iters, int scaled) {
  VOS_COUNT_EXEC();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double rr = outer[2];  // unscaled |r|^2 of the inner right-hand side
    sc->bb = rr;
    sc->rr = rr;
    sc->rz = 0;
    sc->rz_old = 0;
    sc->pq = 0;
    sc->alpha = 0;
    sc->beta = 0;
    sc->omega = 1.0;
    sc->rho = rr;
    sc->rhv = 0;
    sc->tol2 = scaled ? -1.0 : rtol_inner * rtol_inner * rr;
    sc->tol2s = rtol_inner * rtol_inner * outer[0];
    sc->iters = 0;
    sc->max_iters = max_iters;
    sc->breakdown = 0;
    sc->done = (rr == 0.0) ? 1 : 0;
  }
}

// PCG: e += alpha p; r -= alpha q; rr = r.r; convergence check.
// PCG: e += alpha p; r -= alpha q.  With dscale (= omega / diag of the fine
// operator) the pass ends on the diagonally scaled norm |dscale r|^2 <=
// tol2s, the norm of the FP64 refinement test; otherwise on |r|^2 <= tol2.
template <typename T>
__global__ void k_pcg_xr(long long n, const T* __restrict__ p, const T* __restrict__ qv, T* __restrict__ e,
                         T* __restrict__ r, const T* __restrict__ dscale, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const T alpha = (T)sc->alpha;
  PSum<T> ps, pd;
  long long c0 = 0;
  if constexpr (sizeof(T) == 4) {  // FP32 without the scaled norm: 16-byte accesses
    if (!dscale) {
      const long long n4 = n >> 2;
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
           v += (long long)gridDim.x * blockDim.x) {
        const float4 pv = __ldg((const float4*)p + v), qv4 = __ldg((const float4*)qv + v);
        float4 ev = ((float4*)e)[v], rv = ((float4*)r)[v];
        ev = make_float4(fmaf(alpha, pv.x, ev.x), fmaf(alpha, pv.y, ev.y), fmaf(alpha, pv.z, ev.z),
                         fmaf(alpha, pv.w, ev.w));
        rv = make_float4(fmaf(-alpha, qv4.x, rv.x), fmaf(-alpha, qv4.y, rv.y), fmaf(-alpha, qv4.z, rv.z),
                         fmaf(-alpha, qv4.w, rv.w));
        ((float4*)e)[v] = ev;
        ((float4*)r)[v] = rv;
        ps.add(rv.x, rv.x);
        ps.add(rv.y, rv.y);
        ps.add(rv.z, rv.z);
        ps.add(rv.w, rv.w);
      }
      c0 = n4 << 2;
    }
  }
  for (long long c = c0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    e[c] = fma(alpha, p[c], e[c]);
    T rc = fma(-alpha, qv[c], r[c]);
    r[c] = rc;
    ps.add(rc, rc);
    if (dscale) {
      const T rsc = rc * __ldg(dscale + c);
      pd.add(rsc, rsc);
    }
  }
  double acc[2] = {ps.get(), pd.get()};
  if (grid_sum<2>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    sc->rr = acc[0];
    sc->iters += 1;
    const bool conv = dscale ? (acc[1] <= sc->tol2s) : (acc[0] <= sc->tol2);
    if (conv || sc->iters >= sc->max_iters || !isfinite(acc[0])) sc->done = 1;
  }
}

// Constant-link FP32 matvec q = A p fused with p.q (alpha = r.z / p.q).
// Threads outside the box stay for the grid reduction.
__global__ void __launch_bounds__(kThreads) k_matvec_mfc_dot(Box bx, const float* __restrict__ dg, float a,
                                                            const float* __restrict__ x, float* __restrict__ out,
                                                            int zc, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (i < bx.mx && j < bx.my && k0 < k1) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    long long c = i + sy * j + sz * k0;
    float vlo = (k0 > 0) ? __ldg(x + c - sz) : 0.0f;
    float vc = __ldg(x + c);
    float vhi = (k0 + 1 < bx.mz) ? __ldg(x + c + sz) : 0.0f;
    float dc = __ldg(dg + c);
    for (int k = k0; k < k1; ++k, c += sz) {
      const bool nxt = k + 1 < k1;
      const float v2 = (nxt && k + 2 < bx.mz) ? __ldg(x + c + 2 * sz) : 0.0f;
      const float dn = nxt ? __ldg(dg + c + sz) : 0.0f;
      float sum = 0.0f;
      if (i + 1 < bx.mx) sum += __ldg(x + c + 1);
      if (i > 0) sum += __ldg(x + c - 1);
      if (j + 1 < bx.my) sum += __ldg(x + c + sy);
      if (j > 0) sum += __ldg(x + c - sy);
      if (k + 1 < bx.mz) sum += vhi;
      if (k > 0) sum += vlo;
      const float ax = __fmaf_rn(dc, vc, __fmul_rn(a, sum));  // explicit rounding: the same in every kernel
      out[c] = ax;
      ps.add(vc, ax);
      vlo = vc;
      vc = vhi;
      vhi = v2;
      dc = dn;
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    const double pq = acc[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->breakdown = 1;
      sc->done = 1;
      sc->alpha = 0.0;
    } else {
      sc->alpha = sc->rz / pq;
    }
  }
}

// Matrix-free pressure matvec q = A p (links from e, see k_stencil_mf) fused
// with p.q (alpha = r.z / p.q).  Threads outside the box stay for the grid
// reduction.
__global__ void __launch_bounds__(kThreads) k_matvec_mf_dot(Box bx, const float* __restrict__ e, float s,
                                                           const float* __restrict__ x, float* __restrict__ out,
                                                           int zc, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (i < bx.mx && j < bx.my && k0 < k1) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    const float hs = 0.5f * s;
    long long c = i + sy * j + sz * k0;
    float elo = (k0 > 0) ? __ldg(e + c - sz) : 0.0f;
    float ec = __ldg(e + c);
    float ehi = (k0 + 1 < bx.mz) ? __ldg(e + c + sz) : 0.0f;
    float vlo = (k0 > 0) ? __ldg(x + c - sz) : 0.0f;
    float vc = __ldg(x + c);
    float vhi = (k0 + 1 < bx.mz) ? __ldg(x + c + sz) : 0.0f;
    for (int k = k0; k < k1; ++k, c += sz) {
      const bool up2 = (k + 2 < bx.mz) && (k + 1 < k1);
      const float e2 = up2 ? __ldg(e + c + 2 * sz) : 0.0f;
      const float v2 = up2 ? __ldg(x + c + 2 * sz) : 0.0f;
      float d = mf_outlet(ec, s, i == bx.mx - 1);
      float off = 0.0f;
      if (i + 1 < bx.mx) mf_link(ec, __ldg(e + c + 1), __ldg(x + c + 1), hs, true, d, off);
      if (i > 0) mf_link(ec, __ldg(e + c - 1), __ldg(x + c - 1), hs, true, d, off);
      if (j + 1 < bx.my) mf_link(ec, __ldg(e + c + sy), __ldg(x + c + sy), hs, true, d, off);
      if (j > 0) mf_link(ec, __ldg(e + c - sy), __ldg(x + c - sy), hs, true, d, off);
      if (k + 1 < bx.mz) mf_link(ec, ehi, vhi, hs, true, d, off);
      if (k > 0) mf_link(ec, elo, vlo, hs, true, d, off);
      const float ax = mf_result<SK_MV>(d, off, vc, 0.0f, 0.0f);
      out[c] = ax;
      ps.add(vc, ax);
      elo = ec;
      ec = ehi;
      ehi = e2;
      vlo = vc;
      vc = vhi;
      vhi = v2;
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    const double pq = acc[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->breakdown = 1;
      sc->done = 1;
      sc->alpha = 0.0;
    } else {
      sc->alpha = sc->rz / pq;
    }
  }
}

// Four-cells-per-thread forms of the two fused matvec + p.q kernels above
// (16-byte rows: nx % 4 == 0), with the per-cell arithmetic of the one-cell
// kernels; each thread adds its four cells' products in x order to its
// partial sum, so the summation order (and the last bits of p.q) differs
// from the one-cell kernels.
__device__ __forceinline__ void fin_alpha(KScal* sc, double pq) {
  sc->pq = pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    sc->breakdown = 1;
    sc->done = 1;
    sc->alpha = 0.0;
  } else {
    sc->alpha = sc->rz / pq;
  }
}

__global__ void __launch_bounds__(kThreads) k_matvec_mfc4_dot(Box bx, const float* __restrict__ dg, float a,
                                                             const float* __restrict__ x, float* __restrict__ out,
                                                             int zc, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (i0 < bx.mx && j < bx.my && k0 < k1) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    auto ld4 = [](const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); };
    const bool hxm = i0 > 0, hxp = i0 + 4 < bx.mx, hym = j > 0, hyp = j + 1 < bx.my;
    long long c = i0 + sy * j + sz * k0;
    float4 vlo = (k0 > 0) ? ld4(x + c - sz) : z4;
    float4 vc = ld4(x + c);
    float4 vhi = (k0 + 1 < bx.mz) ? ld4(x + c + sz) : z4;
    float4 dc = ld4(dg + c);
    for (int k = k0; k < k1; ++k, c += sz) {
      const bool nxt = k + 1 < k1;
      const float4 v2 = (nxt && k + 2 < bx.mz) ? ld4(x + c + 2 * sz) : z4;
      const float4 dn = nxt ? ld4(dg + c + sz) : z4;
      const float vxm = hxm ? __ldg(x + c - 1) : 0.0f, vxp = hxp ? __ldg(x + c + 4) : 0.0f;
      const float4 vym = hym ? ld4(x + c - sy) : z4, vyp = hyp ? ld4(x + c + sy) : z4;
      float r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q;
        float sum = 0.0f;
        if (i + 1 < bx.mx) sum += q < 3 ? f4get(vc, q + 1) : vxp;
        if (i > 0) sum += q > 0 ? f4get(vc, q - 1) : vxm;
        if (hyp) sum += f4get(vyp, q);
        if (hym) sum += f4get(vym, q);
        if (k + 1 < bx.mz) sum += f4get(vhi, q);
        if (k > 0) sum += f4get(vlo, q);
        const float vq = f4get(vc, q);
        r[q] = __fmaf_rn(f4get(dc, q), vq, __fmul_rn(a, sum));
        ps.add(vq, r[q]);
      }
      *reinterpret_cast<float4*>(out + c) = make_float4(r[0], r[1], r[2], r[3]);
      vlo = vc;
      vc = vhi;
      vhi = v2;
      dc = dn;
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) fin_alpha(sc, acc[0]);
}

__global__ void __launch_bounds__(kThreads, 4) k_matvec_mf4_dot(Box bx, const float* __restrict__ e, float s,
                                                            const float* __restrict__ x, float* __restrict__ out,
                                                            int zc, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  Mf4March<SK_MV, XS_PLAIN> m;
  m.i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  m.j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (m.i0 < bx.mx && m.j < bx.my && k0 < k1) {
    m.bx = bx;
    m.e = e;
    m.b = nullptr;
    m.x = x;
    m.s = s;
    m.omega = 0.0f;
    m.cb = bx;
    m.xc = nullptr;
    m.wc = 0.0f;
      m.init(k0);
    long long c = m.i0 + m.sy * m.j + m.sz * k0;
    for (int k = k0; k < k1; ++k, c += m.sz) {
      const float4 pc = m.vc;
      float r[4];
      m.plane(k, k1, c, r);
      *reinterpret_cast<float4*>(out + c) = make_float4(r[0], r[1], r[2], r[3]);
      ps.add(pc.x, r[0]);
      ps.add(pc.y, r[1]);
      ps.add(pc.z, r[2]);
      ps.add(pc.w, r[3]);
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) fin_alpha(sc, acc[0]);
}


// ---------------------------------------------------------------------------
// Diagonally preconditioned CG on a constant-link operator in two kernels per
// iteration instead of four (direction update, matvec with p.q, x/r update,
// preconditioner with r.z):
//   k_pcg_pmv_mfc*: p = z + beta p_prev (p = z on the first iteration),
//                   q = A p and p.q (alpha = r.z / p.q);
//   k_pcg_xrz:      e += alpha p, r -= alpha q, z = (omega / diag) r, with
//                   r.r, r.z and z.z (beta = r.z / r.z_prev; the pass ends
//                   on z.z, the scaled norm of the FP64 refinement test).
// The matvec needs p at the six neighbours, so the direction update is
// evaluated there too, from z and p_prev; p_prev and the p written are two
// buffers.  Each value is computed with the operations (and each dot summed
// in the order) of the four-kernel form, so both give identical iterates.
// DRAM words per unknown: 5 (read z, p_prev, diagonal; write p, q) and 8
// (read p, q, e, r, omega / diagonal; write e, r, z), against 16 for the
// four-kernel iteration.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pnew(float z, float pp, float beta, bool first) {
  return first ? z : __fmaf_rn(beta, pp, z);
}

__global__ void __launch_bounds__(kThreads) k_pcg_pmv_mfc(Box bx, const float* __restrict__ dg, float a,
                                                         const float* __restrict__ z, const float* __restrict__ pprev,
                                                         float* __restrict__ pout, float* __restrict__ q, int zc,
                                                         KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const bool first = (sc->iters == 0);
  const float beta = first ? 0.0f : (float)sc->beta;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (i < bx.mx && j < bx.my && k0 < k1) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    auto pv = [&](long long c) { return pnew(__ldg(z + c), first ? 0.0f : __ldg(pprev + c), beta, first); };
    long long c = i + sy * j + sz * k0;
    float vlo = (k0 > 0) ? pv(c - sz) : 0.0f;
    float vc = pv(c);
    float vhi = (k0 + 1 < bx.mz) ? pv(c + sz) : 0.0f;
    float dc = __ldg(dg + c);
    for (int k = k0; k < k1; ++k, c += sz) {
      const bool nxt = k + 1 < k1;
      const float v2 = (nxt && k + 2 < bx.mz) ? pv(c + 2 * sz) : 0.0f;
      const float dn = nxt ? __ldg(dg + c + sz) : 0.0f;
      float sum = 0.0f;
      if (i + 1 < bx.mx) sum += pv(c + 1);
      if (i > 0) sum += pv(c - 1);
      if (j + 1 < bx.my) sum += pv(c + sy);
      if (j > 0) sum += pv(c - sy);
      if (k + 1 < bx.mz) sum += vhi;
      if (k > 0) sum += vlo;
      const float ax = __fmaf_rn(dc, vc, __fmul_rn(a, sum));  // explicit rounding: the same in every kernel
      pout[c] = vc;
      q[c] = ax;
      ps.add(vc, ax);
      vlo = vc;
      vc = vhi;
      vhi = v2;
      dc = dn;
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) fin_alpha(sc, acc[0]);
}

// The same, four consecutive x cells per thread (nx % 4 == 0: 16-byte rows).
__global__ void __launch_bounds__(kThreads) k_pcg_pmv_mfc4(Box bx, const float* __restrict__ dg, float a,
                                                          const float* __restrict__ z,
                                                          const float* __restrict__ pprev, float* __restrict__ pout,
                                                          float* __restrict__ q, int zc, KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const bool first = (sc->iters == 0);
  const float beta = first ? 0.0f : (float)sc->beta;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, bx.mz);
  PSum<float> ps;
  if (i0 < bx.mx && j < bx.my && k0 < k1) {
    const long long sy = bx.mx, sz = (long long)bx.mx * bx.my;
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    auto ld4 = [](const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); };
    auto pv = [&](long long c) { return pnew(__ldg(z + c), first ? 0.0f : __ldg(pprev + c), beta, first); };
    auto pv4 = [&](long long c) {
      const float4 zv = ld4(z + c);
      const float4 pp = first ? z4 : ld4(pprev + c);
      return make_float4(pnew(zv.x, pp.x, beta, first), pnew(zv.y, pp.y, beta, first), pnew(zv.z, pp.z, beta, first),
                         pnew(zv.w, pp.w, beta, first));
    };
    const bool hxm = i0 > 0, hxp = i0 + 4 < bx.mx, hym = j > 0, hyp = j + 1 < bx.my;
    long long c = i0 + sy * j + sz * k0;
    float4 vlo = (k0 > 0) ? pv4(c - sz) : z4;
    float4 vc = pv4(c);
    float4 vhi = (k0 + 1 < bx.mz) ? pv4(c + sz) : z4;
    float4 dc = ld4(dg + c);
    for (int k = k0; k < k1; ++k, c += sz) {
      const bool nxt = k + 1 < k1;
      const float4 v2 = (nxt && k + 2 < bx.mz) ? pv4(c + 2 * sz) : z4;
      const float4 dn = nxt ? ld4(dg + c + sz) : z4;
      const float vxm = hxm ? pv(c - 1) : 0.0f, vxp = hxp ? pv(c + 4) : 0.0f;
      const float4 vym = hym ? pv4(c - sy) : z4, vyp = hyp ? pv4(c + sy) : z4;
      float res[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = i0 + t;
        float sum = 0.0f;
        if (i + 1 < bx.mx) sum += t < 3 ? f4get(vc, t + 1) : vxp;
        if (i > 0) sum += t > 0 ? f4get(vc, t - 1) : vxm;
        if (hyp) sum += f4get(vyp, t);
        if (hym) sum += f4get(vym, t);
        if (k + 1 < bx.mz) sum += f4get(vhi, t);
        if (k > 0) sum += f4get(vlo, t);
        const float vt = f4get(vc, t);
        res[t] = __fmaf_rn(f4get(dc, t), vt, __fmul_rn(a, sum));
        ps.add(vt, res[t]);
      }
      *reinterpret_cast<float4*>(pout + c) = vc;
      *reinterpret_cast<float4*>(q + c) = make_float4(res[0], res[1], res[2], res[3]);
      vlo = vc;
      vc = vhi;
      vhi = v2;
      dc = dn;
    }
  }
  double acc[1] = {ps.get()};
  if (grid_sum<1>(acc, rs.partials, rs.counter) && lin_tid() == 0) fin_alpha(sc, acc[0]);
}

__global__ void k_pcg_xrz(long long n, const float* __restrict__ p, const float* __restrict__ qv, float* __restrict__ e,
                          float* __restrict__ r, const float* __restrict__ dinv, float* __restrict__ z, KScal* sc,
                          RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const float alpha = (float)sc->alpha;
  PSum<float> prr, prz, pzz;
  const long long n4 = n >> 2;  // 16-byte accesses (vectors are 256-byte aligned)
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += (long long)gridDim.x * blockDim.x) {
    const float4 pv = __ldg((const float4*)p + v), q4 = __ldg((const float4*)qv + v);
    const float4 dv = __ldg((const float4*)dinv + v);
    float4 ev = ((float4*)e)[v], rv = ((float4*)r)[v];
    ev = make_float4(__fmaf_rn(alpha, pv.x, ev.x), __fmaf_rn(alpha, pv.y, ev.y), __fmaf_rn(alpha, pv.z, ev.z),
                     __fmaf_rn(alpha, pv.w, ev.w));
    rv = make_float4(__fmaf_rn(-alpha, q4.x, rv.x), __fmaf_rn(-alpha, q4.y, rv.y), __fmaf_rn(-alpha, q4.z, rv.z),
                     __fmaf_rn(-alpha, q4.w, rv.w));
    const float4 zv = make_float4(dv.x * rv.x, dv.y * rv.y, dv.z * rv.z, dv.w * rv.w);
    ((float4*)e)[v] = ev;
    ((float4*)r)[v] = rv;
    ((float4*)z)[v] = zv;
    prr.add(rv.x, rv.x);
    prr.add(rv.y, rv.y);
    prr.add(rv.z, rv.z);
    prr.add(rv.w, rv.w);
    prz.add(rv.x, zv.x);
    prz.add(rv.y, zv.y);
    prz.add(rv.z, zv.z);
    prz.add(rv.w, zv.w);
    pzz.add(zv.x, zv.x);
    pzz.add(zv.y, zv.y);
    pzz.add(zv.z, zv.z);
    pzz.add(zv.w, zv.w);
  }
  for (long long c = (n4 << 2) + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    e[c] = __fmaf_rn(alpha, p[c], e[c]);
    const float rc = __fmaf_rn(-alpha, qv[c], r[c]);
    r[c] = rc;
    const float zc = dinv[c] * rc;
    z[c] = zc;
    prr.add(rc, rc);
    prz.add(rc, zc);
    pzz.add(zc, zc);
  }
  double acc[3] = {prr.get(), prz.get(), pzz.get()};
  if (grid_sum<3>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    sc->rr = acc[0];
    sc->iters += 1;
    if (sc->iters >= sc->max_iters || !isfinite(acc[0])) {
      sc->done = 1;
    } else {
      fin_pcg_beta(sc, acc[1]);
      if (acc[2] <= sc->tol2s) sc->done = 1;
    }
  }
}

// BiCGStab: p = r + beta (p - omega v)   (first iteration: p = r)
template <typename T>
__global__ void k_bicg_p(long long n, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ p,
                         const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const bool first = (sc->iters == 0);
  const T beta = (T)sc->beta, omega = (T)sc->omega;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    p[c] = first ? r[c] : r[c] + beta * (p[c] - omega * v[c]);
  }
}

// BiCGStab: s = r - alpha v
template <typename T>
__global__ void k_bicg_s(long long n, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ sv,
                         const KScal* sc) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const T alpha = (T)sc->alpha;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    sv[c] = r[c] - alpha * v[c];
}

// BiCGStab: e += alpha ph + omega sh; r = s - omega t; rr, rho_new = rh.r
template <typename T>
__global__ void k_bicg_x(long long n, const T* __restrict__ ph, const T* __restrict__ sh, const T* __restrict__ sv,
                         const T* __restrict__ t, const T* __restrict__ rh, T* __restrict__ e, T* __restrict__ r,
                         KScal* sc, RedScratch rs) {
  VOS_COUNT_EXEC();
  DONE_RETURN(sc);
  const T alpha = (T)sc->alpha, omega = (T)sc->omega;
  PSum<T> p0, p1;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    e[c] += alpha * ph[c] + omega * sh[c];
    T rc = sv[c] - omega * t[c];
    r[c] = rc;
    p0.add(rc, rc);
    p1.add(rh[c], rc);
  }
  double acc[2] = {p0.get(), p1.get()};
  if (grid_sum<2>(acc, rs.partials, rs.counter) && lin_tid() == 0) {
    double rr = acc[0], rho_new = acc[1];
    sc->rr = rr;
    sc->iters += 1;
    if (rr <= sc->tol2 || sc->iters >= sc->max_iters || !isfinite(rr)) sc->done = 1;
    if (sc->omega == 0.0 || rho_new == 0.0 || !isfinite(rho_new)) {
      sc->breakdown = 1;
      sc->done = 1;
    } else {
      sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
      sc->rho = rho_new;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 outer refinement kernels
// ---------------------------------------------------------------------------
// x += e (x a strided view)
template <typename T>
__global__ void k_outer_update(Box bx, View<double> x, const T* __restrict__ e, float2* __restrict__ xdf,
                               int* dfbad) {
  VOS_COUNT_EXEC();
  const Seg s = make_seg(bx);
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    long long c = i + (long long)bx.mx * (j + (long long)bx.my * k);
    double* px = x.base + i + (long long)x.sy * j + (long long)x.sz * k;
    const double nx = *px + (double)e[c];
    *px = nx;
    if (xdf && !df_split(nx, xdf[c])) *dfbad = 1;  // double-FP32 copy for the next residual
  }
}

// x = 0 on a strided view
__global__ void k_view_zero(Box bx, View<double> x) {
  VOS_COUNT_EXEC();
  const Seg s = make_seg(bx);
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    x.base[i + (long long)x.sy * j + (long long)x.sz * k] = 0.0;
  }
}

// Convert the FP64 operator into T (level 0 of a mixed-precision hierarchy).
// links == 0: diagonal and Jacobi weights only (a constant-link fine level
// without coarse levels reads nothing else).
template <typename T>
__global__ void k_op_convert(Op<double> A, Op<T> B, long long n, int links) {
  VOS_COUNT_EXEC();
  auto cv = [](double v) -> T {
    if constexpr (sizeof(T) == 4)
      return f32_rn(v);
    else
      return (T)v;
  };
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    B.diag[c] = cv(A.diag[c]);
    B.dinv[c] = cv(A.dinv[c]);
    if (!links) continue;
    B.xp[c] = cv(A.xp[c]);
    B.yp[c] = cv(A.yp[c]);
    if (A.box.mz > 1) B.zp[c] = cv(A.zp[c]);
    if (!A.sym) {
      B.xm[c] = cv(A.xm[c]);
      B.ym[c] = cv(A.ym[c]);
      if (A.box.mz > 1) B.zm[c] = cv(A.zm[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int flat_grid(long long n) {
  long long need = (n + kThreads - 1) / kThreads;
  long long cap = (long long)g_num_sms * 8;
  if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
static size_t op_bytes(Box b, int sym) {
  size_t n = (size_t)box_cells(b);
  int narr = 2 + (b.mz > 1 ? 3 : 2) * (sym ? 1 : 2);
  return narr * align256(n * sizeof(T));
}

template <typename T>
static void op_carve(Op<T>& A, Box b, int sym, char*& cur) {
  size_t n = (size_t)box_cells(b);
  size_t sz = align256(n * sizeof(T));
  auto take = [&]() {
    T* p = (T*)cur;
    cur += sz;
    return p;
  };
  A.box = b;
  A.sym = sym;
  A.mfe = nullptr;
  A.mfs = 0.0f;
  A.mfc = 0.0f;
  A.diag = take();
  A.dinv = take();
  A.xp = take();
  A.yp = take();
  A.zp = (b.mz > 1) ? take() : nullptr;
  if (!sym) {
    A.xm = take();
    A.ym = take();
    A.zm = (b.mz > 1) ? take() : nullptr;
  } else {
    A.xm = A.ym = A.zm = nullptr;
  }
}

static int count_levels(Box fine) {
  int n = 1;
  Box b = fine;
  while (n < 16 && box_cells(b) > kThreads) {
    Box c = coarse_box(b);
    if (box_cells(c) == box_cells(b)) break;
    b = c;
    ++n;
  }
  return n;
}

template <typename T>
size_t hier_bytes(Box fine, int sym, bool share_level0) {
  size_t tot = 0;
  int nlev = count_levels(fine);
  Box b = fine;
  for (int l = 0; l < nlev; ++l) {
    size_t n = (size_t)box_cells(b);
    if (!(l == 0 && share_level0)) tot += op_bytes<T>(b, sym);
    if (l > 0) tot += 3 * align256(n * sizeof(T));
    b = coarse_box(b);
  }
  return tot;
}

size_t op64_bytes(Box b, int sym) { return op_bytes<double>(b, sym); }
void op64_carve(Op<double>& A, Box b, int sym, char*& cur) { op_carve<double>(A, b, sym, cur); }

template <typename T>
void hier_carve(Hier<T>& h, Box fine, int sym, char*& cur, const MGParams& mg, bool share_level0,
                const Op<double>* op64) {
  h.nlev = count_levels(fine);
  h.mg = mg;
  h.defl = Defl{0, nullptr, nullptr, nullptr};
  h.net = nullptr;
  h.tail = h.nlev;
  Box b = fine;
  for (int l = 0; l < h.nlev; ++l) {
    Level<T>& L = h.lev[l];
    if (l == 0 && share_level0) {
      std::memcpy(&L.op, op64, sizeof(Op<T>));  // T == double here: level 0 is op64
    } else {
      op_carve<T>(L.op, b, sym, cur);
    }
    size_t n = (size_t)box_cells(b);
    if (l > 0) {
      L.x = (T*)cur;
      cur += align256(n * sizeof(T));
      L.t = (T*)cur;
      cur += align256(n * sizeof(T));
      L.b = (T*)cur;
      cur += align256(n * sizeof(T));
    } else {
      L.x = L.t = L.b = nullptr;
    }
    b = coarse_box(b);
  }
  // cluster-resident coarse cycle, if the device runs the cluster it needs
  const int ts = tail_plan<T>(h);
  if (ts < h.nlev) {
    const size_t smem = tail_smem<T>(h, ts);
    const bool ok = sym ? tail_supported<T, true>(smem) : tail_supported<T, false>(smem);
    if (ok) h.tail = ts;
  }
}

template size_t hier_bytes<double>(Box, int, bool);
template size_t hier_bytes<float>(Box, int, bool);
template void hier_carve<double>(Hier<double>&, Box, int, char*&, const MGParams&, bool, const Op<double>*);
template void hier_carve<float>(Hier<float>&, Box, int, char*&, const MGParams&, bool, const Op<double>*);

size_t solver_work_bytes(long long max_cells) {
  return 18 * align256((size_t)max_cells * sizeof(double)) + align256(sizeof(KScal)) + align256(4 * sizeof(double)) +
         align256(sizeof(int));
}

SolverWork* solver_work_carve(char*& cur, long long max_cells) {
  SolverWork* w = new SolverWork();
  w->cap = max_cells;
  size_t vs = align256((size_t)max_cells * sizeof(double));
  void** vec[12] = {&w->r, &w->z, &w->p, &w->p2, &w->q, &w->e, &w->rh, &w->v, &w->s, &w->t, &w->ph, &w->sh};
  for (int i = 0; i < 12; ++i) {
    *vec[i] = cur;
    cur += vs;
  }
  w->sc = (KScal*)cur;
  cur += align256(sizeof(KScal));
  w->outer = (double*)cur;
  cur += align256(4 * sizeof(double));
  float2** dfv[6] = {&w->df.dg, &w->df.xp, &w->df.yp, &w->df.zp, &w->df.b, &w->df.x};
  for (int i = 0; i < 6; ++i) {
    *dfv[i] = (float2*)cur;
    cur += vs;
  }
  w->dfbad = (int*)cur;
  cur += align256(sizeof(int));
  cudaMallocHost((void**)&w->sc_host, sizeof(KScal));
  cudaMallocHost((void**)&w->outer_host, 2 * sizeof(double));
  return w;
}

void solver_work_free(SolverWork* w) {
  if (!w) return;
  if (w->sc_host) cudaFreeHost(w->sc_host);
  if (w->outer_host) cudaFreeHost(w->outer_host);
  delete w;
}

template <typename T>
void build_coarse_levels(Hier<T>& h, cudaStream_t st) {
  for (int l = 1; l < h.nlev; ++l) {
    Op<T>& F = h.lev[l - 1].op;
    Op<T>& C = h.lev[l].op;
    int g = grid_for(C.box, 0);
    const double gbytes = ((1.0 + n_offs(F)) * ncell(F) + (2.0 + n_offs(C)) * ncell(C)) * sizeof(T);
    if (F.sym)
      vlaunch(KN("mg_galerkin", l == 1), gbytes, k_galerkin<T, true>, g, kThreads, st, F, C, (T)h.mg.omega);
    else
      vlaunch(KN("mg_galerkin", l == 1), gbytes, k_galerkin<T, false>, g, kThreads, st, F, C, (T)h.mg.omega);
  }
}
template void build_coarse_levels<double>(Hier<double>&, cudaStream_t);
template void build_coarse_levels<float>(Hier<float>&, cudaStream_t);

template <typename T, bool SYM>
static void tune_launch(const ZCfg& z, const Op<T>& Z, const T* b, const T* x, T* out, cudaStream_t st) {
  if constexpr (sizeof(T) == 4 && SYM) {
    if (Z.mfe) {
      k_stencil_mf<SK_JAC><<<z.grid, z.block, 0, st>>>(Z.box, Z.mfe, Z.mfs, (const float*)b, (const float*)x,
                                                       (float*)out, 0.7f, z.zc, nullptr);
      return;
    }
  }
  k_stencil<T, SYM, SK_JAC><<<z.grid, z.block, 0, st>>>(Z, b, x, out, T(0.7), z.zc, nullptr);
}

template <typename T>
void autotune_hier(const Hier<T>& h, SolverWork* w, cudaStream_t st) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return;
  }
  T* b = (T*)w->r;
  T* x = (T*)w->z;
  T* out = (T*)w->p;
  for (int l = 0; l < h.nlev; ++l) {
    const Op<T>& A = h.lev[l].op;
    const long long n = box_cells(A.box);
    if (n < kTuneMinCells || n > w->cap) continue;
    const Op<T> Z = zview(A);
    const bool sym = A.sym != 0;
    const int code = (sizeof(T) == 4 && sym && A.mfe) ? 2 : (sym ? 1 : 0);
    const TuneKey key{Z.box.mx, Z.box.my, Z.box.mz, (int)sizeof(T), code};
    {
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      if (g_tuned.count(key)) continue;
    }
    cudaMemsetAsync(b, 0, (size_t)n * sizeof(T), st);
    cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), st);
    ZCfg cand[16];
    const int nc = tune_candidates(Z.box, cand);
    const int reps = n >= (1 << 22) ? 3 : 10;
    float best = 0.0f;
    int bi = -1;
    for (int c = 0; c < nc; ++c) {
      auto run = [&] {
        if (sym)
          tune_launch<T, true>(cand[c], Z, b, x, out, st);
        else
          tune_launch<T, false>(cand[c], Z, b, x, out, st);
      };
      run();  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps; ++r) run();
      cudaEventRecord(e1, st);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (bi < 0 || ms < best) {
        best = ms;
        bi = c;
      }
    }
    if (bi >= 0) {
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      g_tuned[key] = cand[bi];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}
template void autotune_hier<double>(const Hier<double>&, SolverWork*, cudaStream_t);
template void autotune_hier<float>(const Hier<float>&, SolverWork*, cudaStream_t);

void default_sweep_config(int mx, int my, int mz, int* tx, int* ty, int* zc) {
  const ZCfg z = zcfg_sweep(Box{mx, my, mz});
  *tx = (int)z.block.x;
  *ty = (int)z.block.y;
  *zc = z.zc;
}

int tuned_config(int mx, int my, int mz, int tsize, int sym, int* tx, int* ty, int* zc) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  auto it = g_tuned.find(TuneKey{mx, my, mz, tsize, sym});
  if (it == g_tuned.end()) return 0;
  *tx = (int)it->second.block.x;
  *ty = (int)it->second.block.y;
  *zc = it->second.zc;
  return 1;
}

// One V(nu, nu) cycle: out = M^{-1} rhs (level-0 vectors supplied).
// Level l owns (b, x, t).  Pre-smoothing starts with x = w b in t, every
// Jacobi sweep writes the other buffer, the fine residual goes to the free
// buffer, the coarse correction is added in place; after the 2 nu - 1 buffer
// swaps the result is in x.
template <typename T, bool SYM>
static void stencil_launch(const char* name, int kind, const Op<T>& A, const T* b, const T* x, T* out, T omega,
                           const KScal* sc, cudaStream_t st) {
  const Op<T> Z = zview(A);
  if constexpr (sizeof(T) == 4 && SYM) {
    if (A.mfc != 0.0f) {  // constant links: diag is the only coefficient word
      const ZCfg z = zcfg_stencil(Z.box, 4, 1);
      static const char* const mfc_names[4] = {"mg_jac_mfc_f32_L0", "pcg_matvec_mfc_f32_L0", "mg_resid_mfc_f32_L0",
                                               "mg_jac0_mfc_f32_L0"};
      const double words = 1.0 + (kind == SK_MV ? 2.0 : (kind == SK_JAC0 ? 2.0 : 3.0));
      const double n = ncell(A);
      const float om = (float)omega;
      const float* dg = (const float*)Z.diag;
      const float* bb = (const float*)b;
      const float* xx = (const float*)x;
      float* oo = (float*)out;
      if (kind == SK_JAC)
        vlaunch(mfc_names[kind], words * n * 4.0, k_stencil_mfc<SK_JAC>, z.grid, z.block, st, Z.box, dg, A.mfc, bb, xx,
                oo, om, z.zc, sc);
      else if (kind == SK_MV)
        vlaunch(mfc_names[kind], words * n * 4.0, k_stencil_mfc<SK_MV>, z.grid, z.block, st, Z.box, dg, A.mfc, bb, xx,
                oo, om, z.zc, sc);
      else if (kind == SK_RES)
        vlaunch(mfc_names[kind], words * n * 4.0, k_stencil_mfc<SK_RES>, z.grid, z.block, st, Z.box, dg, A.mfc, bb,
                xx, oo, om, z.zc, sc);
      else
        vlaunch(mfc_names[kind], words * n * 4.0, k_stencil_mfc<SK_JAC0>, z.grid, z.block, st, Z.box, dg, A.mfc, bb,
                xx, oo, om, z.zc, sc);
      return;
    }
    if (A.mfe) {  // matrix-free fine level: one coefficient word (e) per cell
      const ZCfg z = zcfg_stencil(Z.box, 4, 2);
      const double n = ncell(A);
      const double words = 1.0 + (kind == SK_MV ? 2.0 : (kind == SK_JAC0 ? 2.0 : 3.0));
      static const char* const mf_names[4] = {"mg_jac_mf_f32_L0", "pcg_matvec_mf_f32_L0", "mg_resid_mf_f32_L0",
                                              "mg_jac0_mf_f32_L0"};
      name = mf_names[kind];
      const float om = (float)omega;
      const float* bb = (const float*)b;
      const float* xx = (const float*)x;
      float* oo = (float*)out;
      if (g_mf4 && Z.box.mx % 4 == 0) {  // 16-byte rows: four cells per thread
        const ZCfg z4 = zcfg_mf4s(Z.box);
        if (kind == SK_JAC)
          vlaunch(name, words * n * 4.0, k_stencil_mf4<SK_JAC, XS_PLAIN>, z4.grid, z4.block, st, Z.box, A.mfe, A.mfs, bb,
                  xx, oo, om, z4.zc, sc, Box{0, 0, 0}, (const float*)nullptr, 0.0f);
        else if (kind == SK_MV)
          vlaunch(name, words * n * 4.0, k_stencil_mf4<SK_MV, XS_PLAIN>, z4.grid, z4.block, st, Z.box, A.mfe, A.mfs, bb,
                  xx, oo, om, z4.zc, sc, Box{0, 0, 0}, (const float*)nullptr, 0.0f);
        else if (kind == SK_RES)
          vlaunch(name, words * n * 4.0, k_stencil_mf4<SK_RES, XS_PLAIN>, z4.grid, z4.block, st, Z.box, A.mfe, A.mfs, bb,
                  xx, oo, om, z4.zc, sc, Box{0, 0, 0}, (const float*)nullptr, 0.0f);
        else
          vlaunch(name, words * n * 4.0, k_stencil_mf4<SK_JAC0, XS_PLAIN>, z4.grid, z4.block, st, Z.box, A.mfe, A.mfs, bb,
                  xx, oo, om, z4.zc, sc, Box{0, 0, 0}, (const float*)nullptr, 0.0f);
        return;
      }
      if (kind == SK_JAC)
        vlaunch(name, words * n * 4.0, k_stencil_mf<SK_JAC>, z.grid, z.block, st, Z.box, A.mfe, A.mfs, bb, xx, oo, om,
                z.zc, sc);
      else if (kind == SK_MV)
        vlaunch(name, words * n * 4.0, k_stencil_mf<SK_MV>, z.grid, z.block, st, Z.box, A.mfe, A.mfs, bb, xx, oo, om,
                z.zc, sc);
      else if (kind == SK_RES)
        vlaunch(name, words * n * 4.0, k_stencil_mf<SK_RES>, z.grid, z.block, st, Z.box, A.mfe, A.mfs, bb, xx, oo, om,
                z.zc, sc);
      else
        vlaunch(name, words * n * 4.0, k_stencil_mf<SK_JAC0>, z.grid, z.block, st, Z.box, A.mfe, A.mfs, bb, xx, oo,
                om, z.zc, sc);
      return;
    }
  }
  const ZCfg z = zcfg_stencil(Z.box, (int)sizeof(T), SYM ? 1 : 0);
  const double wT = sizeof(T), n = ncell(A);
  const double words = (kind == SK_MV ? 2.0 : 3.0) + 1.0 + n_offs(A) + (kind == SK_JAC && sizeof(T) == 8 ? 1.0 : 0.0);
  if (kind == SK_JAC)
    vlaunch(name, words * n * wT, k_stencil<T, SYM, SK_JAC>, z.grid, z.block, st, Z, b, x, out, omega, z.zc, sc);
  else if (kind == SK_MV)
    vlaunch(name, words * n * wT, k_stencil<T, SYM, SK_MV>, z.grid, z.block, st, Z, b, x, out, omega, z.zc, sc);
  else
    vlaunch(name, words * n * wT, k_stencil<T, SYM, SK_RES>, z.grid, z.block, st, Z, b, x, out, omega, z.zc, sc);
}

template <typename T, bool SYM>
// rz (fused MG-PCG only, see fused_mg_pcg): the last fine sweep also sums
// rhs.out (k_jac_mf4_rz; deferred to the deflation when the hierarchy has
// one); jac0_done: the first fine sweep's output is already in scratch
// (k_xr_jac0_mf4).
static void vcycle(Hier<T>& h, const T* rhs, T* out, T* scratch, KScal* sc, cudaStream_t st,
                   const RedScratch* rz = nullptr, bool jac0_done = false) {
  const int L = h.nlev;
  const int nu = h.mg.nu < 1 ? 1 : h.mg.nu;
  const T wc = (T)h.mg.wc, om = (T)h.mg.omega;
  auto bufs = [&](int l, const T*& b, T*& x, T*& t) {
    if (l == 0) {
      b = rhs;
      x = out;
      t = scratch;
    } else {
      b = h.lev[l].b;
      x = h.lev[l].x;
      t = h.lev[l].t;
    }
  };
  // The matrix-free FP32 fine level with four-cell rows fuses its residual
  // with the restriction and its prolongation with the first post-smoothing
  // sweep (bit-identical to the separate passes).
  auto fused_fine = [&](int l) {
    if constexpr (sizeof(T) == 4 && SYM) {
      const Op<T>& A = h.lev[l].op;
      return l == 0 && A.mfe != nullptr && g_mf4 && zview(A).box.mx % 4 == 0 && l + 1 < L;
    }
    return false;
  };
  // coarse (assembled) levels of at most 2^18 cells: residual with
  // restriction, prolongation with the first post-smoothing sweep
  // (bit-identical to the separate launches).  On larger levels the
  // one-thread-per-cell gathers are slower than the z-marching sweep plus a
  // streaming pass.
  auto fused_coarse = [&](int l) {
    return g_mf4 && l >= 1 && l + 1 < L && box_cells(h.lev[l].op.box) <= (1LL << 18);
  };
  auto jac0 = [&](int l, T* dst) {
    const Op<T>& A = h.lev[l].op;
    const T* b;
    T *x, *t;
    bufs(l, b, x, t);
    const long long n = box_cells(A.box);
    if (sizeof(T) == 4 && SYM && (A.mfe || A.mfc != 0.0f)) {
      stencil_launch<T, SYM>(KN("mg_jac0", l == 0), SK_JAC0, A, b, nullptr, dst, om, sc, st);
      return;
    }
    vlaunch(KN("mg_jac0", l == 0), 3.0 * n * sizeof(T), k_jac0<T>, flat_grid(n), kThreads, st, n, (const T*)A.diag,
            (const T*)A.dinv, b, dst, om, (const KScal*)sc);
  };
  if (L == 1) {
    const int cs = h.mg.coarse_sweeps < 2 ? 2 : h.mg.coarse_sweeps;
    const Op<T>& A = h.lev[0].op;
    const T* b;
    T *x, *t;
    bufs(0, b, x, t);
    T* cur = ((cs - 1) % 2 == 0) ? x : t;
    T* oth = (cur == x) ? t : x;
    jac0(0, cur);
    for (int s = 1; s < cs; ++s) {
      stencil_launch<T, SYM>(KN("mg_jac", true), SK_JAC, A, b, cur, oth, om, sc, st);
      T* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    return;
  }
  // levels h.tail..L-1 run as one cluster launch (vos_mgtail.cu) when the
  // hierarchy has a tail; the separate launches below cover the levels above
  const int ts = (h.tail > 0 && h.tail < L) ? h.tail : L;
  const int Ld = (ts < L) ? ts : L - 1;
  T* pre[16];
  for (int l = 0; l < Ld; ++l) {
    const Op<T>& A = h.lev[l].op;
    const T* b;
    T *x, *t;
    bufs(l, b, x, t);
    T* cur = t;
    T* oth = x;
    if (!(l == 0 && jac0_done)) jac0(l, cur);
    for (int s = 1; s < nu; ++s) {
      stencil_launch<T, SYM>(KN("mg_jac", l == 0), SK_JAC, A, b, cur, oth, om, sc, st);
      T* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    pre[l] = cur;
    const Op<T>& C = h.lev[l + 1].op;
    if (fused_fine(l)) {
      const Op<T> Z = zview(A);
      const double rb = (3.0 * ncell(A) + ncell(C)) * 4.0;
      // an even number of planes per block, from an even plane
      auto even = [&](ZCfg z) {
        if (z.zc & 1) {
          z.zc += 1;
          z.grid.z = (unsigned)((Z.box.mz + z.zc - 1) / z.zc);
        }
        return z;
      };
      if (Z.box.my == 1) {
        const ZCfg z = even(zcfg_mf4(Z.box));
        vlaunch("mg_resid_restrict_mf_f32_L0", rb, k_resid_restrict_mf4row, z.grid, z.block, st, Z.box, A.mfe,
                A.mfs, (const float*)b, (const float*)cur, zbox(C.box), (float*)h.lev[l + 1].b, z.zc,
                (const KScal*)sc);
      } else {  // 2 x 2 cells per thread
        const ZCfg z = even(zcfg_tile(Box{(Z.box.mx + 1) / 2, (Z.box.my + 1) / 2, Z.box.mz}, 32, 4096, 2));
        vlaunch("mg_resid_restrict_mf_f32_L0", rb, k_resid_restrict_mf22, z.grid, z.block, st, Z.box, A.mfe,
                A.mfs, (const float*)b, (const float*)cur, zbox(C.box), (float*)h.lev[l + 1].b, z.zc,
                (const KScal*)sc);
      }
    } else if (fused_coarse(l)) {
      const Op<T> Z = zview(A);
      const Box cz = zbox(C.box);
      vlaunch(KN("mg_resid_restrict", false), ((3.0 + n_offs(A)) * ncell(A) + ncell(C)) * sizeof(T),
              k_resid_restrict_c<T, SYM>, grid_for(cz, 0), kThreads, st, Z, b, (const T*)cur, cz, h.lev[l + 1].b,
              (const KScal*)sc);
    } else {
      stencil_launch<T, SYM>(KN("mg_resid", l == 0), SK_RES, A, b, cur, oth, om, sc, st);
      vlaunch(KN("mg_restrict", l == 0), (ncell(A) + ncell(C)) * sizeof(T), k_restrict_sum<T>, grid_for(C.box, 0),
              kThreads, st, A.box, C.box, (const T*)oth, h.lev[l + 1].b, (const KScal*)sc);
    }
  }
  if (ts < L) {
    tail_launch<T, SYM>(h, ts, sc, st);
  } else {
    const Op<T>& A = h.lev[L - 1].op;
    vlaunch(KN("mg_coarse", false), (4.0 + n_offs(A)) * ncell(A) * sizeof(T), k_coarse_solve<T, SYM>, 1, kThreads, st,
            A, h.lev[L - 1].b, h.lev[L - 1].x, h.mg.coarse_sweeps, (const KScal*)sc);
  }
  for (int l = Ld - 1; l >= 0; --l) {
    const Op<T>& A = h.lev[l].op;
    const T* b;
    T *x, *t;
    bufs(l, b, x, t);
    T* cur = pre[l];
    T* oth = (cur == x) ? t : x;
    const Box fz = zbox(A.box), cz = zbox(h.lev[l + 1].op.box);
    int s0 = 0;
    const bool rz_here = (l == 0 && rz != nullptr);
    const int dfr = h.defl.K > 0 ? 1 : 0;
    if (fused_fine(l)) {  // first sweep on x + wc P x_coarse, formed on the fly
      const Op<T> Z = zview(A);
      const ZCfg z4 = zcfg_mf4(Z.box), z4s = zcfg_mf4s(Z.box);
      const double bytes = (4.0 * ncell(A) + ncell(h.lev[l + 1].op)) * 4.0;
      if (rz_here && nu == 1)
        vlaunch("mg_jac_pro_rz_mf_f32_L0", bytes, k_jac_mf4_rz<XS_PRO>, z4.grid, z4.block, st, Z.box, A.mfe, A.mfs,
                (const float*)b, (const float*)cur, (float*)oth, (float)om, z4.zc, sc, *rz, cz,
                (const float*)h.lev[l + 1].x, (float)wc, dfr);
      else
        vlaunch("mg_jac_pro_mf_f32_L0", bytes, k_stencil_mf4<SK_JAC, XS_PRO>, z4s.grid, z4s.block, st, Z.box, A.mfe,
                A.mfs, (const float*)b, (const float*)cur, (float*)oth, (float)om, z4s.zc, (const KScal*)sc, cz,
                (const float*)h.lev[l + 1].x, (float)wc);
      T* tmp = cur;
      cur = oth;
      oth = tmp;
      s0 = 1;
    } else if (fused_coarse(l)) {  // first sweep on x + wc P x_coarse, formed on the fly
      vlaunch(KN("mg_jac_pro", false), ((4.0 + n_offs(A)) * ncell(A) + ncell(h.lev[l + 1].op)) * sizeof(T),
              k_prolong_jac_c<T, SYM>, grid_for(fz, 0), kThreads, st, zview(A), b, (const T*)cur, cz,
              (const T*)h.lev[l + 1].x, wc, om, oth, (const KScal*)sc);
      T* tmp = cur;
      cur = oth;
      oth = tmp;
      s0 = 1;
    } else {
      const ZCfg zc = zcfg_sweep(fz);
      vlaunch(KN("mg_prolong", l == 0), (2.0 * ncell(A) + ncell(h.lev[l + 1].op)) * sizeof(T), k_prolong_add<T>,
              zc.grid, zc.block, st, fz, cz, cur, (const T*)h.lev[l + 1].x, wc, zc.zc, (const KScal*)sc);
    }
    for (int s = s0; s < nu; ++s) {
      if (rz_here && s == nu - 1 && fused_fine(l)) {  // the last fine sweep with rhs.out
        const Op<T> Z = zview(A);
        const ZCfg z4 = zcfg_mf4(Z.box);
        vlaunch("mg_jac_rz_mf_f32_L0", 4.0 * ncell(A) * 4.0, k_jac_mf4_rz<XS_PLAIN>, z4.grid, z4.block, st, Z.box,
                A.mfe, A.mfs, (const float*)b, (const float*)cur, (float*)oth, (float)om, z4.zc, sc, *rz, Z.box,
                (const float*)nullptr, 0.0f, dfr);
      } else {
        stencil_launch<T, SYM>(KN("mg_jac", l == 0), SK_JAC, A, b, cur, oth, om, sc, st);
      }
      T* tmp = cur;
      cur = oth;
      oth = tmp;
    }
  }
}

// Vectors of the inner solves (views of SolverWork).
template <typename T>
struct KVec {
  T *r, *z, *p, *q, *e, *rh, *v, *s, *t, *ph, *sh, *scratch;
};
template <typename T>
static KVec<T> kvec(SolverWork* w, bool bicg) {
  KVec<T> k;
  k.r = (T*)w->r;
  k.z = (T*)w->z;
  k.p = (T*)w->p;
  k.q = (T*)w->q;
  k.e = (T*)w->e;
  k.rh = (T*)w->rh;
  k.v = (T*)w->v;
  k.s = (T*)w->s;
  k.t = (T*)w->t;
  k.ph = (T*)w->ph;
  k.sh = (T*)w->sh;
  k.scratch = bicg ? (T*)w->z : (T*)w->t;
  return k;
}

// MG-PCG on the matrix-free FP32 pressure level with its V-cycle's first
// and last fine sweeps fused with the Krylov x/r update and with r.z
// (k_xr_jac0_mf4, k_jac_mf4_rz; vos_set_fused_pcg).
template <typename T, bool SYM>
static bool fused_mg_pcg(const Hier<T>& h) {
  if constexpr (sizeof(T) == 4 && SYM) {
    const Op<T>& A = h.lev[0].op;
    return (g_fused_pcg & 2) && g_mf4 && A.mfe != nullptr && h.nlev >= 2 && zview(A).box.mx % 4 == 0 &&
           h.defl.K <= kMaxRedBlocks * kMaxRedValues;
  }
  return false;
}

// z = M^-1 r and the PCG beta (multigrid V-cycle plus the floating-cluster
// deflation when the hierarchy has one, or the diagonal).  jac0_done: the
// V-cycle's first fine sweep already ran, fused with the x/r update.
template <typename T, bool SYM>
static void pcg_precond(Hier<T>& h, const KVec<T>& k, long long n, SolverWork* w, const RedScratch& rs,
                        cudaStream_t st, bool use_mg, bool use_net = false, bool jac0_done = false) {
  const int gf = flat_grid(n);
  if (use_mg && !use_net && fused_mg_pcg<T, SYM>(h)) {
    vcycle<T, SYM>(h, k.r, k.z, k.scratch, w->sc, st, &rs, jac0_done);
    if (h.defl.K > 0) launch_defl_apply_rz<float>(h.defl, (const float*)k.r, (float*)k.z, w->sc, rs, st);
    return;
  }
  if (use_net && h.net) {
    unet_precond<T>(h.net, k.r, k.z, &w->sc->rr, st);
    vlaunch(KN("dot_rz_zq", true), 3.0 * n * sizeof(T), k_dots<T, 2, DF_FCG_BETA>, gf, kThreads, st, n,
            (const T*)k.r, (const T*)k.z, (const T*)k.z, (const T*)k.q, w->sc, rs);
  } else if (use_mg) {
    vcycle<T, SYM>(h, k.r, k.z, k.scratch, w->sc, st);
    launch_defl_apply<T>(h.defl, k.r, k.z, w->sc, st);
    vlaunch(KN("dot_rz", true), 2.0 * n * sizeof(T), k_dots<T, 1, DF_PCG_BETA>, gf, kThreads, st, n, (const T*)k.r,
            (const T*)k.z, (const T*)nullptr, (const T*)nullptr, w->sc, rs);
  } else {
    vlaunch(KN("diag_prec", true), 3.0 * n * sizeof(T), k_diag_prec<T>, gf, kThreads, st, n,
            (const T*)h.lev[0].op.dinv, (const T*)k.r, k.z, w->sc, rs);
  }
}

// Process-wide switches of the fused Krylov forms (vos_set_fused_pcg): bit 0
// the two-kernel diagonal PCG on constant-link operators, bit 1 MG-PCG on the
// matrix-free level fused with the V-cycle's first and last fine sweeps, bit
// 2 the double-FP32 refinement residual (see df_residual).
int g_fused_pcg = 7;

// One PCG iteration (kernels early-exit once the solve is done).  parity:
// the iteration's index within its pass modulo 2 (the two-kernel diagonal
// iteration alternates its two direction buffers, k.p and k.s, by it).
template <typename T, bool SYM>
static void pcg_iteration(Hier<T>& h, const KVec<T>& k, long long n, SolverWork* w, const RedScratch& rs,
                          cudaStream_t st, bool use_mg, bool use_net = false, int parity = 0) {
  const Op<T>& A = h.lev[0].op;
  const int gf = flat_grid(n);
  if constexpr (sizeof(T) == 4 && SYM) {
    if ((g_fused_pcg & 1) && A.mfc != 0.0f && !use_mg && !use_net) {
      const Op<T> Z = zview(A);
      const float* pin = (const float*)(parity ? k.s : k.p);
      float* pout = (float*)(parity ? k.p : k.s);
      if (Z.box.mx % 4 == 0) {  // same shape as the four-kernel matvec: the same summation order
        const ZCfg z = zcfg_mf4(Z.box);
        vlaunch("pcg_pmv_mfc_f32_L0", 5.0 * n * 4.0, k_pcg_pmv_mfc4, z.grid, z.block, st, Z.box,
                (const float*)Z.diag, A.mfc, (const float*)k.z, pin, pout, (float*)k.q, z.zc, w->sc, rs);
      } else {
        const ZCfg z = zcfg(Z.box);
        vlaunch("pcg_pmv_mfc_f32_L0", 5.0 * n * 4.0, k_pcg_pmv_mfc, z.grid, z.block, st, Z.box, (const float*)Z.diag,
                A.mfc, (const float*)k.z, pin, pout, (float*)k.q, z.zc, w->sc, rs);
      }
      vlaunch("pcg_xrz_f32_L0", 8.0 * n * 4.0, k_pcg_xrz, gf, kThreads, st, n, (const float*)pout,
              (const float*)k.q, (float*)k.e, (float*)k.r, (const float*)A.dinv, (float*)k.z, w->sc, rs);
      return;
    }
  }
  vlaunch(KN("pcg_p", true), 3.0 * n * sizeof(T), k_pcg_p<T>, gf, kThreads, st, n, (const T*)k.z, k.p,
          (const KScal*)w->sc);
  bool fused_mv = false;
  if constexpr (sizeof(T) == 4 && SYM) {
    if (A.mfc != 0.0f && !use_mg && !use_net) {  // constant-link matvec fused with p.q
      const Op<T> Z = zview(A);
      if (Z.box.mx % 4 == 0) {  // 16-byte rows: four cells per thread (fixed shape, fixed summation order)
        const ZCfg z = zcfg_mf4(Z.box);
        vlaunch("pcg_matvec_dot_mfc_f32_L0", 4.0 * n * 4.0, k_matvec_mfc4_dot, z.grid, z.block, st, Z.box,
                (const float*)Z.diag, A.mfc, (const float*)k.p, (float*)k.q, z.zc, w->sc, rs);
      } else {
        const ZCfg z = zcfg(Z.box);  // grid-reduction kernel: default shape, fixed summation order
        vlaunch("pcg_matvec_dot_mfc_f32_L0", 4.0 * n * 4.0, k_matvec_mfc_dot, z.grid, z.block, st, Z.box,
                (const float*)Z.diag, A.mfc, (const float*)k.p, (float*)k.q, z.zc, w->sc, rs);
      }
      fused_mv = true;
    } else if (A.mfe && !use_net && zview(A).box.mx % 4 == 0) {  // the same, matrix-free pressure, four cells
      const Op<T> Z = zview(A);
      const ZCfg z = zcfg_mf4(Z.box);
      vlaunch("pcg_matvec_dot_mf_f32_L0", 4.0 * n * 4.0, k_matvec_mf4_dot, z.grid, z.block, st, Z.box, A.mfe, A.mfs,
              (const float*)k.p, (float*)k.q, z.zc, w->sc, rs);
      fused_mv = true;
    } else if (A.mfe && !use_net) {  // matrix-free pressure matvec fused with p.q
      const Op<T> Z = zview(A);
      const ZCfg z = zcfg(Z.box);
      vlaunch("pcg_matvec_dot_mf_f32_L0", 4.0 * n * 4.0, k_matvec_mf_dot, z.grid, z.block, st, Z.box, A.mfe, A.mfs,
              (const float*)k.p, (float*)k.q, z.zc, w->sc, rs);
      fused_mv = true;
    }
  }
  if (!fused_mv) {
    stencil_launch<T, SYM>(KN("pcg_matvec", true), SK_MV, A, nullptr, k.p, k.q, T(0), w->sc, st);
    vlaunch(KN("dot_pq", true), 2.0 * n * sizeof(T), k_dots<T, 1, DF_PCG_ALPHA>, gf, kThreads, st, n, (const T*)k.p,
            (const T*)k.q, (const T*)nullptr, (const T*)nullptr, w->sc, rs);
  }
  // FP64 MG-PCG passes end on the scaled norm (the diagonal preconditioner
  // tests z.z itself; FP32 MG-PCG and the learned path keep |r|, see
  // scaled_test)
  const T* dscale = (sizeof(T) == 8 && use_mg && !use_net) ? (const T*)A.dinv : nullptr;
  if (use_mg && !use_net && fused_mg_pcg<T, SYM>(h)) {  // x/r update with the V-cycle's first sweep
    const Op<T> Z = zview(A);
    const ZCfg z = zcfg_mf4(Z.box);
    vlaunch("pcg_xr_jac0_mf_f32_L0", 9.0 * n * 4.0, k_xr_jac0_mf4, z.grid, z.block, st, Z.box, A.mfe, A.mfs,
            (const float*)k.p, (const float*)k.q, (float*)k.e, (float*)k.r, (float*)k.scratch, (float)h.mg.omega,
            z.zc, w->sc, rs);
    pcg_precond<T, SYM>(h, k, n, w, rs, st, use_mg, use_net, true);
    return;
  }
  vlaunch(KN("pcg_xr", true), (dscale ? 7.0 : 6.0) * n * sizeof(T), k_pcg_xr<T>, gf, kThreads, st, n, (const T*)k.p,
          (const T*)k.q, k.e, k.r, dscale, w->sc, rs);
  pcg_precond<T, SYM>(h, k, n, w, rs, st, use_mg, use_net);
}

// One BiCGStab iteration (right preconditioned, two V-cycles).
template <typename T, bool SYM>
static void bicg_iteration(Hier<T>& h, const KVec<T>& k, long long n, SolverWork* w, const RedScratch& rs,
                           cudaStream_t st) {
  const Op<T>& A = h.lev[0].op;
  const int gf = flat_grid(n);
  vlaunch(KN("bicg_p", true), 4.0 * n * sizeof(T), k_bicg_p<T>, gf, kThreads, st, n, (const T*)k.r, (const T*)k.v,
          k.p, (const KScal*)w->sc);
  vcycle<T, SYM>(h, k.p, k.ph, k.scratch, w->sc, st);
  stencil_launch<T, SYM>(KN("bicg_matvec", true), SK_MV, A, nullptr, k.ph, k.v, T(0), w->sc, st);
  vlaunch(KN("dot_rhv", true), 2.0 * n * sizeof(T), k_dots<T, 1, DF_BICG_ALPHA>, gf, kThreads, st, n, (const T*)k.rh,
          (const T*)k.v, (const T*)nullptr, (const T*)nullptr, w->sc, rs);
  vlaunch(KN("bicg_s", true), 3.0 * n * sizeof(T), k_bicg_s<T>, gf, kThreads, st, n, (const T*)k.r, (const T*)k.v, k.s,
          (const KScal*)w->sc);
  vcycle<T, SYM>(h, k.s, k.sh, k.scratch, w->sc, st);
  stencil_launch<T, SYM>(KN("bicg_matvec", true), SK_MV, A, nullptr, k.sh, k.t, T(0), w->sc, st);
  vlaunch(KN("dot_ts_tt", true), 3.0 * n * sizeof(T), k_dots<T, 2, DF_BICG_OMEGA>, gf, kThreads, st, n, (const T*)k.t,
          (const T*)k.s, (const T*)k.t, (const T*)k.t, w->sc, rs);
  vlaunch(KN("bicg_x", true), 8.0 * n * sizeof(T), k_bicg_x<T>, gf, kThreads, st, n, (const T*)k.ph, (const T*)k.sh,
          (const T*)k.s, (const T*)k.t, (const T*)k.rh, k.e, k.r, w->sc, rs);
}

// Which PCG passes end on the diagonally scaled norm (the refinement's own
// test) rather than |r|: diagonal PCG always (z.z is free), MG-PCG in FP64
// (one more read per iteration; the FP64 path is arithmetic-bound, and with
// |r| an FP64 pressure solve of the 1024 x 512 micromodel stalled at 1.7e-10
// in 8 passes).  FP32 MG-PCG keeps |r|: the scaled test cut the rock's
// pressure passes from 4.1 to 2.9 but not the iterations and the extra read
// made the step slower.
template <typename T>
static int scaled_test(bool use_mg, bool use_net) {
  return (!use_net && (!use_mg || sizeof(T) == 8)) ? 1 : 0;
}

// With the learned preconditioner (use_net) the pass stops early, with
// *stagnated = true, when the inner residual norm falls by less than a
// factor 2 over two successive polls (8 iterations): the caller then
// finishes the solve with MG-PCG.
template <typename T, bool SYM>
static int inner_pcg(Hier<T>& h, SolverWork* w, double rtol_inner, int max_iters, const RedScratch& rs,
                     cudaStream_t st, bool use_mg, bool use_net = false, bool* stagnated = nullptr) {
  const long long n = box_cells(h.lev[0].op.box);
  const KVec<T> k = kvec<T>(w, false);
  cudaMemsetAsync(k.e, 0, n * sizeof(T), st);
  vlaunch("kscal_init", 0.0, k_kscal_init, 1, 32, st, w->sc, w->outer, rtol_inner, max_iters,
          scaled_test<T>(use_mg, use_net));
  pcg_precond<T, SYM>(h, k, n, w, rs, st, use_mg, use_net);
  const int chunk = (use_mg || use_net) ? 4 : 8;
  int it = 0;
  double rr_prev = -1.0;
  int slow = 0;
  if (stagnated) *stagnated = false;
  while (true) {
    for (int c = 0; c < chunk; ++c) pcg_iteration<T, SYM>(h, k, n, w, rs, st, use_mg, use_net, c & 1);
    it += chunk;
    cudaMemcpyAsync(w->sc_host, w->sc, sizeof(KScal), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (w->sc_host->done || it >= max_iters + chunk) break;
    if (use_net) {
      const double rr = w->sc_host->rr;
      slow = (rr_prev > 0.0 && rr > 0.25 * rr_prev) ? slow + 1 : 0;
      rr_prev = rr;
      if (slow >= 2) {
        if (stagnated) *stagnated = true;
        break;
      }
    }
  }
  if (use_net && stagnated && w->sc_host->breakdown) *stagnated = true;
  return w->sc_host->iters;
}

template <typename T, bool SYM>
static int inner_bicgstab(Hier<T>& h, SolverWork* w, double rtol_inner, int max_iters, const RedScratch& rs,
                          cudaStream_t st) {
  const long long n = box_cells(h.lev[0].op.box);
  const KVec<T> k = kvec<T>(w, true);
  cudaMemsetAsync(k.e, 0, n * sizeof(T), st);
  cudaMemsetAsync(k.v, 0, n * sizeof(T), st);
  cudaMemcpyAsync(k.rh, k.r, n * sizeof(T), cudaMemcpyDeviceToDevice, st);
  vlaunch("kscal_init", 0.0, k_kscal_init, 1, 32, st, w->sc, w->outer, rtol_inner, max_iters, 0);
  const int chunk = 2;
  int it = 0;
  while (true) {
    for (int c = 0; c < chunk; ++c) bicg_iteration<T, SYM>(h, k, n, w, rs, st);
    it += chunk;
    cudaMemcpyAsync(w->sc_host, w->sc, sizeof(KScal), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (w->sc_host->done || it >= max_iters + chunk) break;
  }
  return w->sc_host->iters;
}

// ---------------------------------------------------------------------------
// Graph mode: device-side loop control
// ---------------------------------------------------------------------------
// Smallest relative tolerance asked of one FP32 inner pass (mixed path).
// Measured on the 256^3 rock: asking an FP32 MG-PCG pass for less than 2e-5
// costs more iterations than the refinement pass it saves, and 1e-6 or 1e-7
// for the diagonally preconditioned momentum passes made the step slower
// (142 vs 138 ms).
static double inner_floor32(bool use_mg) { return use_mg ? 2e-5 : kDiagFloor32; }

__global__ void k_ctrl_init(SolveStats* ss, KScal* sc) {
  VOS_COUNT_EXEC();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ss->relres = 0.0;
    ss->iters = 0;
    ss->outer = 0;
    ss->converged = 0;
    ss->zero = 0;
    ss->started = 0;
    sc->iters = 0;
    sc->done = 1;
  }
}

// Refinement controller (one thread), run after each FP64 true residual:
// decides convergence, sets the outer and inner loop conditions and
// initialises the inner Krylov scalars (the same rules as the host loop).
template <bool MIXED>
__global__ void k_ctrl(SolveStats* ss, KScal* sc, const double* outer, double rtol, int max_outer, int max_iter,
                       double floor32, int scaled, cudaGraphConditionalHandle ho, cudaGraphConditionalHandle hi) {
  VOS_COUNT_EXEC();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ss->started) ss->iters += sc->iters;
  const double rr = outer[0], bb = outer[1];
  bool stop = false;
  if (bb == 0.0) {
    ss->zero = 1;
    ss->relres = 0.0;
    ss->converged = 1;
    stop = true;
  } else {
    const double rel = sqrt(rr / bb);
    ss->relres = rel;
    if (rel <= rtol) {
      ss->converged = 1;
      stop = true;
    } else if (ss->outer >= max_outer || ss->iters >= max_iter || !isfinite(rel)) {
      ss->converged = 0;
      stop = true;
    } else {
      double rin = rtol / rel;
      if (MIXED) {
        if (rin < floor32) rin = floor32;
      } else {
        rin *= 0.5;
        if (rin < 1e-15) rin = 1e-15;
      }
      if (rin > 0.5) rin = 0.5;
      const double r2 = outer[2];
      sc->bb = r2;
      sc->rr = r2;
      sc->rz = 0.0;
      sc->rz_old = 0.0;
      sc->pq = 0.0;
      sc->alpha = 0.0;
      sc->beta = 0.0;
      sc->omega = 1.0;
      sc->rho = r2;
      sc->rhv = 0.0;
      sc->tol2 = scaled ? -1.0 : rin * rin * r2;
      sc->tol2s = rin * rin * rr;
      sc->iters = 0;
      sc->max_iters = max_iter - ss->iters;
      sc->breakdown = 0;
      sc->done = (r2 == 0.0) ? 1 : 0;
      ss->outer += 1;
      ss->started = 1;
    }
  }
  if (stop) {
    sc->done = 1;
    sc->iters = 0;
    ss->started = 0;
  }
  cudaGraphSetConditional(ho, stop ? 0u : 1u);
  cudaGraphSetConditional(hi, sc->done ? 0u : 1u);
}

__global__ void k_loop_check(const KScal* sc, cudaGraphConditionalHandle hi) {
  VOS_COUNT_EXEC();
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(hi, sc->done ? 0u : 1u);
}

// x += e, or x = 0 when the right-hand side was zero.
template <typename T>
__global__ void k_outer_update_g(Box bx, View<double> x, const T* __restrict__ e, const SolveStats* ss,
                                 float2* __restrict__ xdf, int* dfbad) {
  VOS_COUNT_EXEC();
  const bool zero = ss->zero != 0;
  const Seg s = make_seg(bx);
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    long long c = i + (long long)bx.mx * (j + (long long)bx.my * k);
    double* px = x.base + i + (long long)x.sy * j + (long long)x.sz * k;
    const double nx = zero ? 0.0 : *px + (double)e[c];
    *px = nx;
    if (xdf && !df_split(nx, xdf[c])) *dfbad = 1;  // double-FP32 copy for the next residual
  }
}

// Add a WHILE node (condition handle hnd) to the graph being captured on st
// and begin capturing its body on sb.
static cudaError_t begin_while(cudaStream_t st, cudaGraphConditionalHandle hnd, cudaStream_t sb) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  VOS_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  std::memset(pbuf, 0, sizeof(pbuf));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  VOS_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  VOS_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  VOS_CUDA_TRY(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  return cudaSuccess;
}

static cudaError_t end_body(cudaStream_t sb) {
  cudaGraph_t g;
  return cudaStreamEndCapture(sb, &g);
}

static cudaError_t capture_graph_of(cudaStream_t st, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs;
  VOS_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr));
  return cs == cudaStreamCaptureStatusActive ? cudaSuccess : cudaErrorStreamCaptureInvalidated;
}

// The double-FP32 refinement residual (after the first pass) is used by
// mixed-precision solves of symmetric systems to a tolerance of 1e-9 or
// looser: its error, a few 2^-46 of the row's terms (measured about 5e-11 of
// norm(D^-1 b) on the rock's pressure system near its solution, where the
// rows cancel by 2e4), stays well below such a tolerance (vos_set_fused_pcg
// bit 2).
template <typename T>
static bool df_residual(const Op<double>& op64, double rtol) {
  return sizeof(T) == 4 && op64.sym && rtol >= 1e-9 && (g_fused_pcg & 4) != 0;
}
// words moved per cell: b, x (and its six neighbours through L1), diagonal
// and three links as double-FP32 pairs, FP32 omega/diag in, FP32 r out
static double df_bytes(const Op<double>& A) {
  return (double)box_cells(A.box) * ((2.0 + n_offs(A) + 2.0) * 8.0 + 8.0);
}

template <typename T>
cudaError_t solve_capture(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, double rtol,
                          int max_iter, SolverWork* w, const RedScratch& rs, cudaStream_t st, bool use_mg,
                          SolveStats* ss, cudaStream_t s1, cudaStream_t s2) {
  const Box bx = op64.box;
  const long long n = box_cells(bx);
  if (n == 0) return cudaSuccess;
  const bool mixed = (sizeof(T) == 4);
  const int max_outer = mixed ? 30 : 8;
  const bool sym = h.lev[0].op.sym != 0;
  if (mixed) {
    const int links = (use_mg || !sym || h.lev[0].op.mfc == 0.0f) ? 1 : 0;
    vlaunch("op_convert", (2.0 + (links ? n_offs(op64) : 0)) * n * (8.0 + sizeof(T)), k_op_convert<T>, flat_grid(n),
            kThreads, st, op64, h.lev[0].op, n, links);
  }
  if (use_mg || !sym) build_coarse_levels<T>(h, st);
  const bool dfmode = df_residual<T>(op64, rtol);
  if (dfmode) VOS_CUDA_TRY(cudaMemsetAsync(w->dfbad, 0, sizeof(int), st));
  vlaunch("ctrl_init", 0.0, k_ctrl_init, 1, 32, st, ss, w->sc);
  cudaGraph_t g0;
  VOS_CUDA_TRY(capture_graph_of(st, &g0));
  cudaGraphConditionalHandle ho, hi;
  VOS_CUDA_TRY(cudaGraphConditionalHandleCreate(&ho, g0, 1, cudaGraphCondAssignDefault));
  VOS_CUDA_TRY(begin_while(st, ho, s1));
  {
    const Op<double> oz = zview(op64);
    const View<double> xz = zview_x(x, bx);
    const ZCfg zr = zcfg(oz.box);
    const double rbytes = (4.0 + n_offs(op64)) * n * 8.0 + n * sizeof(T);
    const int* pass = &ss->outer;  // 0 until the controller starts the first pass
    if (op64.sym)
      vlaunch("outer_residual_f64", rbytes, k_outer_residual_z<T, true>, zr.grid, zr.block, s1, oz, b, xz, (T*)w->r,
              w->outer, pass, zr.zc, rs, dfmode ? w->df : DFBuf{}, w->dfbad, dfmode ? 1 : 0);
    else
      vlaunch("outer_residual_f64", rbytes, k_outer_residual_z<T, false>, zr.grid, zr.block, s1, oz, b, xz, (T*)w->r,
              w->outer, pass, zr.zc, rs, DFBuf{}, w->dfbad, 0);
    if (dfmode)
      vlaunch("outer_residual_df", df_bytes(op64), k_outer_residual_df<T>, zr.grid, zr.block, s1, w->df,
              (const float*)h.lev[0].op.dinv, oz, b, xz, (T*)w->r, w->outer, pass, (const int*)w->dfbad, zr.zc, rs);
    cudaGraph_t g1;
    VOS_CUDA_TRY(capture_graph_of(s1, &g1));
    VOS_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, g1, 0, cudaGraphCondAssignDefault));
    if (mixed)
      vlaunch("ctrl", 0.0, k_ctrl<true>, 1, 32, s1, ss, w->sc, (const double*)w->outer, rtol, max_outer, max_iter,
              inner_floor32(use_mg), sym ? scaled_test<T>(use_mg, false) : 0, ho, hi);
    else
      vlaunch("ctrl", 0.0, k_ctrl<false>, 1, 32, s1, ss, w->sc, (const double*)w->outer, rtol, max_outer, max_iter,
              inner_floor32(use_mg), sym ? scaled_test<T>(use_mg, false) : 0, ho, hi);
    const KVec<T> k = kvec<T>(w, !sym);
    VOS_CUDA_TRY(cudaMemsetAsync(k.e, 0, n * sizeof(T), s1));
    if (sym) {
      if (h.lev[0].op.sym) pcg_precond<T, true>(h, k, n, w, rs, s1, use_mg);
    } else {
      VOS_CUDA_TRY(cudaMemsetAsync(k.v, 0, n * sizeof(T), s1));
      VOS_CUDA_TRY(cudaMemcpyAsync(k.rh, k.r, n * sizeof(T), cudaMemcpyDeviceToDevice, s1));
    }
    VOS_CUDA_TRY(begin_while(s1, hi, s2));
    if (sym) {
      for (int c = 0; c < 2; ++c) pcg_iteration<T, true>(h, k, n, w, rs, s2, use_mg, false, c);
    } else {
      bicg_iteration<T, false>(h, k, n, w, rs, s2);
    }
    vlaunch("loop_check", 0.0, k_loop_check, 1, 32, s2, (const KScal*)w->sc, hi);
    VOS_CUDA_TRY(end_body(s2));
    vlaunch("outer_update", (double)n * (sizeof(T) + 16.0), k_outer_update_g<T>, grid_for(bx, 0), kThreads, s1, bx, x,
            (const T*)k.e, (const SolveStats*)ss, dfmode ? w->df.x : (float2*)nullptr, w->dfbad);
  }
  VOS_CUDA_TRY(end_body(s1));
  return cudaGetLastError();
}

template cudaError_t solve_capture<double>(const Op<double>&, Hier<double>&, const double*, View<double>, double, int,
                                           SolverWork*, const RedScratch&, cudaStream_t, bool, SolveStats*,
                                           cudaStream_t, cudaStream_t);
template cudaError_t solve_capture<float>(const Op<double>&, Hier<float>&, const double*, View<double>, double, int,
                                          SolverWork*, const RedScratch&, cudaStream_t, bool, SolveStats*,
                                          cudaStream_t, cudaStream_t);

template <typename T>
SolveResult solve(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, double rtol, int max_iter,
                  SolverWork* w, const RedScratch& rs, cudaStream_t st, bool use_mg) {
  SolveResult res{0, 0, 0.0, 1, 0, 0};
  const Box bx = op64.box;
  const long long n = box_cells(bx);
  if (n == 0) return res;
  const bool mixed = (sizeof(T) == 4);
  const int max_outer = mixed ? 30 : 8;
  bool use_net = use_mg && h.net != nullptr && op64.sym;
  const int g = grid_for(bx, 0);
  if (mixed) {
    vlaunch("op_convert", (2.0 + n_offs(op64)) * n * (8.0 + sizeof(T)), k_op_convert<T>, flat_grid(n), kThreads, st, op64, h.lev[0].op, n, 1);
  }
  if (use_mg) build_coarse_levels<T>(h, st);
  int total = 0;
  const double rbytes = (4.0 + n_offs(op64)) * n * 8.0 + n * sizeof(T);
  const Op<double> oz = zview(op64);
  const View<double> xz = zview_x(x, bx);
  const ZCfg zr = zcfg(oz.box);
  const bool dfmode = df_residual<T>(op64, rtol);
  if (dfmode) cudaMemsetAsync(w->dfbad, 0, sizeof(int), st);
  for (int outer = 0;; ++outer) {
    if (dfmode && outer > 0)
      vlaunch("outer_residual_df", df_bytes(op64), k_outer_residual_df<T>, zr.grid, zr.block, st, w->df,
              (const float*)h.lev[0].op.dinv, oz, b, xz, (T*)w->r, w->outer, (const int*)nullptr,
              (const int*)w->dfbad, zr.zc, rs);
    else if (op64.sym)
      vlaunch("outer_residual_f64", rbytes, k_outer_residual_z<T, true>, zr.grid, zr.block, st, oz, b, xz, (T*)w->r,
              w->outer, (const int*)nullptr, zr.zc, rs, dfmode ? w->df : DFBuf{}, w->dfbad, 0);
    else
      vlaunch("outer_residual_f64", rbytes, k_outer_residual_z<T, false>, zr.grid, zr.block, st, oz, b, xz, (T*)w->r,
              w->outer, (const int*)nullptr, zr.zc, rs, DFBuf{}, w->dfbad, 0);
    cudaMemcpyAsync(w->outer_host, w->outer, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const double rr = w->outer_host[0], bb = w->outer_host[1];
    if (bb == 0.0) {
      vlaunch("view_zero", 8.0 * n, k_view_zero, g, kThreads, st, bx, x);
      res.relres = 0.0;
      res.outer = outer;
      break;
    }
    const double rel = std::sqrt(rr / bb);
    res.relres = rel;
    res.outer = outer;
    if (rel <= rtol) break;
    if (outer >= max_outer || total >= max_iter || !std::isfinite(rel)) {
      res.converged = 0;
      break;
    }
    // Inner relative tolerance: just what the outer target needs, but not
    // below 2e-5 in the mixed path (measured: asking an FP32 solve for 1e-6
    // costs more Krylov iterations than the extra refinement pass it saves);
    // the FP64 path asks for a little more than needed.
    double rin = rtol / rel;
    if (mixed) {
      if (rin < inner_floor32(use_mg)) rin = inner_floor32(use_mg);
    } else {
      rin *= 0.5;
      if (rin < 1e-15) rin = 1e-15;
    }
    if (rin > 0.5) rin = 0.5;
    int left = max_iter - total;
    int its;
    if (h.lev[0].op.sym) {
      bool stag = false;
      its = inner_pcg<T, true>(h, w, rin, left, rs, st, use_mg, use_net, &stag);
      if (use_net) {
        res.net_iters += its;
        if (stag) {  // the learned preconditioner stalled: MG-PCG from here on
          use_net = false;
          res.fallback = 1;
        }
      }
    } else {
      its = inner_bicgstab<T, false>(h, w, rin, left, rs, st);
    }
    total += its;
    vlaunch("outer_update", (double)n * (sizeof(T) + 16.0), k_outer_update<T>, g, kThreads, st, bx, x, (const T*)w->e,
            dfmode ? w->df.x : (float2*)nullptr, w->dfbad);
  }
  res.iters = total;
  return res;
}

template <typename T>
__global__ void k_to_float(long long n, const T* __restrict__ src, float* __restrict__ dst) {
  VOS_COUNT_EXEC();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    dst[c] = (float)src[c];
}

// Residuals of MG-PCG (multigrid + deflation, no learned preconditioner) on
// A e = b from e = 0 after iters[i] iterations (0 = b itself), written as
// FP32 to out + i * n.  x must be a zero vector of the box (scratch).
template <typename T>
int residual_snapshots(const Op<double>& op64, Hier<T>& h, const double* b, View<double> x, SolverWork* w,
                       const RedScratch& rs, cudaStream_t st, int count, const int* iters, float* out) {
  const Box bx = op64.box;
  const long long n = box_cells(bx);
  if (sizeof(T) == 4)
    vlaunch("op_convert", 0.0, k_op_convert<T>, flat_grid(n), kThreads, st, op64, h.lev[0].op, n, 1);
  build_coarse_levels<T>(h, st);
  const Op<double> oz = zview(op64);
  const View<double> xz = zview_x(x, bx);
  const ZCfg zr = zcfg(oz.box);
  vlaunch("outer_residual_f64", 0.0, k_outer_residual_z<T, true>, zr.grid, zr.block, st, oz, b, xz, (T*)w->r,
          w->outer, (const int*)nullptr, zr.zc, rs, DFBuf{}, w->dfbad, 0);
  int maxit = 0;
  for (int i = 0; i < count; ++i) maxit = iters[i] > maxit ? iters[i] : maxit;
  const KVec<T> k = kvec<T>(w, false);
  cudaMemsetAsync(k.e, 0, n * sizeof(T), st);
  vlaunch("kscal_init", 0.0, k_kscal_init, 1, 32, st, w->sc, w->outer, 1e-30, maxit + 1, 0);
  pcg_precond<T, true>(h, k, n, w, rs, st, true, false);
  for (int it = 0; it <= maxit; ++it) {
    if (it > 0) pcg_iteration<T, true>(h, k, n, w, rs, st, true, false, (it - 1) & 1);
    for (int i = 0; i < count; ++i)
      if (iters[i] == it)
        vlaunch("to_float", 0.0, k_to_float<T>, flat_grid(n), kThreads, st, n, (const T*)k.r, out + (long long)i * n);
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}
template int residual_snapshots<double>(const Op<double>&, Hier<double>&, const double*, View<double>, SolverWork*,
                                        const RedScratch&, cudaStream_t, int, const int*, float*);
template int residual_snapshots<float>(const Op<double>&, Hier<float>&, const double*, View<double>, SolverWork*,
                                       const RedScratch&, cudaStream_t, int, const int*, float*);

template SolveResult solve<double>(const Op<double>&, Hier<double>&, const double*, View<double>, double, int,
                                   SolverWork*, const RedScratch&, cudaStream_t, bool);
template SolveResult solve<float>(const Op<double>&, Hier<float>&, const double*, View<double>, double, int,
                                  SolverWork*, const RedScratch&, cudaStream_t, bool);

}  // namespace vos
