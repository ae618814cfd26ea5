// Physics kernels of one VoS time step (FP64 fields, MAC-staggered grid).
//
// Cell (i,j,k) -> i + nx*(j + ny*k).  Face arrays of axis a have one more
// entry along a; face index m along a separates cells m-1 and m.
#include <cmath>

#include "vos_phys.cuh"

namespace vos {

// Kernel executions of this file (see VOS_COUNT_EXEC).
static __device__ unsigned long long vos_exec_count = 0;
unsigned long long exec_count_fields() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}


namespace {

__device__ __forceinline__ long long cidx(const Phys& P, int i, int j, int k) {
  return i + (long long)P.nx * (j + (long long)P.ny * k);
}
__device__ __forceinline__ int fdim(const Phys& P, int a, int b) {
  int n = (b == 0) ? P.nx : (b == 1) ? P.ny : P.nz;
  return n + (a == b ? 1 : 0);
}
__device__ __forceinline__ long long fidx(const Phys& P, int a, int i, int j, int k) {
  return i + (long long)fdim(P, a, 0) * (j + (long long)fdim(P, a, 1) * k);
}
__device__ __forceinline__ int ncell(const Phys& P, int b) { return (b == 0) ? P.nx : (b == 1) ? P.ny : P.nz; }

// omega / diag for the Jacobi smoother, the diagonal preconditioner and the
// scaled residual norm (within a couple of ulp of the IEEE quotient; an FP32
// reciprocal here, 6e-8 off, is too coarse for the FP64 solves).
__device__ __forceinline__ double jacobi_weight(double omega, double diag) { return fdiv_nr(omega, diag); }

// Kozeny-Carman inverse permeability (Eq. perm): (1 - eps)^2 / (k0 eps^3).
__device__ __forceinline__ double kinv(double e, double k0) {
  double s = 1.0 - e;
  return fdiv_nr(s * s, k0 * e * e * e);
}

// |x| <= 1e-300 on the bit pattern (no FP64 instruction): the magnitude bits
// of a double order like its absolute value.
__device__ __forceinline__ bool tiny300(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) <= 0x01a56e1fc2f8f359LL;  // bits of 1e-300
}

// van Leer correction of a face value, c_f = c_U + w (c_D - c_U): w = psi(r)/2
// with psi(r) = (r + |r|)/(1 + |r|), r = a/b, a = c_U - c_UU, b = c_D - c_U.
// For r > 0 (a, b non-zero with one sign) psi(r)/2 = r/(1 + r) = a/(a + b),
// so w b = a b / (a + b); psi = 0 otherwise, without a far-upwind cell, or
// for |b| <= 1e-300.  Returns w b; the sign and magnitude tests run on the
// bit patterns (FP64 instructions are the bottleneck of these kernels).
__device__ __forceinline__ double vl_corr(double cUU, double cU, double cD, bool has) {
  const double b = cD - cU;
  if (!has || tiny300(b)) return 0.0;
  const double a = cU - cUU;
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if ((ia ^ ib) < 0 || (ia << 1) == 0) return 0.0;  // a b <= 0
  return fdiv_nr(a * b, a + b);
}

// eps difference across a cell along b (zero-gradient ghosts): 2 dx times the
// centred gradient component
__device__ __forceinline__ double cdiff(const Phys& P, const double* eps, int b, int i, int j, int k) {
  int n = ncell(P, b);
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  lo[b] = lo[b] > 0 ? lo[b] - 1 : 0;
  hi[b] = hi[b] + 1 < n ? hi[b] + 1 : n - 1;
  return eps[cidx(P, hi[0], hi[1], hi[2])] - eps[cidx(P, lo[0], lo[1], lo[2])];
}

// centred gradient component b of eps at a cell, zero-gradient ghosts
__device__ __forceinline__ double cgrad(const Phys& P, const double* eps, int b, int i, int j, int k) {
  int n = ncell(P, b);
  int c[3] = {i, j, k};
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  lo[b] = c[b] > 0 ? c[b] - 1 : 0;
  hi[b] = c[b] + 1 < n ? c[b] + 1 : n - 1;
  return (eps[cidx(P, hi[0], hi[1], hi[2])] - eps[cidx(P, lo[0], lo[1], lo[2])]) * (0.5 / P.dx);
}

__device__ __forceinline__ bool cell_in(const Phys& P, int i, int j, int k) {
  return i >= 0 && i < P.nx && j >= 0 && j < P.ny && k >= 0 && k < P.nz;
}

}  // namespace

// ---------------------------------------------------------------------------
// S1: eps^{n+1} = clamp(eps^n + dt Vm R^n, eps_min, 1)   (Eq. mbs)
// ---------------------------------------------------------------------------
__global__ void k_eps_update(Phys P, double* eps, double* eps_old, const double* R, const double* __restrict__ dtp, double* stats,
                             RedScratch rs, double* __restrict__ kic) {
  VOS_COUNT_EXEC();
  const double dt = *dtp;
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  double acc[2] = {0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    long long c = cidx(P, i, j, k);
    double e = eps[c];
    eps_old[c] = e;
    double raw = e + dt * P.Vm * R[c];
    double nw = fmin(fmax(raw, P.eps_min), 1.0);
    eps[c] = nw;
    kic[c] = kinv(nw, P.k0);  // Kozeny-Carman k^-1 of the new eps, once per cell
    acc[0] += raw - nw;
    acc[1] += nw;
  }
  if (grid_sum<2>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    double V = (P.dim == 2) ? P.dx * P.dx : P.dx * P.dx * P.dx;
    stats[ST_CLAMP] = acc[0] * V;
    stats[ST_EPSSUM] = acc[1];
  }
}

void launch_eps_update(const Phys& P, double* eps, double* eps_old, const double* R, const double* __restrict__ dtp, double* stats,
                       const RedScratch& rs, double* kic, cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  vlaunch("eps_update", 40.0 * box_cells(bx), k_eps_update, grid_for(bx, kMaxRedBlocks), kThreads, st, P, eps, eps_old, R, dtp, stats, rs, kic);
}

// ---------------------------------------------------------------------------
// Inertia term of Eq. momentumDBS (multiplied by eps): N_a = div(u u_a / eps)
// on the staggered control volume (CV) of an a-face, finite volumes with the
// transported quantity phi = u_a / eps_f (eps_f: mean of the two cells of an
// interior face, the adjacent cell of a boundary face) taken by van Leer
// upwinding (App. B) at each CV face and carried by the advecting velocity:
//   b = a: CV faces at cell centres, U = mean of the cell's two a-faces;
//   b != a: CV faces on cell edges, U = mean of the two b-faces meeting
//           there (one for the outlet a-face).
// Domain boundary: no flux through walls / free-slip sides (no normal
// velocity) nor through the inlet plane's edges (no tangential velocity);
// outlet-plane edges take the upwind interior value; the outlet face's CV
// loses u_n phi_n past the outlet.  Explicit in time (u at t^n).
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ double face_eps(const Phys& P, const double* eps, int a, const int g[3]) {
  const int m = g[a], n = ncell(P, a);
  int lo[3] = {g[0], g[1], g[2]};
  lo[a] -= 1;
  if (m == 0) return eps[cidx(P, g[0], g[1], g[2])];
  if (m == n) return eps[cidx(P, lo[0], lo[1], lo[2])];
  return 0.5 * (eps[cidx(P, lo[0], lo[1], lo[2])] + eps[cidx(P, g[0], g[1], g[2])]);
}
__device__ __forceinline__ double phi_face(const Phys& P, const double* eps, const double* ua, int a, const int g[3]) {
  return fdiv_nr(ua[fidx(P, a, g[0], g[1], g[2])], face_eps(P, eps, a, g));
}
// van Leer value of phi between a-faces q and q+1 along d (nq a-faces along
// d; the other coordinates from f), upwind of U
__device__ double phi_between(const Phys& P, const double* eps, const double* ua, int a, const int f[3], int d, int q,
                              int nq, double U) {
  int g[3] = {f[0], f[1], f[2]};
  int qu, qd, quu;
  bool has;
  if (U >= 0.0) {
    qu = q;
    qd = q + 1;
    quu = q - 1;
    has = quu >= 0;
  } else {
    qu = q + 1;
    qd = q;
    quu = q + 2;
    has = quu < nq;
  }
  g[d] = qu;
  const double cU = phi_face(P, eps, ua, a, g);
  g[d] = qd;
  const double cD = phi_face(P, eps, ua, a, g);
  double cUU = cU;
  if (has) {
    g[d] = quu;
    cUU = phi_face(P, eps, ua, a, g);
  }
  return cU + vl_corr(cUU, cU, cD, has);
}
__device__ double inertia_term(const Phys& P, const double* eps, const double* const us[3], int a, const int f[3]) {
  const double* ua = us[a];
  const int m = f[a], na = ncell(P, a);
  const int nb = (P.dim == 2) ? 2 : 3;
  double N = 0.0;
  {  // b = a
    int g[3] = {f[0], f[1], f[2]};
    double Fp;
    const double uf = ua[fidx(P, a, f[0], f[1], f[2])];
    if (m < na) {
      g[a] = m + 1;
      const double U = 0.5 * (uf + ua[fidx(P, a, g[0], g[1], g[2])]);
      Fp = U * phi_between(P, eps, ua, a, f, a, m, na + 1, U);
    } else {  // outlet face
      Fp = uf * phi_face(P, eps, ua, a, f);
    }
    g[a] = m - 1;
    const double U = 0.5 * (ua[fidx(P, a, g[0], g[1], g[2])] + uf);
    const double Fm = U * phi_between(P, eps, ua, a, f, a, m - 1, na + 1, U);
    N += Fp - Fm;
  }
  for (int b = 0; b < nb; ++b) {
    if (b == a) continue;
    const double* ub = us[b];
    const int nbc = ncell(P, b), jb = f[b];
    // advecting velocity at the edge on b-face eb: u_b over the a-face's cells
    auto Uedge = [&](int eb) {
      int g[3] = {f[0], f[1], f[2]};
      g[b] = eb;
      g[a] = m - 1;
      double s = ub[fidx(P, b, g[0], g[1], g[2])];
      if (m < na) {
        g[a] = m;
        s = 0.5 * (s + ub[fidx(P, b, g[0], g[1], g[2])]);
      }
      return s;
    };
    double Fp = 0.0, Fm = 0.0;
    if (jb + 1 < nbc) {
      const double U = Uedge(jb + 1);
      Fp = U * phi_between(P, eps, ua, a, f, b, jb, nbc, U);
    } else if (b == 0) {  // outlet-plane edge: upwind interior value
      Fp = Uedge(nbc) * phi_face(P, eps, ua, a, f);
    }
    if (jb >= 1) {
      const double U = Uedge(jb);
      Fm = U * phi_between(P, eps, ua, a, f, b, jb - 1, nbc, U);
    }
    N += Fp - Fm;
  }
  return N / P.dx;
}
}  // namespace

// ---------------------------------------------------------------------------
// S2: momentum predictor for component a (Eq. momentumDBS x eps; the inertia
// term explicit when P.inertia is set, else dropped)
//   (1/dt + nu eps_f k^-1_f) u_f - nu lap(u)_f = u^n_f/dt - eps_f (grad p^n)_f
// Unknown box: the faces of a except the fixed ones (inlet face for x,
// boundary faces for y/z); unknown (i,j,k) is face (i,j,k) + e_a, whose
// minus cell is cell (i,j,k).
// ---------------------------------------------------------------------------
__global__ void k_mom_assemble(Phys P, int a, Box ub, const double* __restrict__ eps, const double* __restrict__ kic,
                               const double* __restrict__ p, const double* __restrict__ uold,
                               const double* __restrict__ dtp, const double* __restrict__ u0,
                               const double* __restrict__ u1, const double* __restrict__ u2, double omega,
                               Op<double> A, double* __restrict__ rhs) {
  VOS_COUNT_EXEC();
  const double idt = 1.0 / *dtp, idx = 1.0 / P.dx;
  const Seg s = make_seg(ub);
  const double cnu = P.nu / (P.dx * P.dx);
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, ub, q, i, j, k);
    if (i >= ub.mx) continue;
    const long long c = i + (long long)ub.mx * (j + (long long)ub.my * k);
    int f[3] = {i, j, k};
    f[a] += 1;  // face coordinates
    int pc[3] = {i, j, k};
    pc[a] += 1;  // plus cell
    const bool has_plus = pc[a] < ncell(P, a);
    const double em = eps[cidx(P, i, j, k)];
    const double pm = p[cidx(P, i, j, k)];
    double ef, kf, gp;
    if (has_plus) {
      const long long cp = cidx(P, pc[0], pc[1], pc[2]);
      const double ep = eps[cp];
      ef = 0.5 * (em + ep);
      kf = 0.5 * (kic[cidx(P, i, j, k)] + kic[cp]);
      gp = (p[cp] - pm) * idx;
    } else {  // outlet face (a == x): one-sided, Dirichlet p = 0
      ef = em;
      kf = kic[cidx(P, i, j, k)];
      gp = -2.0 * pm * idx;
    }
    double b = uold[fidx(P, a, f[0], f[1], f[2])] * idt - ef * gp;
    if (P.inertia) {
      const double* us3[3] = {u0, u1, u2};
      b -= inertia_term(P, eps, us3, a, f);
    }
    // the viscous part of the diagonal counts its cnu terms in integers:
    // one per unknown or fixed neighbour, two per antisymmetric ghost
    // (no-slip wall, inlet tangential), none per zero-gradient ghost
    int nvis = 0;
    double off[3] = {0.0, 0.0, 0.0};
    const int nb = (P.dim == 2) ? 2 : 3;
    const int um[3] = {ub.mx, ub.my, ub.mz};
    for (int d = 0; d < nb; ++d) {
      for (int sg = -1; sg <= 1; sg += 2) {
        int u2[3] = {i, j, k};
        u2[d] += sg;
        if (u2[d] >= 0 && u2[d] < um[d]) {  // unknown neighbour
          ++nvis;
          if (sg > 0) off[d] = -cnu;
          continue;
        }
        int f2 = f[d] + sg;  // neighbour face coordinate along d
        if (f2 >= 0 && f2 < fdim(P, a, d)) {  // fixed boundary face
          ++nvis;
          if (a == 0 && d == 0 && f2 == 0) b += cnu * P.u_in;
        } else {  // ghost outside the face array
          bool anti;
          if (d == 0) {
            anti = (sg < 0);  // inlet plane: tangential 0; outlet: zero gradient
          } else {
            unsigned bit = (d == 1) ? (sg < 0 ? 1u : 2u) : (sg < 0 ? 4u : 8u);
            anti = (P.wall_mask & bit) != 0;
          }
          if (anti) nvis += 2;
        }
      }
    }
    const double diag = fma((double)nvis, cnu, fma(P.nu * ef, kf, idt));
    A.diag[c] = diag;
    A.dinv[c] = jacobi_weight(omega, diag);
    A.xp[c] = off[0];
    A.yp[c] = off[1];
    if (A.zp) A.zp[c] = off[2];
    rhs[c] = b;
  }
}

void launch_mom_assemble(const Phys& P, int a, const double* eps, const double* kic, const double* p, const double* uold,
                         const double* __restrict__ dtp, double* const u[3], double omega, Op<double> A, double* rhs,
                         cudaStream_t st) {
  if (box_cells(A.box) == 0) return;
  vlaunch("mom_assemble", (6.0 + P.dim + (P.inertia ? P.dim : 0)) * 8.0 * box_cells(A.box), k_mom_assemble,
          grid_for(A.box, 0), kThreads, st, P, a, A.box, eps, kic, p, uold, dtp, (const double*)u[0],
          (const double*)(u[1] ? u[1] : u[0]), (const double*)(u[2] ? u[2] : u[0]), omega, A, rhs);
}

// ---------------------------------------------------------------------------
// S3: pressure correction  -div(eps_f grad phi) = -(div u* - s)/dt
// (Eq. contDBS, s = R Vm (1 - rho_s/rho)); Neumann at inlet and walls,
// phi = 0 on the outlet faces.
// ---------------------------------------------------------------------------
__global__ void k_pres_assemble(Phys P, const double* __restrict__ eps, const double* __restrict__ u0,
                                const double* __restrict__ u1, const double* __restrict__ u2,
                                const double* __restrict__ R, const double* __restrict__ dtp, double omega, Op<double> A,
                                double* __restrict__ rhs, float* __restrict__ eps32) {
  VOS_COUNT_EXEC();
  const double idt = 1.0 / *dtp, idx = 1.0 / P.dx;
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const double idx2 = 1.0 / (P.dx * P.dx);
  const int nb = (P.dim == 2) ? 2 : 3;
  const double* us[3] = {u0, u1, u2};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c = cidx(P, i, j, k);
    const double e = eps[c];
    // diagonal = sum of the links a_n = (e + e_n) idx2 / 2 (plus 2 e idx2 on
    // the outlet column), formed as (n e + sum e_n) idx2 / 2 with the
    // neighbours summed first; plus links stored one by one
    double off[3] = {0.0, 0.0, 0.0}, esum = 0.0, dsum = 0.0;
    int nl = 0;
    for (int d = 0; d < nb; ++d) {
      int lo[3] = {i, j, k}, hi[3] = {i, j, k};
      lo[d] -= 1;
      hi[d] += 1;
      if (cell_in(P, hi[0], hi[1], hi[2])) {
        const double en = eps[cidx(P, hi[0], hi[1], hi[2])];
        off[d] = -0.5 * (e + en) * idx2;
        esum += en;
        ++nl;
      }
      if (cell_in(P, lo[0], lo[1], lo[2])) {
        esum += eps[cidx(P, lo[0], lo[1], lo[2])];
        ++nl;
      }
      int fp[3] = {i, j, k};
      fp[d] += 1;
      dsum += us[d][fidx(P, d, fp[0], fp[1], fp[2])] - us[d][fidx(P, d, i, j, k)];
    }
    double diag = 0.5 * idx2 * fma((double)nl, e, esum);
    if (i == P.nx - 1) diag += 2.0 * e * idx2;
    const double div = dsum * idx;
    const double src = R[c] * P.Vm * (1.0 - P.rho_ratio);
    A.diag[c] = diag;
    A.dinv[c] = jacobi_weight(omega, diag);
    if (eps32) eps32[c] = f32_rn(e);  // the matrix-free FP32 form of this operator
    A.xp[c] = off[0];
    A.yp[c] = off[1];
    if (A.zp) A.zp[c] = off[2];
    rhs[c] = -(div - src) * idt;
  }
}

void launch_pres_assemble(const Phys& P, const double* eps, double* const us[3], const double* R, const double* __restrict__ dtp,
                          double omega, Op<double> A, double* rhs, float* eps32, cudaStream_t st) {
  vlaunch("pres_assemble", (5.0 + 2.0 * P.dim) * 8.0 * box_cells(A.box), k_pres_assemble, grid_for(A.box, 0), kThreads, st, P, eps, us[0], us[1], us[2], R, dtp, omega, A, rhs, eps32);
}

// u^{n+1} = u* - dt eps_f grad phi on interior faces and the outlet face;
// fixed faces copy u*.  SUMS: also reduce sum (u^{n+1} - u^{old})^2 and
// sum (u^{n+1})^2 into sums[0], sums[1] (u^{old} is the value overwritten).
template <bool SUMS>
__global__ void k_project(Phys P, int a, Box fb, const double* __restrict__ eps, const double* __restrict__ phi,
                          const double* __restrict__ dtp, const double* __restrict__ us, double* __restrict__ u,
                          double* sums, RedScratch rs) {
  VOS_COUNT_EXEC();
  const double dt = *dtp, idx = 1.0 / P.dx;
  const Seg s = make_seg(fb);
  double acc[2] = {0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, fb, q, i, j, k);
    if (i >= fb.mx) continue;
    const long long fcx = i + (long long)fb.mx * (j + (long long)fb.my * k);
    int f[3] = {i, j, k};
    const int m = f[a], n = ncell(P, a);
    double val = us[fcx];
    if (m >= 1 && m <= n - 1) {
      int mc[3] = {i, j, k};
      mc[a] -= 1;
      const long long cm = cidx(P, mc[0], mc[1], mc[2]), cp = cidx(P, i, j, k);
      val -= dt * 0.5 * (eps[cm] + eps[cp]) * (phi[cp] - phi[cm]) * idx;
    } else if (a == 0 && m == n) {
      const long long cm = cidx(P, i - 1, j, k);
      val -= dt * eps[cm] * (-2.0 * phi[cm]) * idx;
    }
    if (SUMS) {
      const double du = val - u[fcx];
      acc[0] += du * du;
      acc[1] += val * val;
    }
    u[fcx] = val;
  }
  if (SUMS) {
    if (grid_sum<2>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
      sums[0] = acc[0];
      sums[1] = acc[1];
    }
  }
}

template <bool DIFF>
__global__ void k_qs_sums(long long n, const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ w, double* out, RedScratch rs) {
  VOS_COUNT_EXEC();
  double acc[2] = {0.0, 0.0};
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double wc = w ? w[c] : 1.0;
    const double d = DIFF ? x[c] - y[c] : y[c];
    acc[0] += wc * d * d;
    acc[1] += wc * x[c] * x[c];
  }
  if (grid_sum<2>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

void launch_qs_sums(long long n, bool diff, const double* x, const double* y, const double* w, double* out,
                    const RedScratch& rs, cudaStream_t st) {
  long long g = (n + kThreads - 1) / kThreads;
  const long long cap = (long long)g_num_sms * 8 < kMaxRedBlocks ? (long long)g_num_sms * 8 : kMaxRedBlocks;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  if (diff)
    vlaunch("qs_sums", 24.0 * n, k_qs_sums<true>, (int)g, kThreads, st, n, x, y, w, out, rs);
  else
    vlaunch("qs_sums", 24.0 * n, k_qs_sums<false>, (int)g, kThreads, st, n, x, y, w, out, rs);
}

__global__ void k_add(long long n, double* __restrict__ p, const double* __restrict__ phi) {
  VOS_COUNT_EXEC();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    p[c] += phi[c];
}

void launch_project(const Phys& P, const double* eps, const double* phi, const double* __restrict__ dtp, double* const us[3],
                    double* const u[3], double* p, cudaStream_t st) {
  const int nb = (P.dim == 2) ? 2 : 3;
  for (int a = 0; a < nb; ++a) {
    Box fb{P.nx + (a == 0), P.ny + (a == 1), P.nz + (a == 2)};
    vlaunch("project", 32.0 * box_cells(fb), k_project<false>, grid_for(fb, 0), kThreads, st, P, a, fb, eps, phi, dtp,
            us[a], u[a], (double*)nullptr, RedScratch{nullptr, nullptr});
  }
  long long n = (long long)P.nx * P.ny * P.nz;
  vlaunch("p_update", 24.0 * n, k_add, grid_for(Box{P.nx, P.ny, P.nz}, 0), kThreads, st, n, p, phi);
}

void launch_project_sums(const Phys& P, const double* eps, const double* phi, const double* __restrict__ dtp,
                         double* const us[3], double* const u[3], double* p, double* stats, const RedScratch& rs,
                         cudaStream_t st) {
  const int nb = (P.dim == 2) ? 2 : 3;
  for (int a = 0; a < 3; ++a) {
    if (a >= nb) {
      launch_set_scalar(stats + ST_QSU + 2 * a, 0.0, st);
      launch_set_scalar(stats + ST_QSU + 2 * a + 1, 0.0, st);
      continue;
    }
    Box fb{P.nx + (a == 0), P.ny + (a == 1), P.nz + (a == 2)};
    vlaunch("project", 40.0 * box_cells(fb), k_project<true>, grid_for(fb, 0), kThreads, st, P, a, fb, eps, phi, dtp,
            us[a], u[a], stats + ST_QSU + 2 * a, rs);
  }
  long long n = (long long)P.nx * P.ny * P.nz;
  vlaunch("p_update", 24.0 * n, k_add, grid_for(Box{P.nx, P.ny, P.nz}, 0), kThreads, st, n, p, phi);
}

// ---------------------------------------------------------------------------
// Per-face data of the transport step, one launch per axis.
// Every face: the explicit convective flux (per unit area) of c^n with the
// van Leer face value upwinded along sign(u_f) (Eq. concentrationDBS,
// App. B), evaluated once per face here instead of once from each of the two
// adjacent cells.
// iVoS interior faces along a (Sec. 2.3, App. B):
//   g_f = ((eps_+ - eps_-)/dx along a; tangential: mean of the two cells'
//   centred gradients), n_a = -g_a / (|g_f| + 1e-8/dx),
//   s = k_c n_a / dx  (reactive flux per unit volume per unit c_f),
//   corr = w(c^n) (c_D^n - c_U^n): the van Leer correction of the face
//          value from the previous concentration (deferred correction:
//          c_f = c_U^{n+1} + corr keeps the implicit matrix an upwind
//          M-matrix),
//   evl = van Leer interpolation of eps along the flux direction.
// FP64 arithmetic is scarce on this part, so the square root and division
// of n_a are skipped where the eps gradient vanishes (pore and solid
// interiors): there g2 = 0, the normal difference dn = 0 and n_a = -0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double conv_flux(const Phys& P, int a, int i, int j, int k, const double* cold,
                                            const double* ua) {
  // flux through face (i,j,k) of axis a (face coords), per unit area
  int f[3] = {i, j, k};
  const int m = f[a], n = ncell(P, a);
  const double uf = ua[fidx(P, a, i, j, k)];
  if (m == 0) return (a == 0) ? uf * P.c_in : 0.0;
  if (m == n) return (a == 0) ? uf * cold[cidx(P, (a == 0) ? i - 1 : i, j, k)] : 0.0;
  int mc[3] = {i, j, k};
  mc[a] -= 1;
  const long long cm = cidx(P, mc[0], mc[1], mc[2]), cp = cidx(P, i, j, k);
  const bool pos = uf >= 0.0;
  int uu[3] = {i, j, k};
  long long cU, cD;
  bool has;
  if (pos) {
    cU = cm;
    cD = cp;
    uu[a] = m - 2;
    has = m - 2 >= 0;
  } else {
    cU = cp;
    cD = cm;
    uu[a] = m + 1;
    has = m + 1 <= n - 1;
  }
  const double vU = cold[cU], vD = cold[cD];
  const double vUU = has ? cold[cidx(P, uu[0], uu[1], uu[2])] : vU;
  return uf * (vU + vl_corr(vUU, vU, vD, has));
}

// Convective flux of every face of axis a (VoS-psi methods: no per-face
// reactive data).
__global__ void k_face_flux(Phys P, int a, Box fb, const double* __restrict__ cold, const double* __restrict__ ua,
                            double* __restrict__ cf) {
  VOS_COUNT_EXEC();
  const Seg s = make_seg(fb);
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, fb, q, i, j, k);
    if (i >= fb.mx) continue;
    cf[i + (long long)fb.mx * (j + (long long)fb.my * k)] = conv_flux(P, a, i, j, k, cold, ua);
  }
}

// iVoS data of one interface face (i, j, k) of axis a: interior along a, with
// a non-zero normal eps difference.
__device__ __forceinline__ void ivos_face(const Phys& P, int a, const Box& fb, int i, int j, int k, double kcx,
                                          const double* __restrict__ eps, const double* __restrict__ cold,
                                          const FaceData& fd) {
  const int nb = (P.dim == 2) ? 2 : 3;
  const int n = ncell(P, a);
  int f[3] = {i, j, k};
  const int m = f[a];
  int mc[3] = {i, j, k};
  mc[a] -= 1;
  const long long fcx = i + (long long)fb.mx * (j + (long long)fb.my * k);
  const long long cm = cidx(P, mc[0], mc[1], mc[2]), cp = cidx(P, i, j, k);
  // gradient in eps differences (dx g): normal dn, tangential the mean of
  // the two cells' centred components; n_a = -g_n / (|g| + 1e-8/dx)
  // = -dn / (|dx g| + 1e-8)
  const double dn = eps[cp] - eps[cm];
  double g2 = dn * dn;
  for (int b = 0; b < nb; ++b) {
    if (b == a) continue;
    const double tg = 0.25 * (cdiff(P, eps, b, mc[0], mc[1], mc[2]) + cdiff(P, eps, b, i, j, k));
    g2 += tg * tg;
  }
  const double na = (__double_as_longlong(g2) != 0) ? -fdiv_nr(dn, sqrt(g2) + 1e-8) : -dn * 1e8;
  const long long idn = __double_as_longlong(dn);
  const bool pos = idn < 0 && (idn << 1) != 0;  // n_a > 0
  // upwind U, downwind D, far upwind UU along a
  int uu[3] = {i, j, k};
  long long cU, cD;
  bool has;
  if (pos) {
    cU = cm;
    cD = cp;
    uu[a] = m - 2;
    has = m - 2 >= 0;
  } else {
    cU = cp;
    cD = cm;
    uu[a] = m + 1;
    has = m + 1 <= n - 1;
  }
  const long long cUU = has ? cidx(P, uu[0], uu[1], uu[2]) : cU;
  fd.s[fcx] = kcx * na;
  fd.corr[fcx] = vl_corr(cold[cUU], cold[cU], cold[cD], has);
  fd.evl[fcx] = eps[cU] + vl_corr(eps[cUU], eps[cU], eps[cD], has);
}

// iVoS: the convective flux of every face and the reactive data of the
// interface faces.  About a fifth of the faces of a porous medium carry an
// eps difference, but nearly every warp of 32 consecutive faces holds a few
// of them, and their FP64 work (a square root, three quotients) would run at
// a fraction of the warp's lanes.  So each block collects its interface faces
// (eight row segments per pass) in shared memory and hands them to its first
// threads: the FP64 instructions of that work run on full warps.  Every face
// is computed by the same operations wherever it lands, and outside the
// interface the data are written in the first pass (s = -0 marks "no
// reactive flux" for the transport assembly and the rates).
__global__ void __launch_bounds__(kThreads) k_face_data_ivos(Phys P, int a, Box fb, const double* __restrict__ eps,
                                                            const double* __restrict__ cold,
                                                            const double* __restrict__ ua, double* __restrict__ cf,
                                                            FaceData fd) {
  VOS_COUNT_EXEC();
  __shared__ int sl_i[kThreads], sl_j[kThreads], sl_k[kThreads];
  __shared__ int s_wc[kWarps];
  const Seg s = make_seg(fb);
  const int n = ncell(P, a);
  const double kcx = P.kc / P.dx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // block-uniform trip count: every thread reaches every barrier
  for (long long q0 = (long long)blockIdx.x * kWarps; q0 < s.nseg; q0 += (long long)gridDim.x * kWarps) {
    const long long q = q0 + warp;
    bool iface = false;
    int i = 0, j = 0, k = 0;
    if (q < s.nseg) {
      seg_decode(s, fb, q, i, j, k);
      if (i < fb.mx) {
        const long long fcx = i + (long long)fb.mx * (j + (long long)fb.my * k);
        cf[fcx] = conv_flux(P, a, i, j, k, cold, ua);
        int f[3] = {i, j, k};
        const int m = f[a];
        if (m < 1 || m > n - 1) {
          fd.s[fcx] = 0.0;
          fd.corr[fcx] = 0.0;
          fd.evl[fcx] = 0.0;
        } else {
          int mc[3] = {i, j, k};
          mc[a] -= 1;
          const double dn = eps[cidx(P, i, j, k)] - eps[cidx(P, mc[0], mc[1], mc[2])];
          if ((__double_as_longlong(dn) << 1) == 0) {
            // no normal eps difference: n_a = -0, so s = -0 and the face
            // carries no reactive flux; its correction and eps_vl are never
            // read (the transport assembly and the rates skip s = +-0 faces)
            fd.s[fcx] = -0.0;
            fd.corr[fcx] = 0.0;
            fd.evl[fcx] = 0.0;
          } else {
            iface = true;
          }
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, iface);
    if (lane == 0) s_wc[warp] = __popc(bal);
    __syncthreads();
    int off = 0, cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int c = s_wc[w];
      off += (w < warp) ? c : 0;
      cnt += c;
    }
    if (iface) {
      const int slot = off + __popc(bal & ((1u << lane) - 1u));
      sl_i[slot] = i;
      sl_j[slot] = j;
      sl_k[slot] = k;
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) ivos_face(P, a, fb, sl_i[threadIdx.x], sl_j[threadIdx.x], sl_k[threadIdx.x], kcx, eps, cold, fd);
    __syncthreads();  // the list and the counts are rewritten by the next pass
  }
}

void launch_face_data(const Phys& P, int ivos, const double* eps, const double* cold, double* const u[3],
                      double* const cf[3], const FaceData fd[3], cudaStream_t st) {
  const int nb = (P.dim == 2) ? 2 : 3;
  for (int a = 0; a < nb; ++a) {
    Box fb{P.nx + (a == 0), P.ny + (a == 1), P.nz + (a == 2)};
    if (ivos)
      vlaunch("face_data", 64.0 * box_cells(fb), k_face_data_ivos, grid_for(fb, 0), kThreads, st, P, a, fb, eps, cold,
              u[a], cf[a], fd[a]);
    else
      vlaunch("face_data", 24.0 * box_cells(fb), k_face_flux, grid_for(fb, 0), kThreads, st, P, a, fb, cold, u[a],
              cf[a]);
  }
}

// ---------------------------------------------------------------------------
// VoS-psi / VoS-psi' (Eq. RfVoSpsi, Sec. 2.4): psi = lambda eps (1 - eps),
// centred gradient; psi': lambda = sum|g| / sum|g| eps (1 - eps) (FP64),
// lambda = 4 when the denominator vanishes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double gradmag(const Phys& P, const double* eps, int i, int j, int k) {
  double gx = cgrad(P, eps, 0, i, j, k), gy = cgrad(P, eps, 1, i, j, k);
  double g2 = gx * gx + gy * gy;
  if (P.dim == 3) {
    double gz = cgrad(P, eps, 2, i, j, k);
    g2 += gz * gz;
  }
  return sqrt(g2);
}

__global__ void k_vos_lambda(Phys P, const double* __restrict__ eps, double* stats, RedScratch rs) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  double acc[2] = {0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    double e = eps[cidx(P, i, j, k)];
    double g = gradmag(P, eps, i, j, k);
    acc[0] += g;
    acc[1] += g * e * (1.0 - e);
  }
  if (grid_sum<2>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    double num = acc[0], den = acc[1];
    stats[ST_LAMBDA] = (num == 0.0 || den < 1e-300 * num) ? 4.0 : num / den;
  }
}

__global__ void k_set_scalar(double* dst, double v) {
  VOS_COUNT_EXEC();
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

__global__ void k_div_check(const double* __restrict__ a, const double* __restrict__ d, long long n,
                            double* __restrict__ qf, double* __restrict__ qi) {
  VOS_COUNT_EXEC();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    qf[c] = fdiv_nr(a[c], d[c]);
    qi[c] = a[c] / d[c];
  }
}

void launch_div_check(const double* a, const double* d, long long n, double* q_fast, double* q_ieee,
                      cudaStream_t st) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  vlaunch("div_check", 32.0 * n, k_div_check, (int)g, kThreads, st, a, d, n, q_fast, q_ieee);
}

__global__ void k_extrapolate(long long n, const double* __restrict__ u, double* __restrict__ uprev,
                              double* __restrict__ us) {
  VOS_COUNT_EXEC();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double v = u[c];
    us[c] = 2.0 * v - uprev[c];
    uprev[c] = v;
  }
}

void launch_extrapolate(long long n, const double* u, double* uprev, double* us, cudaStream_t st) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > (long long)g_num_sms * 8) g = (long long)g_num_sms * 8;
  if (g < 1) g = 1;
  vlaunch("u_extrapolate", 32.0 * n, k_extrapolate, (int)g, kThreads, st, n, u, uprev, us);
}

void launch_set_scalar(double* dst, double v, cudaStream_t st) {
  vlaunch("set_scalar", 8.0, k_set_scalar, 1, 32, st, dst, v);
}

void launch_vos_lambda(const Phys& P, const double* eps, double lambda_fixed, int fit, double* stats,
                       const RedScratch& rs, cudaStream_t st) {
  if (fit) {
    Box bx{P.nx, P.ny, P.nz};
    vlaunch("vos_lambda", 8.0 * box_cells(bx), k_vos_lambda, grid_for(bx, kMaxRedBlocks), kThreads, st, P, eps, stats, rs);
  } else {
    vlaunch("set_scalar", 8.0, k_set_scalar, 1, 32, st, stats + ST_LAMBDA, lambda_fixed);
  }
}

__global__ void k_vos_coef(Phys P, const double* __restrict__ eps, const double* __restrict__ stats,
                           double* __restrict__ kr) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const double lam = stats[ST_LAMBDA];
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c = cidx(P, i, j, k);
    const double e = eps[c];
    kr[c] = P.kc * lam * e * (1.0 - e) * gradmag(P, eps, i, j, k);
  }
}

void launch_vos_coef(const Phys& P, const double* eps, const double* stats, double* kr, cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  vlaunch("vos_coef", 16.0 * box_cells(bx), k_vos_coef, grid_for(bx, 0), kThreads, st, P, eps, stats, kr);
}

// ---------------------------------------------------------------------------
// S4 + S5: transport system for c^{n+1} (Eq. concentrationDBS)
//   eps c/dt - div(eps_f D grad c) + zeta R_f(c) = eps^n c^n/dt - div(c^n_f u)
// Explicit van Leer convective flux (upwind along sign(u_f)); inlet faces
// u_in c_in, outlet faces u c_last; Dirichlet c_in at the inlet for
// diffusion (ghost 2 c_in - c_P).  R_f: VoS -> kr c; iVoS -> eps_P sum over
// faces of the outward reactive flux with frozen van Leer weights.
// ---------------------------------------------------------------------------
template <bool IVOS>
__global__ void k_trans_assemble(Phys P, const double* __restrict__ eps, const double* __restrict__ eps_old,
                                 const double* __restrict__ cold, const double* __restrict__ cf0,
                                 const double* __restrict__ cf1, const double* __restrict__ cf2,
                                 const double* __restrict__ kr, FaceData f0, FaceData f1, FaceData f2, const double* __restrict__ dtp,
                                 double omega, Op<double> A, double* __restrict__ rhs) {
  VOS_COUNT_EXEC();
  const double idt = 1.0 / *dtp;
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const double idx2 = 1.0 / (P.dx * P.dx), idx1 = 1.0 / P.dx;
  const double dh = P.D * 0.5 * idx2;  // diffusion link = dh (eps_P + eps_N)
  const int nb = (P.dim == 2) ? 2 : 3;
  const double* cfs[3] = {cf0, cf1, cf2};
  const FaceData fds[3] = {f0, f1, f2};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c = cidx(P, i, j, k);
    const double e = eps[c];
    double diag = e * idt;
    double b = eps_old[c] * cold[c] * idt;
    double offp[3] = {0, 0, 0}, offm[3] = {0, 0, 0};
    double adv = 0.0;
    for (int d = 0; d < nb; ++d) {
      int lo[3] = {i, j, k}, hi[3] = {i, j, k};
      lo[d] -= 1;
      hi[d] += 1;
      const bool hasp = cell_in(P, hi[0], hi[1], hi[2]);
      const bool hasm = cell_in(P, lo[0], lo[1], lo[2]);
      if (hasp) {
        double a = dh * (e + eps[cidx(P, hi[0], hi[1], hi[2])]);
        diag += a;
        offp[d] -= a;
      }
      if (hasm) {
        double a = dh * (e + eps[cidx(P, lo[0], lo[1], lo[2])]);
        diag += a;
        offm[d] -= a;
      }
      // convective fluxes through the plus and minus faces (k_face_flux / k_face_data_ivos)
      int fp[3] = {i, j, k};
      fp[d] += 1;
      adv += (cfs[d][fidx(P, d, fp[0], fp[1], fp[2])] - cfs[d][fidx(P, d, i, j, k)]) * idx1;
      if (IVOS) {
        // reactive flux F = s (c_U^{n+1} + corr): upwind value implicit,
        // the deferred van Leer correction on the right-hand side
        // faces away from the solid surface have s = +-0 (zero eps gradient):
        // their terms vanish and are skipped on the bit pattern
        const double zc = P.zeta * e;
        auto nonzero = [](double v) { return (__double_as_longlong(v) << 1) != 0; };
        if (hasp && nonzero(fds[d].s[fidx(P, d, fp[0], fp[1], fp[2])])) {  // the minus cell of its plus face
          const long long fx = fidx(P, d, fp[0], fp[1], fp[2]);
          const double sf = fds[d].s[fx];
          if (sf > 0.0)
            diag += zc * sf;  // U = this
          else
            offp[d] += zc * sf;  // U = plus
          b -= zc * sf * fds[d].corr[fx];
        }
        if (hasm && nonzero(fds[d].s[fidx(P, d, i, j, k)])) {  // the plus cell of its minus face (outward -F)
          const long long fx = fidx(P, d, i, j, k);
          const double sf = fds[d].s[fx];
          if (sf > 0.0)
            offm[d] -= zc * sf;  // U = minus
          else
            diag -= zc * sf;  // U = this
          b += zc * sf * fds[d].corr[fx];
        }
      }
    }
    if (i == 0) {
      const double a = 2.0 * P.D * e * idx2;
      diag += a;
      b += a * P.c_in;
    }
    if (!IVOS) diag += P.zeta * kr[c];
    b -= adv;
    A.diag[c] = diag;
    A.dinv[c] = jacobi_weight(omega, diag);
    A.xp[c] = offp[0];
    A.yp[c] = offp[1];
    if (A.zp) A.zp[c] = offp[2];
    if (!A.sym) {
      A.xm[c] = offm[0];
      A.ym[c] = offm[1];
      if (A.zm) A.zm[c] = offm[2];
    }
    rhs[c] = b;
  }
}

void launch_trans_assemble(const Phys& P, int ivos, const double* eps, const double* eps_old, const double* cold,
                           double* const cf[3], const double* kr, const FaceData fd[3], const double* __restrict__ dtp, double omega,
                           Op<double> A, double* rhs, cudaStream_t st) {
  int g = grid_for(A.box, 0);
  if (ivos)
    vlaunch("trans_assemble", (6.0 + 5.0 * P.dim) * 8.0 * box_cells(A.box), k_trans_assemble<true>, g, kThreads, st, P,
            eps, eps_old, cold, cf[0], cf[1], cf[2], kr, fd[0], fd[1], fd[2], dtp, omega, A, rhs);
  else
    vlaunch("trans_assemble", (7.0 + 2.0 * P.dim) * 8.0 * box_cells(A.box), k_trans_assemble<false>, g, kThreads, st, P,
            eps, eps_old, cold, cf[0], cf[1], cf[2], kr, fd[0], fd[1], fd[2], dtp, omega, A, rhs);
}

// ---------------------------------------------------------------------------
// S6: reaction rates from c^{n+1}.
//   iVoS (Eq. RfiVoS): R_f = eps_P sum_f outward F_f / V,
//                      R   = R_f - sum_f outward evl_f F_f / V,
//   with F_f / V = s_f (c_U^{n+1} + corr_f) on interior faces (the face
//   values the transport solve used, so the sink and R_f agree exactly).
//   VoS-psi('): R = R_f = kr c.
// Also reduces sum R V, sum R_f V, sum eps c V.
// ---------------------------------------------------------------------------
template <bool IVOS>
__global__ void k_rates(Phys P, const double* __restrict__ eps, const double* __restrict__ cn,
                        const double* __restrict__ kr, FaceData f0, FaceData f1, FaceData f2, double* __restrict__ R,
                        double* __restrict__ Rf, double* stats, RedScratch rs) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const int nb = (P.dim == 2) ? 2 : 3;
  const FaceData fds[3] = {f0, f1, f2};
  double acc[3] = {0.0, 0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c = cidx(P, i, j, k);
    const double e = eps[c];
    double r, rf;
    if (IVOS) {
      // faces with s = +-0 (no eps gradient) carry no reactive flux: skipped
      // on the bit pattern
      auto nonzero = [](double v) { return (__double_as_longlong(v) << 1) != 0; };
      double sumF = 0.0, sumEF = 0.0;
      for (int d = 0; d < nb; ++d) {
        int lo[3] = {i, j, k}, hi[3] = {i, j, k};
        lo[d] -= 1;
        hi[d] += 1;
        int fp[3] = {i, j, k};
        fp[d] += 1;
        if (cell_in(P, hi[0], hi[1], hi[2]) && nonzero(fds[d].s[fidx(P, d, fp[0], fp[1], fp[2])])) {
          const long long fx = fidx(P, d, fp[0], fp[1], fp[2]);
          const double sf = fds[d].s[fx];
          const double cU = sf > 0.0 ? cn[c] : cn[cidx(P, hi[0], hi[1], hi[2])];
          const double F = sf * (cU + fds[d].corr[fx]);
          sumF += F;
          sumEF += fds[d].evl[fx] * F;
        }
        if (cell_in(P, lo[0], lo[1], lo[2]) && nonzero(fds[d].s[fidx(P, d, i, j, k)])) {
          const long long fx = fidx(P, d, i, j, k);
          const double sf = fds[d].s[fx];
          const double cU = sf > 0.0 ? cn[cidx(P, lo[0], lo[1], lo[2])] : cn[c];
          const double F = sf * (cU + fds[d].corr[fx]);
          sumF -= F;
          sumEF -= fds[d].evl[fx] * F;
        }
      }
      rf = e * sumF;
      r = rf - sumEF;
    } else {
      r = kr[c] * cn[c];
      rf = r;
    }
    R[c] = r;
    Rf[c] = rf;
    acc[0] += r;
    acc[1] += rf;
    acc[2] += e * cn[c];
  }
  if (grid_sum<3>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    double V = (P.dim == 2) ? P.dx * P.dx : P.dx * P.dx * P.dx;
    stats[ST_SUMR] = acc[0] * V;
    stats[ST_SUMRF] = acc[1] * V;
    stats[ST_REACT] = acc[2] * V;
  }
}

void launch_rates(const Phys& P, int ivos, const double* eps, const double* c, const double* kr,
                  const FaceData fd[3], double* R, double* Rf, double* stats, const RedScratch& rs,
                  cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  int g = grid_for(bx, kMaxRedBlocks);
  if (ivos)
    vlaunch("rates", (4.0 + 3.0 * P.dim) * 8.0 * box_cells(bx), k_rates<true>, g, kThreads, st, P, eps, c, kr, fd[0], fd[1], fd[2], R, Rf, stats, rs);
  else
    vlaunch("rates", 40.0 * box_cells(bx), k_rates<false>, g, kThreads, st, P, eps, c, kr, fd[0], fd[1], fd[2], R, Rf, stats, rs);
}

// ---------------------------------------------------------------------------
// Time-step limits (App. D): max over faces of |u_f| / eps_f (interior:
// mean of the two cells; boundary: the adjacent cell) and max |Vm R|.  A NaN
// speed or rate counts as +inf (fmax alone would drop it), so the limit
// becomes dt = 0 instead of a finite value.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double nan_inf(double x) { return (x == x) ? x : INFINITY; }

__global__ void k_dt_limits(Phys P, const double* __restrict__ eps, const double* __restrict__ u0,
                            const double* __restrict__ u1, const double* __restrict__ u2,
                            const double* __restrict__ R, double* stats, RedScratch rs) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const int nb = (P.dim == 2) ? 2 : 3;
  const double* us[3] = {u0, u1, u2};
  double acc[2] = {0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c = cidx(P, i, j, k);
    const double e = eps[c];
    for (int d = 0; d < nb; ++d) {
      // minus face of this cell; the plus boundary face for the last cell
      int lo[3] = {i, j, k};
      lo[d] -= 1;
      double ef = cell_in(P, lo[0], lo[1], lo[2]) ? 0.5 * (e + eps[cidx(P, lo[0], lo[1], lo[2])]) : e;
      acc[0] = fmax(acc[0], nan_inf(fabs(us[d][fidx(P, d, i, j, k)]) / ef));
      int f[3] = {i, j, k};
      if (f[d] == ncell(P, d) - 1) {
        f[d] += 1;
        acc[0] = fmax(acc[0], nan_inf(fabs(us[d][fidx(P, d, f[0], f[1], f[2])]) / e));
      }
    }
    acc[1] = fmax(acc[1], nan_inf(fabs(P.Vm * R[c])));
  }
  if (grid_max<2>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    stats[ST_UMAX] = acc[0];
    stats[ST_RMAX] = acc[1];
  }
}

// S7 diagnostics at the end of a step: the two maxima of k_dt_limits on
// u^{n+1}, R^{n+1} (|u_f| / eps_f with the physics kernels' FP64 quotient,
// within 2 ulp of the IEEE one) and, on the inlet (i = 0) and outlet
// (i = nx - 1) columns, q_in = sum u_f A, q_out, the reactant inflow
// (convective u c_in from the face fluxes plus the Dirichlet ghost's
// diffusive flux 2 D eps_P (c_in - c_P) / dx) and outflow (convective flux
// u c^n of the outlet face), all times the face area A = dx^(d-1).
__global__ void k_step_diag(Phys P, const double* __restrict__ eps, const double* __restrict__ u0,
                            const double* __restrict__ u1, const double* __restrict__ u2,
                            const double* __restrict__ R, const double* __restrict__ c,
                            const double* __restrict__ cf0, double* stats, RedScratch rs) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  const int nb = (P.dim == 2) ? 2 : 3;
  const double* us[3] = {u0, u1, u2};
  const double idx = 1.0 / P.dx;
  double mx[2] = {0.0, 0.0};
  double sm[4] = {0.0, 0.0, 0.0, 0.0};
  // the thread's largest abs(u_f) / eps_f is kept as the pair (bu, be) and
  // a face replaces it when abs(u_f) be > bu eps_f, so the quotient is taken
  // once per thread; a NaN velocity makes the maximum infinite
  double bu = 0.0, be = 1.0;
  bool nan_u = false;
  auto consider = [&](double uf, double ef) {
    const double au = fabs(uf);
    if (au != au) nan_u = true;
    else if (au * be > bu * ef) {
      bu = au;
      be = ef;
    }
  };
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c0 = cidx(P, i, j, k);
    const double e = eps[c0];
    for (int d = 0; d < nb; ++d) {
      int lo[3] = {i, j, k};
      lo[d] -= 1;
      const double ef = cell_in(P, lo[0], lo[1], lo[2]) ? 0.5 * (e + eps[cidx(P, lo[0], lo[1], lo[2])]) : e;
      consider(us[d][fidx(P, d, i, j, k)], ef);
      int f[3] = {i, j, k};
      if (f[d] == ncell(P, d) - 1) {
        f[d] += 1;
        consider(us[d][fidx(P, d, f[0], f[1], f[2])], e);
      }
    }
    mx[1] = fmax(mx[1], nan_inf(fabs(P.Vm * R[c0])));
    if (i == 0) {
      const long long fx = fidx(P, 0, 0, j, k);
      sm[0] += u0[fx];
      sm[2] += cf0[fx] + 2.0 * P.D * e * (P.c_in - c[c0]) * idx;
    }
    if (i == P.nx - 1) {
      const long long fx = fidx(P, 0, P.nx, j, k);
      sm[1] += u0[fx];
      sm[3] += cf0[fx];
    }
  }
  mx[0] = nan_u ? INFINITY : nan_inf(fdiv_nr(bu, be));
  if (grid_sum_max<4, 2>(sm, mx, rs.partials, rs.counter) && threadIdx.x == 0) {
    const double A = (P.dim == 2) ? P.dx : P.dx * P.dx;
    stats[ST_UMAX] = mx[0];
    stats[ST_RMAX] = mx[1];
    stats[ST_QIN] = sm[0] * A;
    stats[ST_QOUT] = sm[1] * A;
    stats[ST_FIN] = sm[2] * A;
    stats[ST_FOUT] = sm[3] * A;
  }
}

void launch_step_diag(const Phys& P, const double* eps, double* const u[3], const double* R, const double* c,
                      const double* cf0, double* stats, const RedScratch& rs, cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  vlaunch("step_diag", (2.0 + P.dim) * 8.0 * box_cells(bx), k_step_diag, grid_for(bx, kMaxRedBlocks), kThreads, st,
          P, eps, u[0], u[1], u[2] ? u[2] : u[0], R, c, cf0, stats, rs);
}

// Sums behind the Darcy-scale properties of Sec. 2.5 (FP64, fixed order):
// out[0] sum eps, out[1] sum |grad eps| (centred), out[2] sum c |grad eps|,
// out[3] sum eps c, out[4] sum of p over the first cell column (i = 0),
// out[5] sum of u over the inlet faces.
__global__ void k_upscaled_sums(Phys P, const double* __restrict__ eps, const double* __restrict__ c,
                                const double* __restrict__ p, const double* __restrict__ u0, double* out,
                                RedScratch rs) {
  VOS_COUNT_EXEC();
  const Box bx{P.nx, P.ny, P.nz};
  const Seg s = make_seg(bx);
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  VOS_SEG_LOOP(s, q) {
    int i, j, k;
    seg_decode(s, bx, q, i, j, k);
    if (i >= bx.mx) continue;
    const long long c0 = cidx(P, i, j, k);
    const double e = eps[c0], cc = c[c0];
    const double g = gradmag(P, eps, i, j, k);
    acc[0] += e;
    acc[1] += g;
    acc[2] += cc * g;
    acc[3] += e * cc;
    if (i == 0) {
      acc[4] += p[c0];
      acc[5] += u0[fidx(P, 0, 0, j, k)];
    }
  }
  if (grid_sum<6>(acc, rs.partials, rs.counter) && threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) out[q] = acc[q];
  }
}

void launch_upscaled_sums(const Phys& P, const double* eps, const double* c, const double* p, const double* u0,
                          double* out, const RedScratch& rs, cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  vlaunch("upscaled_sums", 3.0 * 8.0 * box_cells(bx), k_upscaled_sums, grid_for(bx, kMaxRedBlocks), kThreads, st, P,
          eps, c, p, u0, out, rs);
}

void launch_dt_limits(const Phys& P, const double* eps, double* const u[3], const double* R, double* stats,
                      const RedScratch& rs, cudaStream_t st) {
  Box bx{P.nx, P.ny, P.nz};
  vlaunch("dt_limits", (2.0 + P.dim) * 8.0 * box_cells(bx), k_dt_limits, grid_for(bx, kMaxRedBlocks), kThreads, st, P, eps, u[0], u[1],
          u[2] ? u[2] : u[0], R, stats, rs);
}

}  // namespace vos
