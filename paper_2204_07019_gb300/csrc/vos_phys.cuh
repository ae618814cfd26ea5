// Physics kernels of the VoS step (declarations shared by vos_fields.cu and
// vos_capi.cu).
#pragma once

#include "vos_internal.cuh"

namespace vos {

struct Phys {
  int dim, nx, ny, nz;
  double dx, nu, D, kc, k0, Vm, zeta, rho_ratio, c_in, u_in, eps_min;
  unsigned wall_mask;
  int inertia;  // explicit div(u u / eps) in the momentum right-hand side
};

// ---------------------------------------------------------------------------
// FP64 arithmetic is the scarce resource of the physics kernels on this part
// (a few FP64 operations per SM and clock, against 128 FP32 ones), so their
// divisions use this quotient instead of the IEEE one: the FMA-based
// Newton-Raphson division of P. W. Markstein (IBM J. Res. Dev. 34(1), 1990),
// seeded by the hardware reciprocal estimate (PTX rcp.approx.ftz.f64): one
// step on the reciprocal, y1 = y0 + y0 (1 - d y0), then one on the
// quotient, q1 = q0 + y1 (a - d q0) with q0 = a y1.  A seed with relative
// error e leaves e^2 after the first step and e^4 after the second, so q1 is
// within a couple of ulp of a/d (vos_fp64_div_check compares it with the
// IEEE quotient): five FP64 operations.  |d| outside [2^-1000, 2^1000],
// zero, infinite or NaN takes the IEEE division.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fdiv_nr(double a, double d) {
  const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
  if (ex < 23u || ex > 2023u) return a / d;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  y = fma(y, fma(-d, y, 1.0), y);
  const double q = a * y;
  return fma(y, fma(-d, q, a), q);
}

// Device diagnostics (FP64), indices into the stats array.
enum StatIdx {
  ST_CLAMP = 0,   // sum(raw - clamped) V
  ST_EPSSUM = 1,  // sum eps
  ST_SUMR = 2,    // sum R V
  ST_SUMRF = 3,   // sum R_f V
  ST_REACT = 4,   // sum eps c V
  ST_LAMBDA = 5,  // VoS lambda used
  ST_UMAX = 6,    // max |u_f| / eps_f
  ST_RMAX = 7,    // max |Vm R|
  ST_QIN = 8,     // sum over inlet faces of u_f A_f
  ST_QOUT = 9,    // sum over outlet faces of u_f A_f
  ST_FIN = 10,    // reactant inflow: inlet convective + diffusive flux, times A_f
  ST_FOUT = 11,   // reactant outflow: outlet convective flux (c^n), times A_f
  ST_QSU = 12,    // quasi-static sub-iterations: per axis a, [12 + 2a] sum (u - u_old)^2, [13 + 2a] sum u^2
  ST_QSP = 18,    // sum eps phi^2, sum eps p^2 (the pressure change of the sub-iteration)
  ST_QSC = 20,    // sum (c - c_old)^2, sum c^2
  ST_COUNT = 22
};

struct FaceData {  // iVoS per-face data for one axis (face-array layout)
  double *s;     // k_c n_a / dx: reactive flux per unit volume per unit c_f
  double *corr;  // deferred van Leer correction w(c^n) (c_D^n - c_U^n)
  double *evl;   // van Leer interpolation of eps
};

// S1
// kic: receives the Kozeny-Carman k^-1 of the new eps per cell (read by the
// momentum assembly).
void launch_eps_update(const Phys& P, double* eps, double* eps_old, const double* R, const double* dtp, double* stats,
                       const RedScratch& rs, double* kic, cudaStream_t st);
// S2
// u: every velocity component at t^n (read by the inertia term when P.inertia)
void launch_mom_assemble(const Phys& P, int a, const double* eps, const double* kic, const double* p, const double* uold,
                         const double* dtp, double* const u[3],
                         double omega, Op<double> A, double* rhs, cudaStream_t st);
// S3
// eps32 (may be NULL): receives the FP32 fluid fraction that the matrix-free
// FP32 pressure sweeps read.
void launch_pres_assemble(const Phys& P, const double* eps, double* const us[3], const double* R, const double* dtp,
                          double omega, Op<double> A, double* rhs, float* eps32, cudaStream_t st);
void launch_project(const Phys& P, const double* eps, const double* phi, const double* dtp, double* const us[3],
                    double* const u[3], double* p, cudaStream_t st);
// The same projection that also reduces, per axis, sum (u^{new} - u^{old})^2
// and sum (u^{new})^2 into stats[ST_QSU + 2a], stats[ST_QSU + 2a + 1]
// (quasi-static sub-iterations).
void launch_project_sums(const Phys& P, const double* eps, const double* phi, const double* dtp,
                         double* const us[3], double* const u[3], double* p, double* stats, const RedScratch& rs,
                         cudaStream_t st);
// out[0] = sum w (x - y)^2 (DIFF) or sum w y^2, out[1] = sum w x^2 over n
// cells (w NULL: 1).
void launch_qs_sums(long long n, bool diff, const double* x, const double* y, const double* w, double* out,
                    const RedScratch& rs, cudaStream_t st);
// S5/S6
// cf[a]: receives the convective flux of c^n through every face of axis a
// (read by the transport assembly); fd: the iVoS face data (ivos only).
void launch_face_data(const Phys& P, int ivos, const double* eps, const double* cold, double* const u[3],
                      double* const cf[3], const FaceData fd[3], cudaStream_t st);
void launch_vos_lambda(const Phys& P, const double* eps, double lambda_fixed, int fit, double* stats,
                       const RedScratch& rs, cudaStream_t st);
void launch_vos_coef(const Phys& P, const double* eps, const double* stats, double* kr, cudaStream_t st);
void launch_trans_assemble(const Phys& P, int ivos, const double* eps, const double* eps_old, const double* cold,
                           double* const cf[3], const double* kr, const FaceData fd[3], const double* dtp, double omega,
                           Op<double> A, double* rhs, cudaStream_t st);
void launch_rates(const Phys& P, int ivos, const double* eps, const double* c, const double* kr,
                  const FaceData fd[3], double* R, double* Rf, double* stats, const RedScratch& rs,
                  cudaStream_t st);
void launch_set_scalar(double* dst, double v, cudaStream_t st);
// us = 2 u - uprev, then uprev = u (n values): the extrapolated initial guess
// of the momentum solves.
void launch_extrapolate(long long n, const double* u, double* uprev, double* us, cudaStream_t st);
// q_fast[i] = fdiv_nr(a[i], d[i]), q_ieee[i] = a[i] / d[i] (device arrays).
void launch_div_check(const double* a, const double* d, long long n, double* q_fast, double* q_ieee,
                      cudaStream_t st);
void launch_dt_limits(const Phys& P, const double* eps, double* const u[3], const double* R, double* stats,
                      const RedScratch& rs, cudaStream_t st);
// End-of-step diagnostics (S7): ST_UMAX, ST_RMAX of u^{n+1}, R^{n+1} and
// the boundary sums ST_QIN..ST_FOUT.  cf0: convective face fluxes of axis x
// written by launch_face_data (inlet u c_in, outlet u c^n); c: c^{n+1}.
// Sums of the Darcy-scale properties (out: 6 device doubles, see
// k_upscaled_sums).
void launch_upscaled_sums(const Phys& P, const double* eps, const double* c, const double* p, const double* u0,
                          double* out, const RedScratch& rs, cudaStream_t st);
void launch_step_diag(const Phys& P, const double* eps, double* const u[3], const double* R, const double* c,
                      const double* cf0, double* stats, const RedScratch& rs, cudaStream_t st);

}  // namespace vos
