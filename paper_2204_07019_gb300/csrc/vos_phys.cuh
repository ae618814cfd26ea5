// Physics kernels of the VoS step (declarations shared by vos_fields.cu and
// vos_capi.cu).
#pragma once

#include "vos_internal.cuh"

namespace vos {

struct Phys {
  int dim, nx, ny, nz;
  double dx, nu, D, kc, k0, Vm, zeta, rho_ratio, c_in, u_in, eps_min;
  unsigned wall_mask;
};

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
  ST_COUNT = 8
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
void launch_mom_assemble(const Phys& P, int a, const double* eps, const double* kic, const double* p, const double* uold,
                         const double* dtp,
                         double omega, Op<double> A, double* rhs, cudaStream_t st);
// S3
// eps32 (may be NULL): receives the FP32 fluid fraction that the matrix-free
// FP32 pressure sweeps read.
void launch_pres_assemble(const Phys& P, const double* eps, double* const us[3], const double* R, const double* dtp,
                          double omega, Op<double> A, double* rhs, float* eps32, cudaStream_t st);
void launch_project(const Phys& P, const double* eps, const double* phi, const double* dtp, double* const us[3],
                    double* const u[3], double* p, cudaStream_t st);
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
void launch_dt_limits(const Phys& P, const double* eps, double* const u[3], const double* R, double* stats,
                      const RedScratch& rs, cudaStream_t st);

}  // namespace vos
