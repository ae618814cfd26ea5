// C ABI of the VoS step: handle lifetime, device memory, step orchestration.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vos.h"
#include "vos_phys.cuh"

using namespace vos;

namespace {

thread_local std::string g_create_error;

template <typename T>
struct Sys {
  Box box;
  int sym;
  Op<double> op64;
  double* rhs;
  Hier<T> h;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace vos {
const Op<double>* handle_pressure_op(vos_handle* h);
const double* handle_eps(vos_handle* h);
void unet_box(const vos_unet* net, int* px, int* py, int* pz);
void unet_attach_eps(vos_unet* net, const double* eps);
// Error text reported by vos_last_error(NULL) for calls without a handle.
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace vos

struct vos_handle {
  vos_params prm;
  Phys ph;
  cudaStream_t st;
  vos_allocator alloc;
  bool user_alloc;
  std::vector<void*> blocks;
  std::vector<size_t> block_bytes;
  size_t bytes;
  // floating-cluster deflation of the pressure solve (one device block)
  void* defl_mem;
  size_t defl_cap;
  Defl defl;
  // fields
  double *eps, *eps_old, *c, *p, *phi, *R, *Rf, *kr, *kic;
  float* eps32;  // FP32 fluid fraction for the matrix-free pressure sweeps (mixed precision)
  double *u[3], *us[3];
  double* uprev[3];  // u^{n-1} (VOS_PRECOND_U_EXTRAP only)
  FaceData fd[3];
  // solvers: 0..2 momentum, 3 pressure, 4 transport
  Sys<double> sd[5];
  Sys<float> sf[5];
  SolverWork* work;
  RedScratch rs;
  double* dstats;
  double* hstats;  // pinned
  double* d_dt;    // device copy of the step's dt (read by the physics kernels)
  double* dups;    // device sums of vos_upscaled (6)
  // graph mode: the whole step captured once per momentum-preconditioner
  // choice and replayed on an internal stream ordered after the caller's
  SolveStats* dsolve;  // device, one per system
  SolveStats* hsolve;  // pinned copy
  cudaStream_t gs, gs1, gs2;
  cudaEvent_t ev_in, ev_out;
  cudaGraphExec_t exec[2];
  vos_unet* net;       // learned pressure preconditioner (not owned)
  unsigned graph_gen;  // bumped whenever captured launch parameters change
  int net_iters, net_fallback;
  vos_stats stats;
  std::string err;
  int dev;
};

namespace {

bool g_use_graphs = true;

int set_err(vos_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return code;
}

void* dev_alloc(vos_handle* h, size_t bytes) {
  bytes = align256(bytes ? bytes : 256);
  void* p = nullptr;
  if (h->user_alloc) {
    p = h->alloc.alloc(bytes, h->alloc.ctx);
    // the kernels' 16-byte vector accesses and 256-byte carves rely on the
    // allocator's alignment promise: a block that breaks it is released and
    // counts as a failed allocation
    if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {
      h->alloc.free(p, h->alloc.ctx);
      p = nullptr;
    }
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  }
  if (p) {
    h->blocks.push_back(p);
    h->block_bytes.push_back(bytes);
    h->bytes += bytes;
  }
  return p;
}

void dev_free(vos_handle* h, void* p) {
  for (size_t i = 0; i < h->blocks.size(); ++i) {
    if (h->blocks[i] != p) continue;
    if (h->user_alloc)
      h->alloc.free(p, h->alloc.ctx);
    else
      cudaFree(p);
    h->bytes -= h->block_bytes[i];
    h->blocks.erase(h->blocks.begin() + (long)i);
    h->block_bytes.erase(h->block_bytes.begin() + (long)i);
    return;
  }
}

void free_all(vos_handle* h) {
  for (void* p : h->blocks) {
    if (h->user_alloc)
      h->alloc.free(p, h->alloc.ctx);
    else
      cudaFree(p);
  }
  h->blocks.clear();
  h->block_bytes.clear();
  h->defl_mem = nullptr;
  h->defl_cap = 0;
  h->defl = Defl{0, nullptr, nullptr, nullptr};
  if (h->work) solver_work_free(h->work);
  h->work = nullptr;
  if (h->hstats) cudaFreeHost(h->hstats);
  h->hstats = nullptr;
  if (h->hsolve) cudaFreeHost(h->hsolve);
  h->hsolve = nullptr;
  for (int i = 0; i < 2; ++i) {
    if (h->exec[i]) cudaGraphExecDestroy(h->exec[i]);
    h->exec[i] = nullptr;
  }
  if (h->gs) cudaStreamDestroy(h->gs);
  if (h->gs1) cudaStreamDestroy(h->gs1);
  if (h->gs2) cudaStreamDestroy(h->gs2);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  h->gs = h->gs1 = h->gs2 = nullptr;
  h->ev_in = h->ev_out = nullptr;
}

Box unknown_box(const Phys& P, int sys) {
  switch (sys) {
    case 0: return Box{P.nx, P.ny, P.nz};
    case 1: return Box{P.nx, P.ny - 1, P.nz};
    case 2: return Box{P.nx, P.ny, P.nz - 1};
    default: return Box{P.nx, P.ny, P.nz};
  }
}

long long face_count(const Phys& P, int a) {
  return (long long)(P.nx + (a == 0)) * (P.ny + (a == 1)) * (P.nz + (a == 2));
}

View<double> unknown_view(vos_handle* h, int sys) {
  const Phys& P = h->ph;
  switch (sys) {
    case 0: return View<double>{h->us[0] + 1, P.nx + 1, (P.nx + 1) * P.ny};
    case 1: return View<double>{h->us[1] + P.nx, P.nx, P.nx * (P.ny + 1)};
    case 2: return View<double>{h->us[2] + (long long)P.nx * P.ny, P.nx, P.nx * P.ny};
    case 3: return View<double>{h->phi, P.nx, P.nx * P.ny};
    default: return View<double>{h->c, P.nx, P.nx * P.ny};
  }
}

// Smoother and coarse-correction weights.  3D flow systems: Jacobi 0.9 with
// the aggregation correction over-weighted by 2.2 (a sweep on a 128^3 crop of
// the rock with pocket deflation: 55 -> 42 PCG iterations against 0.7 / 1.8;
// 0.9 / 2.4 and 0.85 / 2.6 are worse again).
MGParams mg_for(const Phys& P, int sys) {
  MGParams m;
  const bool flow3d = (P.dim == 3 && sys != 4);
  m.omega = (P.dim == 2) ? 0.8 : (flow3d ? 0.9 : 0.7);
  m.wc = (sys == 4) ? 1.0 : (flow3d ? 2.2 : 1.8);
  m.nu = 2;
  m.coarse_sweeps = 30;
  return m;
}

template <typename T>
bool alloc_sys(vos_handle* h, Sys<T>& S, int sys, int sym) {
  const Phys& P = h->ph;
  S.box = unknown_box(P, sys);
  S.sym = sym;
  std::memset(&S.op64, 0, sizeof(S.op64));
  S.rhs = nullptr;
  S.h.nlev = 0;
  if (box_cells(S.box) == 0) return true;
  const bool share = (sizeof(T) == 8);
  size_t nb = op64_bytes(S.box, sym) + align256((size_t)box_cells(S.box) * 8) + hier_bytes<T>(S.box, sym, share);
  char* cur = (char*)dev_alloc(h, nb);
  if (!cur) return false;
  op64_carve(S.op64, S.box, sym, cur);
  S.rhs = (double*)cur;
  cur += align256((size_t)box_cells(S.box) * 8);
  hier_carve<T>(S.h, S.box, sym, cur, mg_for(P, sys), share, &S.op64);
  return true;
}

// The momentum operator is (1/dt + drag) I - nu lap: when the mass term
// dominates (2 d nu dt / dx^2 <= 30) the diagonally preconditioned CG
// converges in a grid-independent number of iterations at a third of the
// traffic of a multigrid iteration; otherwise use multigrid.  The precond
// flags VOS_PRECOND_MOM_DIAG / VOS_PRECOND_MOM_MG override the rule.
bool mom_mg_for(const vos_handle* h, double dt) {
  if (h->prm.precond & VOS_PRECOND_MOM_DIAG) return false;
  if (h->prm.precond & VOS_PRECOND_MOM_MG) return true;
  const Phys& P = h->ph;
  return 2.0 * P.dim * P.nu * dt / (P.dx * P.dx) > 30.0;
}

template <typename T>
int step_impl(vos_handle* h, Sys<T>* S, double dt) {
  const Phys& P = h->ph;
  cudaStream_t st = h->st;
  const int nd = P.dim;
  const int ivos = (h->prm.method == VOS_IVOS);
  vos_stats& s = h->stats;
  int status = VOS_OK;
  // quasi-static step: M sub-iterations of S2-S6 with eps frozen (see vos.h)
  const int M = h->prm.flow_subiters > 1 ? h->prm.flow_subiters : 1;
  const bool qs = M > 1;
  const double dtau = (qs && h->prm.qs_dtau > 0.0) ? h->prm.qs_dtau : dt;
  const long long N = (long long)P.nx * P.ny * P.nz;
  launch_set_scalar(h->d_dt, dt, st);
  const double* dtp = h->d_dt;
  // S1: solid fraction and (implicitly) permeability
  launch_eps_update(P, h->eps, h->eps_old, h->R, dtp, h->dstats, h->rs, h->kic, st);
  if (qs) {
    // the sub-iterations march in the pseudo step, with eps^{n+1} in both
    // storage terms of the transport equation
    launch_set_scalar(h->d_dt, dtau, st);
    cudaMemcpyAsync(h->eps_old, h->eps, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  const bool mom_mg = mom_mg_for(h, dtau);
  for (int a = 0; a < 3; ++a) {
    s.iters_u[a] = 0;
    s.outer_u[a] = 0;
    s.res_u[a] = 0.0;
  }
  s.iters_p = s.outer_p = s.iters_c = s.outer_c = 0;
  s.qs_iters = 0;
  s.qs_du = s.qs_dp = s.qs_dc = NAN;
  h->net_iters = h->net_fallback = 0;
  bool converged_qs = !qs || !(h->prm.qs_rtol > 0.0);
  for (int m = 0; m < M; ++m) {
    // S2: momentum predictor per component
    for (int a = 0; a < nd; ++a) {
      if (h->uprev[a] && !qs)
        launch_extrapolate(face_count(P, a), h->u[a], h->uprev[a], h->us[a], st);
      else
        cudaMemcpyAsync(h->us[a], h->u[a], face_count(P, a) * sizeof(double), cudaMemcpyDeviceToDevice, st);
      if (box_cells(S[a].box) == 0) continue;
      launch_mom_assemble(P, a, h->eps, h->kic, h->p, h->u[a], dtp, h->u, S[a].h.mg.omega, S[a].op64, S[a].rhs, st);
      SolveResult r = solve<T>(S[a].op64, S[a].h, S[a].rhs, unknown_view(h, a), h->prm.u_rtol, h->prm.max_iter,
                               h->work, h->rs, st, mom_mg);
      s.iters_u[a] += r.iters;
      s.outer_u[a] += r.outer;
      s.res_u[a] = r.relres;
      if (!r.converged) status = VOS_ENOCONV;
    }
    // S3: pressure correction, projection
    launch_pres_assemble(P, h->eps, h->us, h->R, dtp, S[3].h.mg.omega, S[3].op64, S[3].rhs, h->eps32, st);
    launch_defl_energy(S[3].h.defl, S[3].op64, st);
    // initial guess of the correction: zero, or the previous step's
    // correction (VOS_PRECOND_P_WARM; transient steps only -- in a
    // quasi-static step phi holds the previous concentration)
    if (qs || !(h->prm.precond & VOS_PRECOND_P_WARM)) cudaMemsetAsync(h->phi, 0, (size_t)N * sizeof(double), st);
    {
      SolveResult r = solve<T>(S[3].op64, S[3].h, S[3].rhs, unknown_view(h, 3), h->prm.p_rtol, h->prm.max_iter,
                               h->work, h->rs, st, true);
      h->net_iters += r.net_iters;
      h->net_fallback |= r.fallback;
      s.iters_p += r.iters;
      s.outer_p += r.outer;
      s.res_p = r.relres;
      if (!r.converged) status = VOS_ENOCONV;
    }
    if (qs) {
      launch_project_sums(P, h->eps, h->phi, dtp, h->us, h->u, h->p, h->dstats, h->rs, st);
      launch_qs_sums(N, false, h->p, h->phi, h->eps, h->dstats + ST_QSP, h->rs, st);  // phi is p^{m+1} - p^m
      // phi is dead from here on: it keeps c^m for the change of c
      cudaMemcpyAsync(h->phi, h->c, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
      launch_project(P, h->eps, h->phi, dtp, h->us, h->u, h->p, st);
    }
    // S4-S6: face data (convective fluxes of c^n; iVoS: reactive surface data
    // from eps^{n+1}, c^n), transport, rates.  us[a] is dead from the
    // projection until the next step copies u into it, so it holds the
    // convective face fluxes meanwhile.
    launch_face_data(P, ivos, h->eps, h->c, h->u, h->us, h->fd, st);
    if (!ivos) {
      launch_vos_lambda(P, h->eps, h->prm.lambda, h->prm.method == VOS_PSI_PRIME, h->dstats, h->rs, st);
      launch_vos_coef(P, h->eps, h->dstats, h->kr, st);
    }
    launch_trans_assemble(P, ivos, h->eps, h->eps_old, h->c, h->us, h->kr, h->fd, dtp, S[4].h.mg.omega, S[4].op64,
                          S[4].rhs, st);
    {
      SolveResult r = solve<T>(S[4].op64, S[4].h, S[4].rhs, unknown_view(h, 4), h->prm.c_rtol, h->prm.max_iter,
                               h->work, h->rs, st, true);
      s.iters_c += r.iters;
      s.outer_c += r.outer;
      s.res_c = r.relres;
      if (!r.converged) status = VOS_ENOCONV;
    }
    launch_rates(P, ivos, h->eps, h->c, h->kr, h->fd, h->R, h->Rf, h->dstats, h->rs, st);
    s.qs_iters = m + 1;
    if (qs) {
      launch_qs_sums(N, true, h->c, h->phi, nullptr, h->dstats + ST_QSC, h->rs, st);
      double q[10];
      cudaMemcpyAsync(q, h->dstats + ST_QSU, sizeof(q), cudaMemcpyDeviceToHost, st);
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_step: %s", cudaGetErrorString(e));
      const double dun = q[0] + q[2] + q[4], dud = q[1] + q[3] + q[5];
      s.qs_du = dud > 0.0 ? std::sqrt(dun / dud) : 0.0;
      s.qs_dp = q[7] > 0.0 ? std::sqrt(q[6] / q[7]) : 0.0;
      s.qs_dc = q[9] > 0.0 ? std::sqrt(q[8] / q[9]) : 0.0;
      const double tol = h->prm.qs_rtol;
      if (tol > 0.0 && s.qs_du <= tol && s.qs_dp <= tol && s.qs_dc <= tol) {
        converged_qs = true;
        break;
      }
    }
  }
  if (!converged_qs) status = VOS_ENOCONV;
  launch_step_diag(P, h->eps, h->u, h->R, h->c, h->us[0], h->dstats, h->rs, st);  // S7
  cudaMemcpyAsync(h->hstats, h->dstats, ST_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_step: %s", cudaGetErrorString(e));
  s.step += 1;
  s.t += dt;
  s.status = status;
  if (status == VOS_ENOCONV)
    set_err(h, VOS_ENOCONV, converged_qs ? "vos_step: a linear solve reached max_iter"
                                         : "vos_step: the quasi-static sub-iterations reached flow_subiters");
  return status;
}

// The step enqueued for graph capture (no host synchronisation inside).
template <typename T>
cudaError_t enqueue_step(vos_handle* h, Sys<T>* S, bool mom_mg) {
  const Phys& P = h->ph;
  cudaStream_t st = h->gs;
  const int nd = P.dim;
  const int ivos = (h->prm.method == VOS_IVOS);
  const double* dtp = h->d_dt;
  launch_eps_update(P, h->eps, h->eps_old, h->R, dtp, h->dstats, h->rs, h->kic, st);
  for (int a = 0; a < nd; ++a) {
    if (h->uprev[a])
      launch_extrapolate(face_count(P, a), h->u[a], h->uprev[a], h->us[a], st);
    else
      VOS_CUDA_TRY(cudaMemcpyAsync(h->us[a], h->u[a], face_count(P, a) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (box_cells(S[a].box) == 0) continue;
    launch_mom_assemble(P, a, h->eps, h->kic, h->p, h->u[a], dtp, h->u, S[a].h.mg.omega, S[a].op64, S[a].rhs, st);
    VOS_CUDA_TRY(solve_capture<T>(S[a].op64, S[a].h, S[a].rhs, unknown_view(h, a), h->prm.u_rtol, h->prm.max_iter,
                                  h->work, h->rs, st, mom_mg, h->dsolve + a, h->gs1, h->gs2));
  }
  launch_pres_assemble(P, h->eps, h->us, h->R, dtp, S[3].h.mg.omega, S[3].op64, S[3].rhs, h->eps32, st);
  launch_defl_energy(S[3].h.defl, S[3].op64, st);
  if (!(h->prm.precond & VOS_PRECOND_P_WARM))
    VOS_CUDA_TRY(cudaMemsetAsync(h->phi, 0, (size_t)P.nx * P.ny * P.nz * sizeof(double), st));
  VOS_CUDA_TRY(solve_capture<T>(S[3].op64, S[3].h, S[3].rhs, unknown_view(h, 3), h->prm.p_rtol, h->prm.max_iter,
                                h->work, h->rs, st, true, h->dsolve + 3, h->gs1, h->gs2));
  launch_project(P, h->eps, h->phi, dtp, h->us, h->u, h->p, st);
  launch_face_data(P, ivos, h->eps, h->c, h->u, h->us, h->fd, st);  // us: face-flux scratch (see the eager step)
  if (!ivos) {
    launch_vos_lambda(P, h->eps, h->prm.lambda, h->prm.method == VOS_PSI_PRIME, h->dstats, h->rs, st);
    launch_vos_coef(P, h->eps, h->dstats, h->kr, st);
  }
  launch_trans_assemble(P, ivos, h->eps, h->eps_old, h->c, h->us, h->kr, h->fd, dtp, S[4].h.mg.omega, S[4].op64,
                        S[4].rhs, st);
  VOS_CUDA_TRY(solve_capture<T>(S[4].op64, S[4].h, S[4].rhs, unknown_view(h, 4), h->prm.c_rtol, h->prm.max_iter,
                                h->work, h->rs, st, true, h->dsolve + 4, h->gs1, h->gs2));
  launch_rates(P, ivos, h->eps, h->c, h->kr, h->fd, h->R, h->Rf, h->dstats, h->rs, st);
  launch_step_diag(P, h->eps, h->u, h->R, h->c, h->us[0], h->dstats, h->rs, st);  // S7
  VOS_CUDA_TRY(cudaMemcpyAsync(h->hstats, h->dstats, ST_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  VOS_CUDA_TRY(cudaMemcpyAsync(h->hsolve, h->dsolve, 5 * sizeof(SolveStats), cudaMemcpyDeviceToHost, st));
  return cudaGetLastError();
}

template <typename T>
int finish_graph_step(vos_handle* h, Sys<T>* S, double dt);

template <typename T>
int step_graph(vos_handle* h, Sys<T>* S, double dt) {
  const bool mom_mg = mom_mg_for(h, dt);
  const int gi = mom_mg ? 1 : 0;
  if (!h->exec[gi]) {
    cudaError_t e = cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_step: begin capture: %s", cudaGetErrorString(e));
    cudaError_t ee = enqueue_step<T>(h, S, mom_mg);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->gs, &g);
    if (ee != cudaSuccess || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return set_err(h, VOS_ECUDA, "vos_step: graph capture failed: %s",
                     cudaGetErrorString(ee != cudaSuccess ? ee : e));
    }
    e = cudaGraphInstantiate(&h->exec[gi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->exec[gi] = nullptr;
      return set_err(h, VOS_ECUDA, "vos_step: graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  cudaEventRecord(h->ev_in, h->st);
  cudaStreamWaitEvent(h->gs, h->ev_in, 0);
  launch_set_scalar(h->d_dt, dt, h->gs);
  cudaGraphLaunch(h->exec[gi], h->gs);
  cudaEventRecord(h->ev_out, h->gs);
  cudaStreamWaitEvent(h->st, h->ev_out, 0);
  cudaError_t e = cudaStreamSynchronize(h->gs);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_step: %s", cudaGetErrorString(e));
  return finish_graph_step<T>(h, S, dt);
}

// Host side of a graph-replayed step once its graph has run: the solver
// statistics from the pinned copy the graph wrote.
template <typename T>
int finish_graph_step(vos_handle* h, Sys<T>* S, double dt) {
  const Phys& P = h->ph;
  vos_stats& s = h->stats;
  int status = VOS_OK;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < P.dim && box_cells(S[a].box) > 0;
    s.iters_u[a] = on ? h->hsolve[a].iters : 0;
    s.outer_u[a] = on ? h->hsolve[a].outer : 0;
    s.res_u[a] = on ? h->hsolve[a].relres : 0.0;
    if (on && !h->hsolve[a].converged) status = VOS_ENOCONV;
  }
  s.iters_p = h->hsolve[3].iters;
  s.outer_p = h->hsolve[3].outer;
  s.res_p = h->hsolve[3].relres;
  s.iters_c = h->hsolve[4].iters;
  s.outer_c = h->hsolve[4].outer;
  s.res_c = h->hsolve[4].relres;
  s.qs_iters = 1;
  s.qs_du = s.qs_dp = s.qs_dc = NAN;
  if (!h->hsolve[3].converged || !h->hsolve[4].converged) status = VOS_ENOCONV;
  s.step += 1;
  s.t += dt;
  s.status = status;
  if (status == VOS_ENOCONV) set_err(h, VOS_ENOCONV, "vos_step: a linear solve reached max_iter");
  return status;
}

void drop_graphs(vos_handle* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->exec[i]) cudaGraphExecDestroy(h->exec[i]);
    h->exec[i] = nullptr;
  }
  h->graph_gen += 1;  // graphs that captured this handle elsewhere (batch) are stale too
}

// Label the floating pore clusters of the pressure operator for the host
// fluid fraction eps and upload them; the pressure hierarchies of both
// precisions point at the result.  Captured graphs hold the old launch
// configuration, so they are dropped.
int setup_deflation(vos_handle* h, const double* eps) {
  const Phys& P = h->ph;
  Defl D{0, nullptr, nullptr, nullptr};
  if (!(h->prm.precond & VOS_PRECOND_NO_DEFLATION)) {
    std::vector<int> ptr;
    std::vector<unsigned long long> ent;
    const int K = floating_clusters(eps, P.nx, P.ny, P.nz, kDeflTheta, ptr, ent, nullptr);
    if (K > 0) {
      const size_t b0 = align256((size_t)(K + 1) * sizeof(int)), b1 = align256(ent.size() * sizeof(unsigned long long));
      const size_t need = b0 + b1 + align256((size_t)K * sizeof(double));
      if (need > h->defl_cap) {
        if (h->defl_mem) dev_free(h, h->defl_mem);
        h->defl_cap = 0;
        h->defl_mem = dev_alloc(h, need);
        if (!h->defl_mem) return set_err(h, VOS_ENOMEM, "device allocation failed (deflation)");
        h->defl_cap = need;
      }
      char* cur = (char*)h->defl_mem;
      D.K = K;
      D.ptr = (const int*)cur;
      D.ent = (const unsigned long long*)(cur + b0);
      D.Einv = (double*)(cur + b0 + b1);
      cudaMemcpyAsync((void*)D.ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, h->st);
      cudaMemcpyAsync((void*)D.ent, ent.data(), ent.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, h->st);
      cudaMemsetAsync(D.Einv, 0, (size_t)K * sizeof(double), h->st);
      // the copies read the host vectors: finish them before they go away
      cudaError_t e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "deflation upload: %s", cudaGetErrorString(e));
    }
  }
  h->defl = D;
  h->sd[3].h.defl = D;
  h->sf[3].h.defl = D;
  drop_graphs(h);
  return VOS_OK;
}

int validate(const vos_params* p) {
  if (!p) return set_err(nullptr, VOS_EINVAL, "params is NULL");
  if (p->dim != 2 && p->dim != 3) return set_err(nullptr, VOS_EINVAL, "dim must be 2 or 3 (got %d)", p->dim);
  if (p->nx < 2 || p->ny < 1 || p->nz < 1) return set_err(nullptr, VOS_EINVAL, "need nx >= 2, ny >= 1, nz >= 1");
  if (p->dim == 2 && p->nz != 1) return set_err(nullptr, VOS_EINVAL, "dim 2 needs nz == 1");
  if ((double)p->nx * p->ny * p->nz > 1.0e9) return set_err(nullptr, VOS_EINVAL, "grid too large");
  const double vals[] = {p->dx, p->k0, p->eps_min};
  for (double v : vals)
    if (!(v > 0.0) || !std::isfinite(v)) return set_err(nullptr, VOS_EINVAL, "dx, k0, eps_min must be > 0");
  if (!(p->eps_min < 1.0)) return set_err(nullptr, VOS_EINVAL, "eps_min must be < 1");
  const double nn[] = {p->nu, p->D, p->kc, p->Vm, p->zeta, p->rho_ratio, p->c_in, p->lambda};
  for (double v : nn)
    if (!(v >= 0.0) || !std::isfinite(v))
      return set_err(nullptr, VOS_EINVAL, "nu, D, kc, Vm, zeta, rho_ratio, c_in, lambda must be finite and >= 0");
  if (!std::isfinite(p->u_in)) return set_err(nullptr, VOS_EINVAL, "u_in must be finite");
  if (p->method < 0 || p->method > 2) return set_err(nullptr, VOS_EINVAL, "unknown method %d", p->method);
  if (p->precision < 0 || p->precision > 1) return set_err(nullptr, VOS_EINVAL, "unknown precision %d", p->precision);
  if (p->precond & ~(VOS_PRECOND_NO_DEFLATION | VOS_PRECOND_MOM_DIAG | VOS_PRECOND_MOM_MG | VOS_PRECOND_P_WARM |
                     VOS_PRECOND_U_EXTRAP))
    return set_err(nullptr, VOS_EINVAL, "unknown precond flags %d", p->precond);
  if ((p->precond & VOS_PRECOND_MOM_DIAG) && (p->precond & VOS_PRECOND_MOM_MG))
    return set_err(nullptr, VOS_EINVAL, "VOS_PRECOND_MOM_DIAG and VOS_PRECOND_MOM_MG exclude each other");
  if (p->flow_subiters < 1) return set_err(nullptr, VOS_EINVAL, "flow_subiters must be >= 1");
  if (p->inertia != 0 && p->inertia != 1) return set_err(nullptr, VOS_EINVAL, "inertia must be 0 or 1");
  if (!(p->qs_rtol >= 0.0) || !std::isfinite(p->qs_rtol) || !(p->qs_dtau >= 0.0) || !std::isfinite(p->qs_dtau))
    return set_err(nullptr, VOS_EINVAL, "qs_rtol and qs_dtau must be finite and >= 0");
  const double tol[] = {p->p_rtol, p->u_rtol, p->c_rtol};
  for (double v : tol)
    if (!(v > 0.0) || !(v < 1.0)) return set_err(nullptr, VOS_EINVAL, "tolerances must be in (0, 1)");
  if (p->max_iter < 1) return set_err(nullptr, VOS_EINVAL, "max_iter must be >= 1");
  return VOS_OK;
}

}  // namespace

extern "C" {

int vos_create(const double* eps_s_host, const vos_params* prm, void* stream, const vos_allocator* alloc,
               vos_handle** out) {
  if (!out) return set_err(nullptr, VOS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(prm);
  if (rc) return rc;
  if (!eps_s_host) return set_err(nullptr, VOS_EINVAL, "eps_s is NULL");
  if (alloc && (!alloc->alloc || !alloc->free)) return set_err(nullptr, VOS_EINVAL, "allocator needs alloc and free");
  const long long N = (long long)prm->nx * prm->ny * prm->nz;
  for (long long c = 0; c < N; ++c) {
    double v = eps_s_host[c];
    if (!(v >= 0.0 && v <= 1.0)) return set_err(nullptr, VOS_EINVAL, "eps_s[%lld] = %g not in [0, 1]", c, v);
  }
  vos_handle* h = new vos_handle();
  h->prm = *prm;
  Phys& P = h->ph;
  P.dim = prm->dim;
  P.nx = prm->nx;
  P.ny = prm->ny;
  P.nz = prm->nz;
  P.dx = prm->dx;
  P.nu = prm->nu;
  P.D = prm->D;
  P.kc = prm->kc;
  P.k0 = prm->k0;
  P.Vm = prm->Vm;
  P.zeta = prm->zeta;
  P.rho_ratio = prm->rho_ratio;
  P.c_in = prm->c_in;
  P.u_in = prm->u_in;
  P.eps_min = prm->eps_min;
  P.wall_mask = prm->wall_mask;
  P.inertia = prm->inertia != 0;
  h->st = (cudaStream_t)stream;
  h->user_alloc = (alloc != nullptr);
  if (alloc) h->alloc = *alloc;
  h->bytes = 0;
  h->work = nullptr;
  h->hstats = nullptr;
  h->hsolve = nullptr;
  h->dsolve = nullptr;
  h->gs = h->gs1 = h->gs2 = nullptr;
  h->ev_in = h->ev_out = nullptr;
  h->exec[0] = h->exec[1] = nullptr;
  h->defl_mem = nullptr;
  h->defl_cap = 0;
  h->defl = Defl{0, nullptr, nullptr, nullptr};
  h->net = nullptr;
  h->graph_gen = 0;
  h->net_iters = h->net_fallback = 0;
  std::memset(&h->stats, 0, sizeof(h->stats));
  cudaGetDevice(&h->dev);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev) == cudaSuccess && sms > 0) g_num_sms = sms;

  const size_t cb = (size_t)N * sizeof(double);
  auto fail = [&](int code, const char* what) {
    set_err(nullptr, code, "vos_create: %s", what);
    free_all(h);
    delete h;
    return code;
  };
  double** cells[] = {&h->eps, &h->eps_old, &h->c, &h->p, &h->phi, &h->R, &h->Rf, &h->kr, &h->kic};
  for (double** f : cells) {
    *f = (double*)dev_alloc(h, cb);
    if (!*f) return fail(VOS_ENOMEM, "device allocation failed (cell fields)");
  }
  for (int a = 0; a < 3; ++a) {
    h->u[a] = h->us[a] = h->uprev[a] = nullptr;
    h->fd[a] = FaceData{nullptr, nullptr, nullptr};
    if (a >= P.dim) continue;
    size_t fb = (size_t)face_count(P, a) * sizeof(double);
    h->u[a] = (double*)dev_alloc(h, fb);
    h->us[a] = (double*)dev_alloc(h, fb);
    if (!h->u[a] || !h->us[a]) return fail(VOS_ENOMEM, "device allocation failed (face fields)");
    if (prm->precond & VOS_PRECOND_U_EXTRAP) {
      h->uprev[a] = (double*)dev_alloc(h, fb);
      if (!h->uprev[a]) return fail(VOS_ENOMEM, "device allocation failed (face fields)");
    }
    if (prm->method == VOS_IVOS) {
      h->fd[a].s = (double*)dev_alloc(h, fb);
      h->fd[a].corr = (double*)dev_alloc(h, fb);
      h->fd[a].evl = (double*)dev_alloc(h, fb);
      if (!h->fd[a].s || !h->fd[a].corr || !h->fd[a].evl) return fail(VOS_ENOMEM, "device allocation failed (iVoS)");
    }
  }
  h->eps32 = nullptr;
  if (prm->precision != VOS_FP64) {
    h->eps32 = (float*)dev_alloc(h, (size_t)N * sizeof(float));
    if (!h->eps32) return fail(VOS_ENOMEM, "device allocation failed (eps32)");
    cudaMemsetAsync(h->eps32, 0, (size_t)N * sizeof(float), h->st);
  }
  const int trans_sym = (prm->method == VOS_IVOS) ? 0 : 1;
  for (int sys = 0; sys < 5; ++sys) {
    if (sys < 3 && sys >= P.dim) {
      h->sd[sys].box = Box{0, 0, 0};
      h->sf[sys].box = Box{0, 0, 0};
      continue;
    }
    int sym = (sys == 4) ? trans_sym : 1;
    bool ok = (prm->precision == VOS_FP64) ? alloc_sys<double>(h, h->sd[sys], sys, sym)
                                           : alloc_sys<float>(h, h->sf[sys], sys, sym);
    if (!ok) return fail(VOS_ENOMEM, "device allocation failed (solver)");
  }
  if (prm->precision != VOS_FP64) {  // FP32 momentum fine levels: constant links -nu/dx^2
    for (int a = 0; a < P.dim; ++a)
      if (h->sf[a].h.nlev > 0) h->sf[a].h.lev[0].op.mfc = (float)(-P.nu / (P.dx * P.dx));
  }
  if (h->eps32 && h->sf[3].h.nlev > 0) {  // the FP32 pressure fine level runs matrix-free
    h->sf[3].h.lev[0].op.mfe = h->eps32;
    h->sf[3].h.lev[0].op.mfs = (float)(1.0 / (P.dx * P.dx));
  }
  {
    long long maxc = 0;
    for (int sys = 0; sys < 5; ++sys) {
      Box b = (prm->precision == VOS_FP64) ? h->sd[sys].box : h->sf[sys].box;
      if (box_cells(b) > maxc) maxc = box_cells(b);
    }
    char* cur = (char*)dev_alloc(h, solver_work_bytes(maxc));
    if (!cur) return fail(VOS_ENOMEM, "device allocation failed (Krylov vectors)");
    h->work = solver_work_carve(cur, maxc);
    char* rsb = (char*)dev_alloc(h, kMaxRedValues * kMaxRedBlocks * sizeof(double) + 256 + ST_COUNT * sizeof(double) + 256);
    if (!rsb) return fail(VOS_ENOMEM, "device allocation failed (reduction scratch)");
    h->rs.partials = (double*)rsb;
    h->rs.counter = (unsigned int*)(rsb + kMaxRedValues * kMaxRedBlocks * sizeof(double));
    h->dstats = (double*)(rsb + kMaxRedValues * kMaxRedBlocks * sizeof(double) + 256);
    h->d_dt = h->dstats + ST_COUNT;
    h->dups = h->d_dt + 1;  // 6 doubles, inside the block's 256-byte tail
  }
  for (int sys = 0; sys < 5; ++sys) {
    if (prm->precision == VOS_FP64) {
      if (box_cells(h->sd[sys].box) > 0) autotune_hier<double>(h->sd[sys].h, h->work, h->st);
    } else {
      if (box_cells(h->sf[sys].box) > 0) autotune_hier<float>(h->sf[sys].h, h->work, h->st);
    }
  }
  if (cudaMallocHost((void**)&h->hstats, ST_COUNT * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hsolve, 5 * sizeof(SolveStats)) != cudaSuccess)
    return fail(VOS_ENOMEM, "pinned host allocation failed");
  h->dsolve = (SolveStats*)dev_alloc(h, 5 * sizeof(SolveStats));
  if (!h->dsolve) return fail(VOS_ENOMEM, "device allocation failed (solve stats)");
  if (cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->gs1, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->gs2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(VOS_ECUDA, "stream/event creation failed");
  std::memset(h->hstats, 0, ST_COUNT * sizeof(double));
  // initial fields (App. C: eps = max(1 - eps_s, eps_min))
  std::vector<double> e0(N);
  double esum = 0.0;
  for (long long c = 0; c < N; ++c) {
    e0[c] = std::fmax(1.0 - eps_s_host[c], prm->eps_min);
    esum += e0[c];
  }
  cudaStream_t st = h->st;
  cudaMemcpyAsync(h->eps, e0.data(), cb, cudaMemcpyHostToDevice, st);
  for (double* f : {h->eps_old, h->c, h->p, h->phi, h->R, h->Rf, h->kr, h->kic}) cudaMemsetAsync(f, 0, cb, st);
  for (int a = 0; a < P.dim; ++a) {
    size_t fb = (size_t)face_count(P, a) * sizeof(double);
    cudaMemsetAsync(h->u[a], 0, fb, st);
    cudaMemsetAsync(h->us[a], 0, fb, st);
  }
  {
    // inlet faces u = u_in (face i = 0 of every (j,k) row)
    std::vector<double> u0((size_t)face_count(P, 0), 0.0);
    for (long long r = 0; r < (long long)P.ny * P.nz; ++r) u0[(size_t)r * (P.nx + 1)] = prm->u_in;
    cudaMemcpyAsync(h->u[0], u0.data(), u0.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    for (int a = 0; a < P.dim; ++a)  // no history yet: the extrapolation starts from u
      if (h->uprev[a])
        cudaMemcpyAsync(h->uprev[a], h->u[a], (size_t)face_count(P, a) * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(h->rs.counter, 0, sizeof(unsigned int), st);
    cudaMemsetAsync(h->dstats, 0, ST_COUNT * sizeof(double), st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(cudaGetLastError()));
  }
  rc = setup_deflation(h, e0.data());
  if (rc != VOS_OK) return fail(rc, h->err.c_str());
  h->stats.porosity = esum / (double)N;
  h->stats.lambda = (prm->method == VOS_PSI) ? prm->lambda : NAN;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VOS_ECUDA, cudaGetErrorString(e));
  *out = h;
  return VOS_OK;
}

int vos_step(vos_handle* h, double dt) {
  if (!h) return set_err(nullptr, VOS_EINVAL, "handle is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(h, VOS_EINVAL, "dt must be finite and > 0");
  // CUDA-graph replay unless per-kernel timing is on (timing brackets each
  // launch with events, so it uses the eager launch sequence -- the same
  // kernels in the same order).
  const bool graphs = g_use_graphs && !vos::g_prof_any && !h->net && h->prm.flow_subiters <= 1;
  h->net_iters = h->net_fallback = 0;
  if (h->prm.precision == VOS_FP64) return graphs ? step_graph<double>(h, h->sd, dt) : step_impl<double>(h, h->sd, dt);
  return graphs ? step_graph<float>(h, h->sf, dt) : step_impl<float>(h, h->sf, dt);
}

int vos_fields(vos_handle* h, uint32_t mask, double* eps, double* c, double* u, double* v, double* w, double* p,
               double* R, double* Rf) {
  if (!h) return set_err(nullptr, VOS_EINVAL, "handle is NULL");
  const Phys& P = h->ph;
  const size_t cb = (size_t)P.nx * P.ny * P.nz * sizeof(double);
  struct Item {
    uint32_t bit;
    double* dst;
    const double* src;
    size_t bytes;
  } items[] = {
      {VOS_F_EPS, eps, h->eps, cb},
      {VOS_F_C, c, h->c, cb},
      {VOS_F_U, u, h->u[0], (size_t)face_count(P, 0) * 8},
      {VOS_F_V, v, h->u[1], (size_t)face_count(P, 1) * 8},
      {VOS_F_W, w, h->u[2], P.dim == 3 ? (size_t)face_count(P, 2) * 8 : 0},
      {VOS_F_P, p, h->p, cb},
      {VOS_F_R, R, h->R, cb},
      {VOS_F_RF, Rf, h->Rf, cb},
  };
  for (auto& it : items) {
    if (!(mask & it.bit) || !it.dst || !it.src || it.bytes == 0) continue;
    cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost, h->st);
  }
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_fields: %s", cudaGetErrorString(e));
  return VOS_OK;
}

int vos_set_fields(vos_handle* h, uint32_t mask, const double* eps, const double* c, const double* u, const double* v,
                   const double* w, const double* p, const double* R, const double* Rf) {
  if (!h) return set_err(nullptr, VOS_EINVAL, "handle is NULL");
  const Phys& P = h->ph;
  const size_t cb = (size_t)P.nx * P.ny * P.nz * sizeof(double);
  struct Item {
    uint32_t bit;
    double* dst;
    const double* src;
    size_t bytes;
  } items[] = {
      {VOS_F_EPS, h->eps, eps, cb},
      {VOS_F_C, h->c, c, cb},
      {VOS_F_U, h->u[0], u, (size_t)face_count(P, 0) * 8},
      {VOS_F_V, h->u[1], v, (size_t)face_count(P, 1) * 8},
      {VOS_F_W, h->u[2], w, P.dim == 3 ? (size_t)face_count(P, 2) * 8 : 0},
      {VOS_F_P, h->p, p, cb},
      {VOS_F_R, h->R, R, cb},
      {VOS_F_RF, h->Rf, Rf, cb},
  };
  for (auto& it : items) {
    if (!(mask & it.bit) || !it.dst || !it.src || it.bytes == 0) continue;
    cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyHostToDevice, h->st);
  }
  for (int a = 0; a < P.dim; ++a)  // a resumed velocity has no history: restart the extrapolation
    if (h->uprev[a] && (mask & (VOS_F_U | VOS_F_V | VOS_F_W)))
      cudaMemcpyAsync(h->uprev[a], h->u[a], (size_t)face_count(P, a) * sizeof(double), cudaMemcpyDeviceToDevice,
                      h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_set_fields: %s", cudaGetErrorString(e));
  if ((mask & VOS_F_EPS) && eps) return setup_deflation(h, eps);
  return VOS_OK;
}

int vos_device_fields_get(vos_handle* h, vos_device_fields* out) {
  if (!h || !out) return set_err(h, VOS_EINVAL, "NULL argument");
  out->eps = h->eps;
  out->c = h->c;
  out->p = h->p;
  out->u = h->u[0];
  out->v = h->u[1];
  out->w = h->u[2];
  out->R = h->R;
  out->Rf = h->Rf;
  return VOS_OK;
}

int vos_get_stats(vos_handle* h, vos_stats* out) {
  if (!h || !out) return set_err(h, VOS_EINVAL, "NULL argument");
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_get_stats: %s", cudaGetErrorString(e));
  const Phys& P = h->ph;
  vos_stats s = h->stats;
  if (s.step > 0) {
    s.clamp_excess = h->hstats[ST_CLAMP];
    s.porosity = h->hstats[ST_EPSSUM] / ((double)P.nx * P.ny * P.nz);
    s.sum_R = h->hstats[ST_SUMR];
    s.sum_Rf = h->hstats[ST_SUMRF];
    s.reactant = h->hstats[ST_REACT];
    s.lambda = (h->prm.method == VOS_IVOS) ? NAN : h->hstats[ST_LAMBDA];
    s.q_in = h->hstats[ST_QIN];
    s.q_out = h->hstats[ST_QOUT];
    s.flux_in = h->hstats[ST_FIN];
    s.flux_out = h->hstats[ST_FOUT];
    s.umax = h->hstats[ST_UMAX];
    s.rmax = h->hstats[ST_RMAX];
  }
  *out = s;
  return VOS_OK;
}

int vos_upscaled(vos_handle* h, vos_upscaled_props* out) {
  if (!h || !out) return set_err(h, VOS_EINVAL, "vos_upscaled: NULL argument");
  const Phys& P = h->ph;
  launch_upscaled_sums(P, h->eps, h->c, h->p, h->u[0], h->dups, h->rs, h->st);
  double v[6];
  cudaMemcpyAsync(v, h->dups, sizeof(v), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_upscaled: %s", cudaGetErrorString(e));
  const double N = (double)P.nx * P.ny * P.nz;
  const double A = (P.dim == 2) ? P.dx : P.dx * P.dx;
  const double V = A * P.dx;
  vos_upscaled_props r;
  r.phi = v[0] / N;
  r.Q_in = v[5] * A;
  r.A_in = (double)P.ny * P.nz * A;
  r.U_D = r.Q_in / r.A_in;
  r.dP = v[4] / ((double)P.ny * P.nz);
  r.L_D = (P.nx - 0.5) * P.dx;
  r.K = (r.dP != 0.0) ? P.nu * r.U_D * r.L_D / r.dP : NAN;
  r.a = v[1] * V / (N * V);
  const double cs = v[2] * V, cv = v[3] * V;
  r.alpha = (r.a != 0.0 && cv != 0.0) ? (cs / cv) / r.a : NAN;
  const double f = (P.dim == 2) ? 12.0 : 8.0;
  r.L_ref = (r.K == r.K && r.K > 0.0) ? std::sqrt(f * r.K / r.phi) : NAN;
  r.U_ref = r.U_D / r.phi;
  r.Pe = (P.D > 0.0) ? r.U_ref * r.L_ref / P.D : NAN;
  r.Da = (r.U_ref != 0.0) ? P.kc / r.U_ref : NAN;
  r.Ki = r.Da * r.Pe;
  *out = r;
  return VOS_OK;
}

int vos_suggest_dt(vos_handle* h, double cfl, double deps_max, double* dt) {
  if (!h || !dt) return set_err(h, VOS_EINVAL, "NULL argument");
  if (!(cfl > 0.0) || !(deps_max > 0.0)) return set_err(h, VOS_EINVAL, "cfl and deps_max must be > 0");
  launch_dt_limits(h->ph, h->eps, h->u, h->R, h->dstats, h->rs, h->st);
  double v[2];
  cudaMemcpyAsync(v, h->dstats + ST_UMAX, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_suggest_dt: %s", cudaGetErrorString(e));
  double d1 = v[0] > 0.0 ? cfl * h->ph.dx / v[0] : INFINITY;
  double d2 = v[1] > 0.0 ? deps_max / v[1] : INFINITY;
  *dt = d1 < d2 ? d1 : d2;
  return VOS_OK;
}

const char* vos_last_error(const vos_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void vos_destroy(vos_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  free_all(h);
  delete h;
}

size_t vos_device_bytes(const vos_handle* h) { return h ? h->bytes : 0; }

int vos_fp64_div_check(const double* a, const double* d, int64_t n, double* q_fast, double* q_ieee) {
  if (n < 0) return set_err(nullptr, VOS_EINVAL, "vos_fp64_div_check: n < 0");
  if (n == 0) return VOS_OK;
  if (!a || !d || !q_fast || !q_ieee) return set_err(nullptr, VOS_EINVAL, "vos_fp64_div_check: NULL array");
  launch_div_check(a, d, (long long)n, q_fast, q_ieee, 0);
  cudaError_t e = cudaStreamSynchronize(0);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(nullptr, VOS_ECUDA, "vos_fp64_div_check: %s", cudaGetErrorString(e));
  return VOS_OK;
}

int vos_tile_config(const vos_handle* h, int32_t sys, int32_t level, int32_t* tx, int32_t* ty, int32_t* zc,
                    int32_t* tuned) {
  if (!h || !tx || !ty || !zc || !tuned) return set_err(nullptr, VOS_EINVAL, "vos_tile_config: NULL argument");
  if (sys < 0 || sys > 4) return set_err(nullptr, VOS_EINVAL, "vos_tile_config: sys must be 0..4");
  const bool fp64 = h->prm.precision == VOS_FP64;
  const int nlev = fp64 ? h->sd[sys].h.nlev : h->sf[sys].h.nlev;
  if (level < 0 || level >= nlev) return set_err(nullptr, VOS_EINVAL, "vos_tile_config: level out of range");
  Box b = fp64 ? h->sd[sys].h.lev[level].op.box : h->sf[sys].h.lev[level].op.box;
  int sym = fp64 ? h->sd[sys].h.lev[level].op.sym : h->sf[sys].h.lev[level].op.sym;
  if (!fp64 && sym && h->sf[sys].h.lev[level].op.mfe) sym = 2;  // matrix-free sweep, tuned on its own
  if (b.mz == 1 && b.my > 1) b = Box{b.mx, 1, b.my};  // 2D boxes march along y
  int x = 0, y = 0, z = 0;
  if (tuned_config(b.mx, b.my, b.mz, fp64 ? 8 : 4, sym, &x, &y, &z)) {
    *tuned = 1;
  } else {
    *tuned = 0;
    default_sweep_config(b.mx, b.my, b.mz, &x, &y, &z);
  }
  *tx = x;
  *ty = y;
  *zc = z;
  return VOS_OK;
}

int vos_set_unet_preconditioner(vos_handle* h, vos_unet* net) {
  if (!h) return set_err(nullptr, VOS_EINVAL, "vos_set_unet_preconditioner: handle is NULL");
  if (net) {
    const Box b = h->sd[3].box.mx ? h->sd[3].box : h->sf[3].box;
    int px = 0, py = 0, pz = 0;
    unet_box(net, &px, &py, &pz);
    if (px != b.mx || py != b.my || pz != b.mz)
      return set_err(h, VOS_EINVAL, "vos_set_unet_preconditioner: network box %dx%dx%d, grid %dx%dx%d", px, py, pz,
                     b.mx, b.my, b.mz);
    unet_attach_eps(net, h->eps);
  }
  h->net = net;
  h->graph_gen += 1;
  h->sd[3].h.net = net;
  h->sf[3].h.net = net;
  return VOS_OK;
}

int vos_unet_solve_stats(const vos_handle* h, int32_t* net_iters, int32_t* fallback) {
  if (!h || !net_iters || !fallback) return set_err(nullptr, VOS_EINVAL, "vos_unet_solve_stats: NULL argument");
  *net_iters = h->net_iters;
  *fallback = h->net_fallback;
  return VOS_OK;
}

int vos_pressure_snapshots(vos_handle* h, int32_t count, const int32_t* iters, float* out) {
  if (!h || count < 1 || !iters || !out) return set_err(nullptr, VOS_EINVAL, "vos_pressure_snapshots: bad argument");
  for (int i = 0; i < count; ++i)
    if (iters[i] < 0 || iters[i] > 100000) return set_err(h, VOS_EINVAL, "vos_pressure_snapshots: iters out of range");
  if (h->stats.step < 1) return set_err(h, VOS_EINVAL, "vos_pressure_snapshots: no step taken yet");
  const Phys& P = h->ph;
  cudaStream_t st = h->st;
  cudaMemsetAsync(h->phi, 0, (size_t)P.nx * P.ny * P.nz * sizeof(double), st);
  std::vector<int> it(iters, iters + count);
  int rc;
  if (h->prm.precision == VOS_FP64)
    rc = residual_snapshots<double>(h->sd[3].op64, h->sd[3].h, h->sd[3].rhs, unknown_view(h, 3), h->work, h->rs, st,
                                    count, it.data(), out);
  else
    rc = residual_snapshots<float>(h->sf[3].op64, h->sf[3].h, h->sf[3].rhs, unknown_view(h, 3), h->work, h->rs, st,
                                   count, it.data(), out);
  cudaError_t e = cudaGetLastError();
  if (rc != 0 || e != cudaSuccess) return set_err(h, VOS_ECUDA, "vos_pressure_snapshots: %s", cudaGetErrorString(e));
  return VOS_OK;
}

int vos_floating_clusters(const double* eps, const vos_params* prm, int32_t* label, int32_t* nclusters,
                          int64_t* ncells) {
  if (!eps || !nclusters) return set_err(nullptr, VOS_EINVAL, "vos_floating_clusters: NULL argument");
  int rc = validate(prm);
  if (rc) return rc;
  std::vector<int> ptr;
  std::vector<unsigned long long> ent;
  *nclusters = floating_clusters(eps, prm->nx, prm->ny, prm->nz, kDeflTheta, ptr, ent, label);
  if (ncells) *ncells = (int64_t)ent.size();
  return VOS_OK;
}

int vos_set_launch_mode(int graphs) {
  g_use_graphs = graphs != 0;
  return VOS_OK;
}

int vos_set_vector_sweeps(int on) {
  vos::g_mf4 = on != 0;
  return VOS_OK;
}

int vos_set_fused_pcg(int mask) {
  if (mask < 0 || mask > 7) return VOS_EINVAL;
  vos::g_fused_pcg = mask;
  return VOS_OK;
}

int vos_set_coarse_cycle(int on) {
  vos::g_tail_enabled = on != 0;
  return VOS_OK;
}

}  // extern "C"

namespace vos {
const Op<double>* handle_pressure_op(vos_handle* h) {
  if (!h) return nullptr;
  return h->prm.precision == VOS_FP64 ? &h->sd[3].op64 : &h->sf[3].op64;
}
const double* handle_eps(vos_handle* h) { return h ? h->eps : nullptr; }
}  // namespace vos

// ---------------------------------------------------------------------------
// Batch support (vos_batch.cu): one CUDA graph holding the steps of many
// handles as parallel branches.
// ---------------------------------------------------------------------------
namespace vos {
bool graphs_enabled() { return g_use_graphs && !g_prof_any; }
bool batch_graphable(const vos_handle* h) { return h->net == nullptr && h->prm.flow_subiters <= 1; }
unsigned batch_generation(const vos_handle* h) { return h->graph_gen; }
int batch_key(const vos_handle* h, double dt) { return mom_mg_for(h, dt) ? 1 : 0; }
double* batch_dt_slot(vos_handle* h) { return h->d_dt; }
// Enqueue h's step on its internal stream inside an active capture: fork
// from `fork` (recorded on the capture's origin stream), join into `join`,
// which the origin then waits for.
cudaError_t batch_enqueue(vos_handle* h, int key, cudaEvent_t fork, cudaEvent_t* join) {
  VOS_CUDA_TRY(cudaStreamWaitEvent(h->gs, fork, 0));
  cudaError_t e = (h->prm.precision == VOS_FP64) ? enqueue_step<double>(h, h->sd, key != 0)
                                                 : enqueue_step<float>(h, h->sf, key != 0);
  if (e != cudaSuccess) return e;
  VOS_CUDA_TRY(cudaEventRecord(h->ev_out, h->gs));
  *join = h->ev_out;
  return cudaSuccess;
}
int batch_finish(vos_handle* h, double dt) {
  return (h->prm.precision == VOS_FP64) ? finish_graph_step<double>(h, h->sd, dt)
                                        : finish_graph_step<float>(h, h->sf, dt);
}
}  // namespace vos
