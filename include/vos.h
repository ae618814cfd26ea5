/*
 * vos.h -- C ABI of the GB300 micro-continuum dissolution step.
 *
 * Method: Maes, Soulaine & Menke, "Improved Volume-of-Solid formulations for
 * micro-continuum simulation of mineral dissolution at the pore-scale".
 * One call to vos_step advances, on a uniform Cartesian grid (2D or 3D):
 *   S1  solid fraction eps by the solid mass balance (Sec. 2.2, Eq. mbs) and
 *       the Kozeny-Carman permeability (Eq. perm);
 *   S2  Darcy-Brinkman-Stokes momentum predictor (Eq. momentumDBS);
 *   S3  pressure correction and projection (Eq. contDBS);
 *   S4  explicit van Leer advection of the reactant (App. B);
 *   S5  implicit diffusion + reaction of the reactant (Eq. concentrationDBS);
 *   S6  reaction rates R (solid source) and R_f (transport sink) by
 *       VoS-psi (Eq. RfVoSpsi, lambda = 4), VoS-psi' (lambda fitted from
 *       global integrals, Sec. 2.4) or iVoS (Eq. RfiVoS, Sec. 2.3);
 *   S7  global FP64 diagnostics.
 * Grid: MAC staggered -- scalars at cell centres, velocity components on
 * the faces normal to them.  Cell index i + nx*(j + ny*k) (x fastest).
 * u: (nx+1)*ny*nz values, index i + (nx+1)*(j + ny*k), i = 0 the inlet face;
 * v: nx*(ny+1)*nz, index i + nx*(j + (ny+1)*k);
 * w: nx*ny*(nz+1), index i + nx*(j + ny*k), k in [0, nz] (3D only).
 * Boundaries: x- inlet (u = u_in, c = c_in), x+ outlet (p = 0, zero
 * gradient), y+-/z+- no-slip walls where wall_mask has the bit, free-slip
 * otherwise.
 *
 * Every function returns VOS_OK (0) or a negative error code; the message
 * of the last error on a handle is returned by vos_last_error.  A handle is
 * not thread-safe; different handles are independent.  All device work is
 * enqueued on the stream given to vos_create.
 */
#ifndef VOS_H_
#define VOS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VOS_OK 0
#define VOS_EINVAL (-1)   /* bad size, parameter, NaN or NULL pointer        */
#define VOS_ENOMEM (-2)   /* device allocation failed                       */
#define VOS_ECUDA (-3)    /* a CUDA call failed (message has the CUDA text) */
#define VOS_ETIMEOUT (-5) /* a bounded device wait gave up (tensor-core path) */
#define VOS_ENOCONV (-4)  /* a linear solve hit max_iter; the step was still
                             applied with the last iterate                  */

typedef enum { VOS_PSI = 0, VOS_PSI_PRIME = 1, VOS_IVOS = 2 } vos_method;
typedef enum { VOS_FP64 = 0, VOS_MIXED = 1 } vos_precision;

/* wall_mask bits: no-slip wall on that side (else free-slip) */
#define VOS_WALL_YM 1u
#define VOS_WALL_YP 2u
#define VOS_WALL_ZM 4u
#define VOS_WALL_ZP 8u

/* field mask bits for vos_fields / vos_set_fields */
#define VOS_F_EPS 1u
#define VOS_F_C 2u
#define VOS_F_U 4u
#define VOS_F_V 8u
#define VOS_F_W 16u
#define VOS_F_P 32u
#define VOS_F_R 64u
#define VOS_F_RF 128u

/* Preconditioner flags (vos_params.precond).  0 (default): the pressure and
 * transport solves use the multigrid V-cycle (Galerkin aggregation, damped
 * Jacobi); each momentum solve uses it when the viscous term dominates the
 * mass term (2 dim nu dt / dx^2 > 30) and the diagonal (Jacobi)
 * preconditioner otherwise; the pressure solve adds the deflation of
 * floating pore clusters (pockets of pore cells joined to the outlet only
 * through solid cells; see vos_floating_clusters).
 * VOS_PRECOND_NO_DEFLATION drops the deflation; VOS_PRECOND_MOM_DIAG /
 * VOS_PRECOND_MOM_MG make every momentum solve use the diagonal / the
 * multigrid preconditioner whatever dt is (at most one of the two);
 * VOS_PRECOND_P_WARM starts the pressure-correction solve of a transient
 * step from the previous step's correction instead of zero;
 * VOS_PRECOND_U_EXTRAP starts the momentum solves of a transient step from
 * the extrapolation 2 u^n - u^{n-1} instead of u^n (one more velocity field
 * in device memory; restarted from u when vos_set_fields sets it).
 * Solver aids, not part of the paper's method: they change the iteration
 * count, not the converged solution. */
#define VOS_PRECOND_NO_DEFLATION 1
#define VOS_PRECOND_MOM_DIAG 2
#define VOS_PRECOND_MOM_MG 4
#define VOS_PRECOND_P_WARM 8
#define VOS_PRECOND_U_EXTRAP 16

/* Physical and numerical parameters (non-dimensional units are fine).
 * Symbols follow Sec. 2.2-2.5: nu kinematic viscosity, D diffusion
 * coefficient (D* = D), kc reaction constant (R = kc c), k0 Kozeny-Carman
 * constant, Vm = M_ws / rho_s molar volume of the solid, zeta
 * stoichiometric coefficient, rho_ratio = rho_s / rho (1 gives the
 * divergence-free flow of Eq. contDBSQS), c_in / u_in inlet concentration
 * and velocity, eps_min the fluid fraction kept inside the solid (App. C,
 * 1e-4), lambda the VoS-psi constant (4).  p_rtol / u_rtol / c_rtol:
 * diagonally scaled relative residual ||D^-1 (b - Ax)|| / ||D^-1 b|| (D the
 * diagonal of A, FP64) at which the pressure, momentum and concentration
 * solves stop; max_iter caps the Krylov iterations of one solve. */
typedef struct vos_params {
  int32_t dim, nx, ny, nz; /* dim 2 (nz = 1) or 3 */
  double dx, nu, D, kc, k0, Vm, zeta, rho_ratio, c_in, u_in, eps_min, lambda;
  int32_t method;    /* vos_method */
  int32_t precision; /* vos_precision */
  int32_t precond;   /* vos_precond flags; 0: multigrid + pocket deflation */
  double p_rtol, u_rtol, c_rtol;
  int32_t max_iter;
  int32_t flow_subiters; /* 1: one transient step; M > 1: quasi-static step,
                            at most M sub-iterations (see vos_step)        */
  uint32_t wall_mask;
  double qs_rtol;        /* quasi-static stop test (0: always M iterations)  */
  double qs_dtau;        /* pseudo time step of the sub-iterations (0: dt)   */
  int32_t inertia;       /* 1: keep the inertia term div(u u / eps) of
                            Eq. momentumDBS, explicit (van Leer upwinded on
                            the staggered control volumes); 0 (default):
                            creeping flow, the term is dropped              */
} vos_params;

/* Statistics of the last completed step (FP64 device reductions; S7).
 * V = dx^dim is the cell volume, A = dx^(dim-1) the face area.  The flux
 * terms close the reactant balance of the step (Eq. concentrationDBS
 * integrated over the domain):
 *   reactant^{n+1} - reactant^n = dt (flux_in - flux_out - zeta sum_Rf). */
typedef struct vos_stats {
  int64_t step;
  double t;
  int32_t iters_u[3], iters_p, iters_c;  /* Krylov iterations (inner, summed) */
  int32_t outer_u[3], outer_p, outer_c;  /* refinement passes                */
  double res_u[3], res_p, res_c;         /* final scaled relative residuals  */
  double lambda;       /* psi' fit (psi: the constant; iVoS: NaN)            */
  double porosity;     /* mean eps (the total porosity phi of Sec. 2.5)      */
  double clamp_excess; /* sum(raw - clamped eps) * V of the S1 update        */
  double sum_R, sum_Rf;/* sum R V, sum R_f V                                 */
  double reactant;     /* sum eps c V                                        */
  int32_t status;      /* VOS_OK or VOS_ENOCONV                              */
  double q_in, q_out;  /* sum over inlet / outlet faces of u_f A (Q_i, Sec. 2.5) */
  double flux_in;      /* reactant inflow: inlet faces u_f c_in plus the
                          diffusive flux 2 D eps_P (c_in - c_P) / dx, times A */
  double flux_out;     /* reactant outflow: outlet faces u_f c_P^n, times A  */
  double umax;         /* max over faces of |u_f| / eps_f (interior faces:
                          mean of the two cells; boundary: adjacent cell)    */
  double rmax;         /* max |Vm R|: dt <= deps_max / rmax bounds the change
                          of eps per step (App. D)                          */
  int32_t qs_iters;    /* sub-iterations of the step (1 for a transient step) */
  double qs_du, qs_dp, qs_dc; /* last relative changes of u, p (eps-weighted)
                          and c between sub-iterations (quasi-static steps;
                          NaN otherwise)                                     */
} vos_stats;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc(bytes, ctx) returns a device pointer aligned to >= 256 bytes or
 * NULL (a pointer with less alignment is handed back to free and the
 * allocation fails: VOS_ENOMEM); free(ptr, ctx) releases it.  NULL selects
 * cudaMalloc/cudaFree. */
typedef struct vos_allocator {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} vos_allocator;

typedef struct vos_handle vos_handle;

/* Device pointers of the fields (owned by the handle, valid until destroy).
 * Layouts as above; all FP64. */
typedef struct vos_device_fields {
  double *eps, *c, *p, *u, *v, *w, *R, *Rf;
} vos_device_fields;

/* Create a simulation from the solid fraction eps_s (host, nx*ny*nz FP64
 * values in [0, 1]): eps = max(1 - eps_s, eps_min) (App. C), u = u_in on
 * the inlet faces, all other fields zero.  stream: a cudaStream_t (NULL =
 * legacy default stream).  alloc may be NULL.  The handle owns all device
 * memory; eps_s is copied and not retained.  Errors: VOS_EINVAL (sizes,
 * parameters, values), VOS_ENOMEM, VOS_ECUDA; *out is NULL on error. */
int vos_create(const double* eps_s_host, const vos_params* prm, void* stream,
               const vos_allocator* alloc, vos_handle** out);

/* Advance one time step of length dt (> 0) through S1-S7 (see top).  The
 * linear solves converge on the device: in the default launch mode the step
 * is one CUDA-graph replay whose solver loops are device-driven, and the
 * host waits once, at the end, for the solver statistics; in the eager mode
 * (vos_set_launch_mode(0)) the host reads the residual once per refinement
 * pass and every few Krylov iterations.  Returns VOS_ENOCONV if a solve
 * reached max_iter (the step is still applied).
 * Quasi-static step (flow_subiters = M > 1; App. A and B: flow and
 * transport iterated to a steady state with eps frozen, the rate refreshed
 * after every iteration): S1 advances eps by dt once; S2-S6 then repeat with
 * the latest iterate as the old velocity and concentration, eps^{n+1} in
 * both storage terms and qs_dtau (0: dt) as the time step, so that a fixed
 * point solves the quasi-static equations (Eq. momentumDBSQS without
 * inertia, Eq. contDBSQS, Eq. concentrationDBSQS).  The loop ends after M
 * sub-iterations or when the relative L2 changes of u, of p (weighted by
 * eps: the pressure inside the solid relaxes far more slowly and barely
 * moves the flow) and of c are all <= qs_rtol; with qs_rtol > 0 a loop that
 * reaches M without meeting the test returns VOS_ENOCONV (step applied).
 * Quasi-static steps always launch eagerly (no CUDA graph); vos_stats
 * reports the sub-iterations and the last relative changes, and its solver
 * iteration counts are summed over the sub-iterations. */
int vos_step(vos_handle* h, double dt);

/* Copy the selected fields (mask of VOS_F_*) to caller-owned host buffers
 * (NULL pointers are skipped).  Synchronous on the handle's stream. */
int vos_fields(vos_handle* h, uint32_t mask, double* eps, double* c, double* u,
               double* v, double* w, double* p, double* R, double* Rf);

/* Overwrite the selected fields from host buffers (checkpoint resume).
 * Synchronous. */
int vos_set_fields(vos_handle* h, uint32_t mask, const double* eps, const double* c,
                   const double* u, const double* v, const double* w, const double* p,
                   const double* R, const double* Rf);

/* Device pointers of the fields (no copy). */
int vos_device_fields_get(vos_handle* h, vos_device_fields* out);

/* Statistics of the last step (synchronises the stream). */
int vos_get_stats(vos_handle* h, vos_stats* out);

/* Time step limit min(cfl dx / max_f(|u_f| / eps_f), deps_max / max|Vm R|)
 * (App. D: the step is limited by the largest change of eps; the
 * convective limit uses the interstitial speed).  eps_f is the mean of the
 * two cells of an interior face and the one cell of a boundary face.
 * Synchronous.  Returns +inf in *dt when neither limit applies and 0 when a
 * face speed or a rate is NaN. */
int vos_suggest_dt(vos_handle* h, double cfl, double deps_max, double* dt);

/* Darcy-scale properties of the current fields (Sec. 2.5), FP64 device
 * reductions; synchronous.  V_Omega = nx ny nz dx^dim, face area
 * A = dx^(dim-1).
 *   phi    total porosity, mean eps;
 *   Q_in   inlet flow rate, sum over the inlet faces of u_f A;
 *   A_in   inlet area ny nz A;  U_D = Q_in / A_in (Darcy velocity);
 *   dP     kinematic pressure drop: mean p of the first cell column (i = 0)
 *          minus the outlet face value 0 (the inlet condition is
 *          zero-gradient, so the first cell centres carry the inlet
 *          pressure);  L_D = (nx - 1/2) dx, the distance between them;
 *   K      permeability nu U_D L_D / dP (uniform Darcy flow gives exactly
 *          k = k0 eps^3 / (1 - eps)^2 of Eq. perm);
 *   a      specific surface area (1/V_Omega) int |grad eps| dV (centred
 *          gradient; |grad eps| is the surface-area density of the
 *          micro-continuum);
 *   alpha  (1/a) sum c |grad eps| / sum eps c: the surface-averaged over
 *          the volume-averaged concentration (1/phi for uniform c);
 *   L_ref  sqrt(f K / phi), f = 12 in 2D (channel width of a bundle of
 *          straight channels) and 8 in 3D (throat radius of a capillary
 *          bundle);  U_ref = U_D / phi;
 *   Pe = U_ref L_ref / D, Da = kc / U_ref, Ki = Da Pe.
 * A quantity whose denominator vanishes is NaN.  Errors: VOS_EINVAL,
 * VOS_ECUDA. */
typedef struct vos_upscaled_props {
  double phi, Q_in, A_in, U_D, dP, L_D, K, a, alpha, L_ref, U_ref, Pe, Da, Ki;
} vos_upscaled_props;
int vos_upscaled(vos_handle* h, vos_upscaled_props* out);

/* Batches of independent simulations (e.g. many micromodels of uneven
 * sizes and parameters stepped together; no counterpart in the paper's
 * single-sample runs).  vos_batch_create makes n instances from eps_s[i]
 * and prm[i] (as vos_create); each instance gets its own non-blocking CUDA
 * stream.  In the default launch mode a batch step is one CUDA-graph launch
 * that holds every instance's whole step as a parallel branch (captured
 * again when an instance's momentum-preconditioner choice or captured
 * parameters change); in the eager mode, or while an instance has a learned
 * preconditioner, a pool of nthreads host worker threads (<= 0: 8) advances
 * the instances, so their kernels overlap on the GPU.  stream is the
 * caller's stream: vos_batch_step orders every instance after the work
 * already on it and makes it wait for all instances, so events recorded
 * there bracket a whole batch step.  vos_batch_step(b, dt) advances
 * instance i by dt[i] > 0 and returns VOS_OK, VOS_ENOCONV (some solve hit
 * max_iter) or the first hard error.  vos_batch_handle gives instance i's
 * handle (for vos_fields, vos_get_stats, vos_suggest_dt; do not destroy it
 * and do not use it while a batch step runs).  Per-kernel timing
 * (vos_prof_enable) is not supported while a batch steps.  Errors are
 * reported by vos_last_error(NULL). */
typedef struct vos_batch vos_batch;
int vos_batch_create(int n, const double* const* eps_s, const vos_params* prm, void* stream,
                     int nthreads, const vos_allocator* alloc, vos_batch** out);
int vos_batch_step(vos_batch* b, const double* dt);
int vos_batch_handle(vos_batch* b, int i, vos_handle** h);
void vos_batch_destroy(vos_batch* b);

/* Allocation-free form of vos_suggest_dt (the paper has no counterpart: it
 * exists for callers that cannot let a library allocate device memory --
 * hosts that keep the GPU's memory in their own pool, or loops that must not
 * pay the device-wide synchronisation a cudaMalloc/cudaFree can cause).
 * Computes the same limit as vos_suggest_dt from caller-owned device fields
 * in the layouts above (eps, u, v, w, R; w is required in 3D; v is required
 * when ny > 1 and may be NULL when ny == 1, where every v face is a wall
 * face: the y faces are then not read); only dim, nx, ny, nz, dx and Vm of
 * prm are used (nx >= 2, as vos_create).  It allocates nothing: its scratch
 * is a fixed file-scope device array of about 1 MiB that every GPU loading
 * the library holds until exit, so grids above 16,777,216 cells are
 * rejected with VOS_EINVAL.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) and should come before any
 * stream capture.  All calls share the one array: calls that overlap on the
 * GPU (other streams or threads) race.  Work runs on `stream`, which must
 * belong to the current device (NULL = legacy default stream); the call
 * synchronises it and writes the result to the host double *dt (0 when a
 * speed or rate is NaN, as vos_suggest_dt).  Errors: VOS_EINVAL (NULL or
 * bad arguments, too many cells, a stream of another device), VOS_ECUDA (a
 * failed copy or launch; *dt is then not written); message via
 * vos_last_error(NULL). */
int vos_suggest_dt_noalloc(const vos_params* prm, const double* eps, const double* u,
                           const double* v, const double* w, const double* R, double cfl,
                           double deps_max, void* stream, double* dt);

/* Floating pore clusters of the pressure operator for a fluid fraction
 * field (host only, no GPU needed; a solver aid with no counterpart in the
 * paper).  eps: host, nx*ny*nz FP64, x fastest, the fluid fraction (the
 * solver's eps = max(1 - eps_s, eps_min)).  A face is strong when the
 * arithmetic mean of its two cells' eps (the face porosity of the pressure
 * operator, Sec. 2.2) is >= 0.01; a cluster is a connected set of cells
 * joined by strong faces with at least 2 cells and no cell in the outlet
 * column i = nx - 1 (the Dirichlet row).  label (may be NULL): host int32,
 * nx*ny*nz, receives the cluster id (0..K-1, numbered in order of each
 * cluster's smallest cell index) or -1.  *nclusters = K, *ncells (may be
 * NULL) = cells in clusters.  Errors: VOS_EINVAL (NULL eps/prm/nclusters,
 * invalid prm). */
int vos_floating_clusters(const double* eps, const vos_params* prm, int32_t* label, int32_t* nclusters,
                          int64_t* ncells);

/* Message of the last error on h (or of the last failed vos_create when h
 * is NULL).  The string is owned by the library. */
const char* vos_last_error(const vos_handle* h);

/* Free all device memory of h.  NULL is accepted. */
void vos_destroy(vos_handle* h);

/* Bytes of device memory held by h. */
size_t vos_device_bytes(const vos_handle* h);

/* 3x3x3 zero-padded convolution on the tensor cores (BF16 operands, FP32
 * accumulation): the building block of the learned pressure preconditioner
 * (no counterpart in the paper).  All pointers are device memory; the call
 * runs on `stream` and synchronises it.
 *   x: BF16 [nx*ny*nz][cin], voxel i + nx*(j + ny*k), channels last;
 *   w: BF16 [cout][27][cin], tap = (dz+1)*9 + (dy+1)*3 + (dx+1);
 *   bias: FP32 [cout] or NULL; relu: clamp the result at 0;
 *   y_f32 (FP32) and/or y_bf16 (BF16, round to nearest even): [V][cout].
 *   y[v][o] = bias[o] + sum over taps t and channels c of
 *             w[o][t][c] x[v + t][c], x = 0 outside the box.
 * cin must be a multiple of 8, cout a multiple of 16 in [16, 96].  The call
 * allocates (and frees) a device buffer of 27 * cout * 16 * ceil(cin / 16)
 * BF16 values for the weights in the kernel's shared-memory layout.
 * Errors: VOS_EINVAL, VOS_ENOMEM, VOS_ECUDA, VOS_ETIMEOUT (a tensor-core
 * wait gave up after 2 s; the output is invalid); message via
 * vos_last_error(NULL). */
int vos_conv3d_bf16(const uint16_t* x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const uint16_t* w,
                    const float* bias, int32_t cout, int32_t relu, float* y_f32, uint16_t* y_bf16, void* stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner for the pressure correction (a solver aid with no
 * counterpart in the paper).  A 3-level U-Net on the pressure grid: inputs
 * r / rms(r) and eps, 3x3x3 convolutions 2->16->16 | pool | 16->32->32 |
 * pool | 32->64->64 | up, concat | 96->32->32 | up, concat | 48->16->16 |
 * 1x1x1 head 16->1, ReLU after every 3x3x3 conv, 2x2x2 average pooling,
 * nearest-neighbour upsampling, zero padding.  Convolutions run on the
 * tensor cores (BF16 operands and activations, FP32 accumulation); training
 * uses the library's own backward kernels and Adam.  Attached to a handle,
 * the pressure solve becomes flexible CG with z = UNet(r / rms(r)) rms(r)
 * and falls back to MG-PCG when the residual stops falling, so it always
 * reaches p_rtol.  Boxes whose sides are not multiples of 4 are padded with
 * zeros inside the network.
 *
 * Parameters travel as one FP32 host vector: for each conv in the order
 * above, W[cout][3][3][3][cin] (taps z, y, x; channels of a concat in the
 * order coarse, skip) then b[cout]; then the head's w[16] and b.
 * vos_unet_num_params() gives its length.  Device vectors are FP32 (r, z,
 * dz) or FP64 (eps), one value per cell, cell i + nx*(j + ny*k).
 * -------------------------------------------------------------------------*/
typedef struct vos_unet vos_unet;

/* Network for an nx x ny x nz grid (each >= 4), weights zero until
 * vos_unet_set_params; train != 0 also allocates gradient and optimiser
 * buffers.  Work is enqueued on `stream`.  Errors: VOS_EINVAL, VOS_ENOMEM. */
int vos_unet_create(int32_t nx, int32_t ny, int32_t nz, int32_t train, void* stream, vos_unet** out);
int64_t vos_unet_num_params(void);
/* Copy parameters in (resets the optimiser state) or out; gradients of the
 * last vos_unet_backward out.  n must equal vos_unet_num_params(). */
int vos_unet_set_params(vos_unet* net, const float* host, int64_t n);
int vos_unet_get_params(vos_unet* net, float* host, int64_t n);
int vos_unet_get_grads(vos_unet* net, float* host, int64_t n);
/* z = UNet(r / rms(r), eps) (no rescaling), device pointers; synchronises.
 * Errors: VOS_EINVAL, VOS_ECUDA, VOS_ETIMEOUT. */
int vos_unet_forward(vos_unet* net, const float* r, const double* eps, float* z);
/* Gradients of sum(dz * z) for the last forward (training networks only). */
int vos_unet_backward(vos_unet* net, const float* dz);
/* One Adam step (learning rate lr > 0) on L = |A z - r_hat|^2 / |r_hat|^2,
 * r_hat = r / rms(r), z = UNet(r_hat, eps), A the pressure operator and eps
 * the fluid fraction of h's last step (same grid).  *loss = L before the
 * step.  vos_unet_eval_loss computes L only. */
int vos_unet_train_step(vos_unet* net, vos_handle* h, const float* r, float lr, float* loss);
int vos_unet_eval_loss(vos_unet* net, vos_handle* h, const float* r, float* loss);
void vos_unet_destroy(vos_unet* net);

/* Use net (NULL: none) as the pressure preconditioner of h.  The network is
 * not owned by h and must outlive its use; its grid must be h's.  While a
 * network is attached vos_step launches kernels one by one (no CUDA graph). */
int vos_set_unet_preconditioner(vos_handle* h, vos_unet* net);
/* Of the last step's pressure solve: flexible-CG iterations with the
 * network, and 1 if it stalled and MG-PCG finished the solve. */
int vos_unet_solve_stats(const vos_handle* h, int32_t* net_iters, int32_t* fallback);
/* Training data: residuals of MG-PCG on the last step's pressure system
 * A e = b from e = 0 after iters[i] iterations (0 gives b), as FP32 device
 * vectors out + i * nx*ny*nz.  Needs one completed step; uses the pressure
 * correction field as scratch (it is rebuilt by every step). */
int vos_pressure_snapshots(vos_handle* h, int32_t count, const int32_t* iters, float* out);

/* Self-check of the FP64 quotient the physics kernels use in place of IEEE
 * division (no counterpart in the paper; FP64 instructions are the scarce
 * resource of those kernels): Newton-Raphson refinement of the hardware
 * reciprocal estimate, one step on the reciprocal and one on the quotient,
 * IEEE division for |d| outside [2^-1000, 2^1000] or not finite (a zero
 * numerator gives +0 whatever its sign).  For the
 * n pairs (a[i], d[i]) writes q_fast[i] = that quotient and q_ieee[i] = the
 * IEEE-rounded a[i] / d[i].  All four arrays are device memory of n doubles
 * owned by the caller; the call runs on the legacy default stream and
 * synchronises it.  Errors: VOS_EINVAL (n < 0, NULL array with n > 0),
 * VOS_ECUDA; message via vos_last_error(NULL). */
int vos_fp64_div_check(const double* a, const double* d, int64_t n, double* q_fast, double* q_ieee);

/* Stencil tile of one multigrid level of one linear system of h: sys 0-2
 * the momentum components u, v, w, 3 the pressure correction, 4 the
 * concentration; level 0 is the fine grid.  *tx, *ty: threads of a block
 * along x and y (tx * ty = 256); *zc: planes each block marches along z
 * (along y for 2D grids); *tuned: 1 when the autotuner measured this shape
 * at create (levels of >= 65,536 cells; the fastest Jacobi sweep among tile
 * widths 32/64/128 and z chunks of one or more planes for about 1024-8192
 * blocks), 0 for the default (32 x 8, or 256 x 1 on 2D grids, about 4096
 * blocks of one or more planes).  Errors:
 * VOS_EINVAL (NULL argument, sys or level out of range). */
int vos_tile_config(const vos_handle* h, int32_t sys, int32_t level, int32_t* tx, int32_t* ty, int32_t* zc,
                    int32_t* tuned);

/* Diagnostics (process-wide, not tied to a handle; not thread-safe while
 * timing is on).
 * vos_kernel_launches: number of kernel executions of the step so far
 *   (counted on the device, so kernels replayed by graphs are included;
 *   synchronises the device).
 * vos_prof_enable: time every launch of the kernels whose name contains
 *   one of the comma-separated substrings of filter ("*" = all, NULL or ""
 *   = off) with CUDA events on the launching stream.
 * vos_prof_report: write one line per timed kernel name,
 *   "name<TAB>launches<TAB>total_ms<TAB>algorithmic_bytes\n", into buf
 *   (synchronises on the recorded events).  Returns VOS_OK, or the buffer
 *   size needed if len is too small.
 * vos_prof_reset: drop the accumulated timings. */
uint64_t vos_kernel_launches(void);
/* vos_set_launch_mode(1) (default): vos_step replays the whole step as one
 *   CUDA graph whose refinement and Krylov loops are conditional WHILE nodes
 *   driven on the device (captured at the first step of each momentum-
 *   preconditioner choice; replayed on an internal stream ordered after the
 *   handle's stream by events).  vos_set_launch_mode(0): the same kernels
 *   launched one by one with host polls of the device scalars.  While
 *   per-kernel timing is on the eager sequence is used. */
int vos_set_launch_mode(int graphs);
/* vos_set_coarse_cycle(1): in every multigrid hierarchy set up afterwards
 *   (vos_create, vos_batch_create), the levels from the first one with at
 *   most 32,768 cells down to the coarsest run as ONE launch per V-cycle of
 *   one thread-block cluster of 8 CTAs that keeps those levels in
 *   distributed shared memory (when the device can run that cluster);
 *   vos_set_coarse_cycle(0) (default): one launch per sweep, residual,
 *   restriction and prolongation on every level, replayed from the step's
 *   CUDA graph, which measured faster on the 256^3 rock.  Both give
 *   bit-identical results (the same arithmetic per cell, in the same
 *   order). */
int vos_set_coarse_cycle(int on);
/* vos_set_vector_sweeps(1) (default): the matrix-free FP32 sweeps of the
 *   pressure fine level (mixed precision) give each thread four consecutive
 *   cells along x with 16-byte loads and stores when nx is a multiple of 4,
 *   and the multigrid cycles fuse the residual with the restriction and the
 *   prolongation with the first post-smoothing sweep on every level but the
 *   coarsest; vos_set_vector_sweeps(0): one cell per thread and separate
 *   passes.  Identical results (each cell's arithmetic and each sum's order
 *   are the same); takes effect at the next launch. */
int vos_set_vector_sweeps(int on);
/* vos_set_fused_pcg(mask): fused forms of the mixed path's solves; default
 *   7 (all three), 0 for the separate kernels and the FP64 residual.
 *   Bit 0 (VOS_FUSED_DIAG_PCG): diagonally preconditioned CG on a
 *   constant-link operator (the momentum systems when they take the
 *   diagonal preconditioner) in two kernels per iteration -- the direction
 *   update fused with the matrix-vector product and p.q, the x/r update
 *   fused with the preconditioner and r.r, r.z, z.z (20 + 32 bytes per
 *   unknown against 64).  Every value is computed with the operations, and
 *   every dot summed in the order, of the four separate kernels: identical
 *   results.
 *   Bit 1 (VOS_FUSED_MG_PCG): multigrid PCG on the matrix-free pressure level
 *   (rows of a multiple of 4 cells) with the x/r update fused into the
 *   V-cycle's first fine sweep and r.z into its last (the floating-cluster
 *   deflation adds its share of r.z): two fewer passes over the vectors per
 *   iteration.  The cell values are the separate kernels'; two dot products
 *   are summed in another order, so the iterates agree to rounding.
 *   Bit 2 (VOS_FUSED_DF_RESIDUAL): the refinement residual b - A x of a
 *   symmetric system solved to 1e-9 or looser is evaluated after the first
 *   pass in double-FP32 arithmetic on the FP32 pipes (FP32 hi + lo pairs of
 *   b, x and the operator, cut from the FP64 values by integer operations,
 *   relative error below 2^-46 per value) instead of FP64; the first pass,
 *   tighter solves and values of magnitude 2^127 or more keep the FP64
 *   residual.  The solves still reach their tolerance; the fields agree with
 *   the FP64-residual path to that tolerance.
 *   Returns VOS_EINVAL for a mask outside 0..7.  Takes effect at the next
 *   launch; a step already captured as a CUDA graph keeps the form it was
 *   captured with. */
#define VOS_FUSED_DIAG_PCG 1
#define VOS_FUSED_MG_PCG 2
#define VOS_FUSED_DF_RESIDUAL 4
int vos_set_fused_pcg(int mask);
int vos_prof_enable(const char* filter);
int vos_prof_report(char* buf, size_t len);
void vos_prof_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* VOS_H_ */
