"""FP64 CPU oracle of the micro-continuum (Volume-of-Solid) time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA path; both read the same seeded inputs from
``paper_2204_07019_gb300.inputs``.

Follows Maes, Soulaine & Menke, "Improved Volume-of-Solid formulations for
micro-continuum simulation of mineral dissolution at the pore-scale":

* Sec. 2.2: volume-averaged fields, Darcy-Brinkman-Stokes momentum
  (Eq. momentumDBS), Kozeny-Carman permeability (Eq. perm), averaged
  advection-diffusion-reaction (Eq. concentrationDBS), solid mass balance
  (Eq. mbs), continuity with a dissolution source (Eq. contDBS).
* Sec. 2.3: iVoS reaction rate from the divergence of the reactive flux
  (Eq. RfiVoS), split into the mass-transfer part eps div(Phi) and the
  conservative part -div(eps Phi).
* Sec. 2.4: VoS-psi (Eq. RfVoSpsi) with psi = lambda eps (1 - eps), lambda = 4,
  and VoS-psi' with lambda refitted from global integrals.
* App. B: order of the sub-steps (eps, permeability, velocity, pressure,
  concentration, reaction rate), van Leer interpolation of convective and
  reactive fluxes.
* App. C: eps_f = 1e-4 inside the solid.

The discrete scheme (a transient step on a MAC-staggered Cartesian grid; the
paper's OpenFOAM discretisation is prior art) is fixed by the readings listed
in the project's design notes; every reading is restated in the docstring
of the function that applies it.

Arrays are numpy float64 with shape (nz, ny, nx) (x fastest; nz = 1 in 2D).
Face arrays for axis a (0 = x, 1 = y, 2 = z) have one more entry along that
axis.  Each linear system is assembled face by face as a scipy.sparse
matrix and solved by a library routine (SuperLU, or CG/BiCGStab for large
grids); there is no blocking, fusion or reordering beyond that.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

VOS_PSI, VOS_PSI_PRIME, VOS_IVOS = 0, 1, 2
WALL_YM, WALL_YP, WALL_ZM, WALL_ZP = 1, 2, 4, 8

# numpy axis of spatial axis a (x is the last, fastest axis)
def _nax(a):
    return 2 - a


def _shape(prm):
    return (int(prm["nz"]), int(prm["ny"]), int(prm["nx"]))


def _axes(prm):
    return (0, 1) if int(prm["dim"]) == 2 else (0, 1, 2)


def _sl(a, lo, hi):
    """Slice [lo:hi] along spatial axis a of a (nz, ny, nx)-like array."""
    s = [slice(None)] * 3
    s[_nax(a)] = slice(lo, hi)
    return tuple(s)


# --------------------------------------------------------------------------
# Closure relations
# --------------------------------------------------------------------------

def kozeny_carman_kinv(eps, k0):
    """Inverse permeability k^-1 = (1 - eps)^2 / (k0 eps^3)  (Eq. perm, Sec. 2.2).

    Stored as the inverse so that it is finite (zero) in pure fluid.
    """
    return (1.0 - eps) ** 2 / (k0 * eps ** 3)


def van_leer_psi(r):
    """van Leer limiter psi(r) = (r + |r|) / (1 + |r|)  (ref. 1974-vanLeer, App. B)."""
    return (r + np.abs(r)) / (1.0 + np.abs(r))


def van_leer_weight(cUU, cU, cD, has_uu):
    """Weight w in c_f = c_U + w (c_D - c_U), w = psi(r)/2, r = (c_U - c_UU)/(c_D - c_U).

    Reading: a far-upwind cell outside the domain takes the zero-gradient
    ghost (r = 0, w = 0); |c_D - c_U| <= 1e-300 gives w = 0.
    """
    den = cD - cU
    ok = has_uu & (np.abs(den) > 1e-300)
    r = np.where(ok, (cU - cUU) / np.where(ok, den, 1.0), 0.0)
    return np.where(ok, 0.5 * van_leer_psi(r), 0.0)


# --------------------------------------------------------------------------
# Geometry helpers on the cell grid
# --------------------------------------------------------------------------

def central_gradient(eps, dx, axes):
    """Centred gradient of eps with zero-gradient ghosts at every boundary.

    Used by VoS-psi (Sec. 2.4: "centered difference scheme for the gradient")
    and for the tangential part of the iVoS face normal.  Returns a list of
    3 arrays (zero for axes not in ``axes``).
    """
    g = [np.zeros_like(eps) for _ in range(3)]
    for a in axes:
        n = eps.shape[_nax(a)]
        lo = np.concatenate([np.take(eps, [0], axis=_nax(a)),
                             np.take(eps, np.arange(0, n - 1), axis=_nax(a))], axis=_nax(a))
        hi = np.concatenate([np.take(eps, np.arange(1, n), axis=_nax(a)),
                             np.take(eps, [n - 1], axis=_nax(a))], axis=_nax(a))
        g[a] = (hi - lo) / (2.0 * dx)
    return g


def face_average(cell, a):
    """Arithmetic mean of the two cells adjacent to each interior face along a."""
    n = cell.shape[_nax(a)]
    return 0.5 * (cell[_sl(a, 0, n - 1)] + cell[_sl(a, 1, n)])


# --------------------------------------------------------------------------
# Linear solves (library primitives)
# --------------------------------------------------------------------------

def _solve(A, b, symmetric, solver, rtol):
    A = A.tocsr()
    if solver == "direct" or A.shape[0] <= 4096:
        return spla.spsolve(A.tocsc(), b)
    d = A.diagonal()
    M = sp.diags(1.0 / d)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b)
    if symmetric:
        x, info = spla.cg(A, b, rtol=rtol, atol=0.0, M=M, maxiter=200000)
    else:
        x, info = spla.bicgstab(A, b, rtol=rtol, atol=0.0, M=M, maxiter=200000)
    if info != 0:
        raise RuntimeError(f"oracle iterative solve failed (info={info})")
    return x


# --------------------------------------------------------------------------
# State
# --------------------------------------------------------------------------

def init_state(eps_s, prm):
    """Initial fields (App. C: eps_f = max(1 - eps_s, 1e-4); reading: u = p = c = 0).

    The inlet faces carry u_in from t = 0 (acid injected at t = 0, Sec. 3.1).
    """
    shp = _shape(prm)
    eps_s = np.asarray(eps_s, dtype=np.float64).reshape(shp)
    eps = np.maximum(1.0 - eps_s, prm["eps_min"])
    u = []
    for a in range(3):
        fs = list(shp)
        fs[_nax(a)] += 1
        u.append(np.zeros(fs))
    u[0][_sl(0, 0, 1)] = prm["u_in"]
    if int(prm["dim"]) == 2:
        u[2] = np.zeros((0,))
    z = np.zeros(shp)
    return dict(eps=eps, c=z.copy(), p=z.copy(), u=u, R=z.copy(), Rf=z.copy(),
                t=0.0, step=0)


# --------------------------------------------------------------------------
# S1: solid update
# --------------------------------------------------------------------------

def solid_update(eps, R, dt, prm):
    """eps^{n+1} = clamp(eps^n + dt V_m R^n, eps_min, 1)  (Eq. mbs, Sec. 2.2).

    Reading: explicit Euler in time with the rate of the previous step; the
    clamp keeps eps >= eps_min (App. C).  Returns (eps_new, clamp_excess)
    where clamp_excess = sum(raw - clamped) * V.
    """
    raw = eps + dt * prm["Vm"] * R
    new = np.clip(raw, prm["eps_min"], 1.0)
    V = prm["dx"] ** int(prm["dim"])
    return new, float(np.sum(raw - new) * V)


# --------------------------------------------------------------------------
# S2: momentum predictor
# --------------------------------------------------------------------------

def _face_unknown_range(a, shp):
    """Index range along a of the unknown faces of component a.

    x: faces 1..nx (face 0 = inlet, fixed u_in; face nx = outlet, unknown).
    y, z: faces 1..n-1 (boundary faces carry zero normal velocity).
    """
    n = shp[_nax(a)]
    return (1, n + 1) if a == 0 else (1, n)


def face_porosity(eps, a, prm):
    """eps_f on every face of axis a: mean of the two cells on interior faces,
    the adjacent cell on boundary faces."""
    shp = _shape(prm)
    n = shp[_nax(a)]
    fs = list(shp)
    fs[_nax(a)] += 1
    ef = np.zeros(fs)
    ef[_sl(a, 1, n)] = face_average(eps, a)
    ef[_sl(a, 0, 1)] = eps[_sl(a, 0, 1)]
    ef[_sl(a, n, n + 1)] = eps[_sl(a, n - 1, n)]
    return ef


def _vl_face(phi, b, U):
    """van Leer value of ``phi`` (an array along axis b with n entries) at the
    n - 1 interior points between consecutive entries, upwinded along the
    advecting velocity U (U >= 0: the lower entry is upwind); a far-upwind
    entry outside the array gives the upwind value (R14)."""
    cUU, cU, cD, h = _upwind_triplets(phi, b, U >= 0.0)
    return cU + van_leer_weight(cUU, cU, cD, h) * (cD - cU)


def inertia(u, eps, prm):
    """Explicit inertia term N_a = div(u u_a / eps) of Eq. momentumDBS
    (multiplied by eps, the form of ``momentum_system``) on the faces of each
    velocity component a, from the face velocities u (App. B: convection by
    the second-order van Leer scheme).

    Finite volumes on the staggered control volume (CV) of each a-face: the
    transported quantity is phi_a = u_a / eps_f (eps_f from
    ``face_porosity``), carried through the CV faces by the advecting
    velocity U_b and taken there by van Leer upwinding along b:
    * b = a: CV faces at cell centres, U = mean of the cell's two a-faces,
      phi interpolated between those two faces;
    * b != a: CV faces on the cell edges, U = mean of the two b-faces that
      meet at the edge (the a-face's two cells; the outlet a-face has one),
      phi interpolated between the a-faces on either side of the edge.
    N_a = sum over b of (F_b(plus CV face) - F_b(minus CV face)) / dx.
    Readings at the domain boundary: walls and free-slip sides carry no
    normal velocity, so no flux; the inlet plane carries no tangential
    velocity, so its edges carry no tangential momentum; at the outlet (zero
    gradient) the outermost edges take the upwind (interior) value, and the
    outlet face's own CV, which reaches half a cell past the outlet, loses
    u_n phi_n there.  Returned on every face of axis a (the fixed faces'
    values are not used)."""
    shp = _shape(prm)
    axes = _axes(prm)
    N = []
    for a in range(3):
        if a not in axes:
            N.append(np.zeros((0,)))
            continue
        ua = u[a]
        fs = ua.shape
        phi = ua / face_porosity(eps, a, prm)
        Na = np.zeros(fs)
        na = shp[_nax(a)]  # cells along a (a-faces 0..na)
        for b in axes:
            if b == a:
                U = 0.5 * (ua[_sl(a, 0, na)] + ua[_sl(a, 1, na + 1)])  # cell centres
                F = U * _vl_face(phi, a, U)  # between a-faces m and m+1
                Na[_sl(a, 0, na)] += F       # plus CV face of a-face m
                Na[_sl(a, 1, na + 1)] -= F   # minus CV face of a-face m+1
                if a == 0:                   # outlet face: its CV reaches past the outlet
                    Na[_sl(0, na, na + 1)] += ua[_sl(0, na, na + 1)] * phi[_sl(0, na, na + 1)]
                continue
            mb = shp[_nax(b)]  # a-faces along b
            ub = u[b]
            # u_b at the edges: b-faces 0..mb along b, averaged over the
            # a-face's cells along a
            es = list(fs)
            es[_nax(b)] += 1
            Ue = np.zeros(es)
            Ue[_sl(a, 1, na)] = 0.5 * (ub[_sl(a, 0, na - 1)] + ub[_sl(a, 1, na)])
            if a == 0:
                Ue[_sl(0, na, na + 1)] = ub[_sl(0, na - 1, na)]
            Ui = Ue[_sl(b, 1, mb)]                # interior edges
            F = Ui * _vl_face(phi, b, Ui)         # between a-faces j and j+1 along b
            Na[_sl(b, 0, mb - 1)] += F
            Na[_sl(b, 1, mb)] -= F
            if b == 0:  # outlet-plane edges: zero gradient (upwind interior value)
                Na[_sl(0, mb - 1, mb)] += Ue[_sl(0, mb, mb + 1)] * phi[_sl(0, mb - 1, mb)]
        N.append(Na / prm["dx"])
    return N


def momentum_system(a, eps, p, u_old, dt, prm, u_all=None):
    """Linear system for the face velocity component a (Eq. momentumDBS, Sec. 2.2).

    Multiplying Eq. momentumDBS by eps and, by default (inertia = 0),
    dropping the inertia term (reading: creeping flow, Re = Pe/Sc <= 0.1)
    gives, per face f,

      (1/dt + nu eps_f k^-1_f) u_f - nu lap(u)_f = u^n_f/dt - eps_f (grad p^n)_f

    eps_f, k^-1_f: arithmetic means of the adjacent cells (the outlet face
    takes its one cell).  lap: 5/7-point with ghosts -- no-slip walls and the
    inlet plane for tangential components: ghost = -u (zero at the boundary);
    outlet and free-slip sides: ghost = +u; fixed boundary faces (inlet u_in,
    zero normal velocity on walls) enter as known values.  Outlet pressure
    p = 0 on the boundary face (ghost p = -p_P).
    With prm["inertia"] set, the explicit inertia term of the old velocity
    field u_all (``inertia``) moves to the right-hand side:
    ... = u^n_f/dt - eps_f (grad p^n)_f - div(u^n u^n_a / eps)_f
    (Eq. momentumDBS multiplied by eps; reading: explicit in time).
    Returns (A, b, idx) with idx the flat face indices of the unknowns.
    """
    shp = _shape(prm)
    axes = _axes(prm)
    dx, nu = prm["dx"], prm["nu"]
    fs = list(shp)
    fs[_nax(a)] += 1
    fs = tuple(fs)
    lo, hi = _face_unknown_range(a, shp)
    unk = np.zeros(fs, dtype=bool)
    unk[_sl(a, lo, hi)] = True
    nun = int(unk.sum())
    num = -np.ones(fs, dtype=np.int64)
    num[unk] = np.arange(nun)
    # known boundary face values (inlet u_in for x, zero otherwise)
    known = np.zeros(fs)
    if a == 0:
        known[_sl(0, 0, 1)] = prm["u_in"]

    kinv = kozeny_carman_kinv(eps, prm["k0"])
    n_a = shp[_nax(a)]
    eps_f = np.zeros(fs)
    kin_f = np.zeros(fs)
    gp = np.zeros(fs)
    eps_f[_sl(a, 1, n_a)] = face_average(eps, a)
    kin_f[_sl(a, 1, n_a)] = face_average(kinv, a)
    gp[_sl(a, 1, n_a)] = (p[_sl(a, 1, n_a)] - p[_sl(a, 0, n_a - 1)]) / dx
    if a == 0:  # outlet face: one-sided values, Dirichlet p = 0
        eps_f[_sl(0, n_a, n_a + 1)] = eps[_sl(0, n_a - 1, n_a)]
        kin_f[_sl(0, n_a, n_a + 1)] = kinv[_sl(0, n_a - 1, n_a)]
        gp[_sl(0, n_a, n_a + 1)] = -2.0 * p[_sl(0, n_a - 1, n_a)] / dx

    diag = 1.0 / dt + nu * eps_f * kin_f
    rhs = u_old / dt - eps_f * gp
    if u_all is not None and int(prm.get("inertia", 0)):
        rhs = rhs - inertia(u_all, eps, prm)[a]
    rows, cols, vals = [], [], []
    coef = nu / dx ** 2
    wall = int(prm["wall_mask"])
    for b in axes:
        nb_len = fs[_nax(b)]
        for sgn in (-1, 1):
            # neighbour index along b for every face
            idx_b = np.arange(nb_len).reshape([-1 if k == _nax(b) else 1 for k in range(3)])
            nidx = idx_b + sgn
            inside = (nidx >= 0) & (nidx < nb_len)
            inside = np.broadcast_to(inside, fs)
            # ghost factor s for neighbours outside the face array
            if b == 0:
                s_ghost = -1.0 if sgn < 0 else 1.0   # inlet plane: 0; outlet: zero-gradient
            else:
                bit = (WALL_YM if sgn < 0 else WALL_YP) if b == 1 else (WALL_ZM if sgn < 0 else WALL_ZP)
                s_ghost = -1.0 if (wall & bit) else 1.0
            # contributions of unknown faces
            sel = unk & ~inside
            diag = diag + np.where(sel, coef * (1.0 - s_ghost), 0.0)
            # inside neighbours
            shifted_num = np.full(fs, -1, dtype=np.int64)
            shifted_known = np.zeros(fs)
            src = _sl(b, max(sgn, 0), nb_len + min(sgn, 0))
            dst = _sl(b, max(-sgn, 0), nb_len + min(-sgn, 0))
            shifted_num[dst] = num[src]
            shifted_known[dst] = known[src]
            m_unk = unk & inside & (shifted_num >= 0)
            m_fix = unk & inside & (shifted_num < 0)
            diag = diag + np.where(m_unk | m_fix, coef, 0.0)
            rhs = rhs + np.where(m_fix, coef * shifted_known, 0.0)
            rows.append(num[m_unk]); cols.append(shifted_num[m_unk])
            vals.append(np.full(int(m_unk.sum()), -coef))
    rows.append(num[unk]); cols.append(num[unk]); vals.append(diag[unk])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nun, nun)).tocsr()
    return A, rhs[unk], unk


# --------------------------------------------------------------------------
# S3: pressure Poisson and projection
# --------------------------------------------------------------------------

def divergence(u, prm):
    """Cell divergence of a face field: sum over faces of the outward flux / dx."""
    shp = _shape(prm)
    div = np.zeros(shp)
    for a in _axes(prm):
        n = shp[_nax(a)]
        div += (u[a][_sl(a, 1, n + 1)] - u[a][_sl(a, 0, n)]) / prm["dx"]
    return div


def pressure_system(eps, ustar, R, dt, prm):
    """Pressure-correction system  -div(eps_f grad phi) = -(div u* - s)/dt.

    The correction u^{n+1} = u* - dt eps_f grad phi makes div u^{n+1} = s with
    s = R V_m (1 - rho_s/rho)  (Eq. contDBS; zero for rho_s = rho, the
    quasi-static continuity of Eq. contDBSQS).  Boundary conditions: zero
    normal gradient at the inlet and walls (velocity prescribed), phi = 0 on
    the outlet faces (ghost -phi_P).  Face coefficient eps_f = mean of the two
    cells.
    """
    shp = _shape(prm)
    N = int(np.prod(shp))
    dx = prm["dx"]
    num = np.arange(N).reshape(shp)
    rows, cols, vals = [], [], []
    diag = np.zeros(shp)
    for a in _axes(prm):
        n = shp[_nax(a)]
        ef = face_average(eps, a) / dx ** 2
        P = num[_sl(a, 0, n - 1)].ravel(); Q = num[_sl(a, 1, n)].ravel(); cf = ef.ravel()
        rows += [P, Q, P, Q]; cols += [P, Q, Q, P]; vals += [cf, cf, -cf, -cf]
    # outlet Dirichlet faces
    nx = shp[2]
    diag[_sl(0, nx - 1, nx)] += 2.0 * eps[_sl(0, nx - 1, nx)] / dx ** 2
    rows.append(num.ravel()); cols.append(num.ravel()); vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    s = R * prm["Vm"] * (1.0 - prm["rho_ratio"])
    b = -(divergence(ustar, prm) - s) / dt
    return A, b.ravel()


def project(ustar, phi, eps, dt, prm):
    """u^{n+1} = u* - dt eps_f grad phi on interior and outlet faces."""
    shp = _shape(prm)
    dx = prm["dx"]
    u = [x.copy() for x in ustar]
    for a in _axes(prm):
        n = shp[_nax(a)]
        ef = face_average(eps, a)
        u[a][_sl(a, 1, n)] -= dt * ef * (phi[_sl(a, 1, n)] - phi[_sl(a, 0, n - 1)]) / dx
    nx = shp[2]
    u[0][_sl(0, nx, nx + 1)] -= dt * eps[_sl(0, nx - 1, nx)] * (-2.0 * phi[_sl(0, nx - 1, nx)]) / dx
    return u


# --------------------------------------------------------------------------
# S4: explicit van Leer advection
# --------------------------------------------------------------------------

def _upwind_triplets(c, a, positive):
    """(c_UU, c_U, c_D, has_UU) on the interior faces along a.

    ``positive``: boolean array on those faces, True where the upwind cell is
    the minus-side cell.
    """
    n = c.shape[_nax(a)]
    m1 = c[_sl(a, 0, n - 1)]          # minus-side cell of face m (cells m-1)
    p0 = c[_sl(a, 1, n)]              # plus-side cell (m)
    # far cells: m-2 for positive, m+1 for negative
    mm2 = np.zeros_like(m1); has_m = np.zeros(m1.shape, dtype=bool)
    pp1 = np.zeros_like(m1); has_p = np.zeros(m1.shape, dtype=bool)
    if n >= 3:
        mm2[_sl(a, 1, n - 1)] = c[_sl(a, 0, n - 2)]; has_m[_sl(a, 1, n - 1)] = True
        pp1[_sl(a, 0, n - 2)] = c[_sl(a, 2, n)]; has_p[_sl(a, 0, n - 2)] = True
    cU = np.where(positive, m1, p0)
    cD = np.where(positive, p0, m1)
    cUU = np.where(positive, mm2, pp1)
    hUU = np.where(positive, has_m, has_p)
    return cUU, cU, cD, hUU


def advection_divergence(c, u, prm):
    """Cell divergence of the explicit van Leer convective flux c_f u_f (App. B).

    Interior faces: c_f = van Leer interpolation upwind of sign(u_f)
    (u_f >= 0: minus cell upwind).  Inlet faces: inflow u_in c_in.  Outlet
    faces: c of the last cell.  Wall faces: zero flux.
    """
    shp = _shape(prm)
    dx = prm["dx"]
    div = np.zeros(shp)
    for a in _axes(prm):
        n = shp[_nax(a)]
        F = np.zeros_like(u[a])
        uf = u[a][_sl(a, 1, n)]
        cUU, cU, cD, h = _upwind_triplets(c, a, uf >= 0.0)
        cf = cU + van_leer_weight(cUU, cU, cD, h) * (cD - cU)
        F[_sl(a, 1, n)] = uf * cf
        if a == 0:
            F[_sl(0, 0, 1)] = u[0][_sl(0, 0, 1)] * prm["c_in"]
            F[_sl(0, n, n + 1)] = u[0][_sl(0, n, n + 1)] * c[_sl(0, n - 1, n)]
        div += (F[_sl(a, 1, n + 1)] - F[_sl(a, 0, n)]) / dx
    return div


# --------------------------------------------------------------------------
# S6: reactive surface
# --------------------------------------------------------------------------

def vos_lambda(eps, prm):
    """VoS-psi' parameter lambda(eps) = int |grad eps| / int |grad eps| eps (1 - eps)
    (Sec. 2.4), from the centred gradient.  Reading: a vanishing denominator
    (< 1e-300 x numerator, or a zero numerator) gives lambda = 4."""
    g = central_gradient(eps, prm["dx"], _axes(prm))
    mag = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    num = float(np.sum(mag))
    den = float(np.sum(mag * eps * (1.0 - eps)))
    if num == 0.0 or den < 1e-300 * num:
        return 4.0
    return num / den


def vos_coefficient(eps, prm, lam):
    """k_c psi |grad eps| with psi = lam eps (1 - eps), centred gradient
    (Eq. RfVoSpsi, Sec. 2.4); R = coefficient * c."""
    g = central_gradient(eps, prm["dx"], _axes(prm))
    mag = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    return prm["kc"] * lam * eps * (1.0 - eps) * mag


def ivos_faces(eps, c_old, prm):
    """Per-face data of the iVoS reactive flux (Sec. 2.3, App. B).

    For each interior face along a: g_f has normal part (eps_plus - eps_minus)/dx
    and tangential parts equal to the mean of the two cells' centred
    gradients; n_f = -g_f / (|g_f| + delta) with delta = 1e-8/dx (reading);
    Phi_R . e_a = k_c c_f n_a.  Upwind = the cell the flux leaves
    (n_a > 0: minus cell).  Reading: c_f = c_U^{n+1} + corr with the van
    Leer correction corr = w(c^n) (c_D^n - c_U^n) taken from the previous
    concentration (implicit upwind + explicit deferred correction), so the
    implicit reaction matrix is an upwind M-matrix; eps_f is the van Leer
    interpolation of eps.
    Returns per axis a dict with n_a (normal component), positive (bool),
    corr (deferred van Leer correction) and eps_vl.
    """
    axes = _axes(prm)
    dx = prm["dx"]
    g = central_gradient(eps, dx, axes)
    delta = 1e-8 / dx
    out = {}
    shp = _shape(prm)
    for a in axes:
        n = shp[_nax(a)]
        gn = (eps[_sl(a, 1, n)] - eps[_sl(a, 0, n - 1)]) / dx
        g2 = gn ** 2
        for b in axes:
            if b != a:
                g2 = g2 + face_average(g[b], a) ** 2
        na = -gn / (np.sqrt(g2) + delta)
        pos = na > 0.0
        cUU, cU, cD, h = _upwind_triplets(c_old, a, pos)
        corr = van_leer_weight(cUU, cU, cD, h) * (cD - cU)
        eUU, eU, eD, h2 = _upwind_triplets(eps, a, pos)
        evl = eU + van_leer_weight(eUU, eU, eD, h2) * (eD - eU)
        out[a] = dict(na=na, pos=pos, corr=corr, eps_vl=evl)
    return out


def ivos_face_flux(c, a, fd, prm):
    """F_f / V = k_c n_a c_f / dx on interior faces along a (sign along +a),
    with c_f = c_U + corr (upwind value of c plus the deferred van Leer
    correction of ``ivos_faces``)."""
    n = c.shape[_nax(a)]
    m1 = c[_sl(a, 0, n - 1)]; p0 = c[_sl(a, 1, n)]
    cU = np.where(fd["pos"], m1, p0)
    cf = cU + fd["corr"]
    return prm["kc"] * fd["na"] * cf / prm["dx"]


def ivos_rates(eps, c, faces, prm):
    """R_f = eps div(Phi) (mass transfer) and R = eps div(Phi) - div(eps_vl Phi)
    (Eq. RfiVoS, Sec. 2.3).  Reading: R_f is the transport sink and R the
    solid source, so the reactant consumed in one cell may dissolve solid in
    its neighbour; boundary faces carry no reactive flux."""
    shp = _shape(prm)
    divF = np.zeros(shp)
    divEF = np.zeros(shp)
    for a in _axes(prm):
        n = shp[_nax(a)]
        F = ivos_face_flux(c, a, faces[a], prm)
        EF = faces[a]["eps_vl"] * F
        divF[_sl(a, 0, n - 1)] += F; divF[_sl(a, 1, n)] -= F
        divEF[_sl(a, 0, n - 1)] += EF; divEF[_sl(a, 1, n)] -= EF
    Rf = eps * divF
    return Rf - divEF, Rf


# --------------------------------------------------------------------------
# S5: implicit diffusion-reaction for the concentration
# --------------------------------------------------------------------------

def transport_system(eps_old, eps, c_old, u, prm, dt, kr=None, faces=None):
    """Implicit transport system for c^{n+1} (Eq. concentrationDBS, Sec. 2.2).

      eps^{n+1} c^{n+1}/dt - div(eps_f D grad c^{n+1}) + zeta R_f(c^{n+1})
          = eps^n c^n/dt - div(c^n_f u^{n+1})

    with D* = D (Sec. 2.2), eps_f = mean of the two cells, c = c_in on the
    inlet faces (ghost 2 c_in - c_P), zero diffusive flux at the outlet and
    walls.  R_f: VoS-psi(') -> kr c (diagonal, kr from ``vos_coefficient``);
    iVoS -> eps div(Phi_R) with face values c_U^{n+1} + corr (implicit
    upwind; the van Leer correction from c^n goes to the right-hand side).
    Reading: the stoichiometric coefficient zeta multiplies the transport
    sink (boundary condition Eq. bcc1).
    """
    shp = _shape(prm)
    N = int(np.prod(shp))
    dx, D, zeta = prm["dx"], prm["D"], prm["zeta"]
    num = np.arange(N).reshape(shp)
    rows, cols, vals = [], [], []
    diag = eps / dt
    rhs = eps_old * c_old / dt - advection_divergence(c_old, u, prm)
    for a in _axes(prm):
        n = shp[_nax(a)]
        ef = D * face_average(eps, a) / dx ** 2
        P = num[_sl(a, 0, n - 1)].ravel(); Q = num[_sl(a, 1, n)].ravel(); cf = ef.ravel()
        rows += [P, Q, P, Q]; cols += [P, Q, Q, P]; vals += [cf, cf, -cf, -cf]
    inl = _sl(0, 0, 1)
    diag = diag.copy()
    diag[inl] += 2.0 * D * eps[inl] / dx ** 2
    rhs[inl] += 2.0 * D * eps[inl] * prm["c_in"] / dx ** 2
    if kr is not None:
        diag = diag + zeta * kr
    rhs = rhs.ravel().copy()
    if faces is not None:
        kc = prm["kc"]
        for a in _axes(prm):
            n = shp[_nax(a)]
            fd = faces[a]
            Pm = num[_sl(a, 0, n - 1)]; Qp = num[_sl(a, 1, n)]
            U = np.where(fd["pos"], Pm, Qp)
            s = kc * fd["na"] / dx
            eP = eps[_sl(a, 0, n - 1)]; eQ = eps[_sl(a, 1, n)]
            for row, sign, ecell in ((Pm, 1.0, eP), (Qp, -1.0, eQ)):
                coef = zeta * sign * ecell * s
                rows.append(row.ravel()); cols.append(U.ravel()); vals.append(coef.ravel())
                np.subtract.at(rhs, row.ravel(), (coef * fd["corr"]).ravel())
    rows.append(num.ravel()); cols.append(num.ravel()); vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    return A, rhs


# --------------------------------------------------------------------------
# One time step
# --------------------------------------------------------------------------

def step(state, dt, prm, solver="direct", rtol=1e-13):
    """One micro-continuum time step (App. B order).

    S1 eps (Eq. mbs) and k (Eq. perm); S2 momentum predictor per component;
    S3 pressure correction and projection; S4 explicit van Leer advection;
    S5 implicit diffusion + reaction; S6 reaction rates R, R_f from c^{n+1};
    S7 diagnostics.  Returns (new_state, stats).

    Transient reading (flow_subiters = 1): S2-S6 run once.  Quasi-static
    reading (flow_subiters = M > 1, App. A and B: flow and transport iterated
    to a steady state with eps frozen, the rate refreshed after every
    iteration): S1 runs once, then S2-S6 are repeated with the latest
    iterate as the "old" velocity and concentration and eps^{n+1} in both
    storage terms, so that a fixed point u = u^m, p = p^m, c = c^m satisfies
    the quasi-static equations (Eq. momentumDBSQS without inertia,
    Eq. contDBSQS, Eq. concentrationDBSQS) exactly; the sub-iterations
    march in a pseudo time step qs_dtau (0: dt), while dt itself only
    advances eps (App. A: with the flow and transport quasi-static, the
    time step is set by the motion of the solid).  The loop stops after M iterations or when the
    relative changes |u^{m+1} - u^m| / |u^{m+1}|, |p^{m+1} - p^m|_eps /
    |p^{m+1}|_eps and |c^{m+1} - c^m| / |c^{m+1}| are all <= qs_rtol
    (qs_rtol = 0: always M iterations); L2 norms over all faces / cells, the
    pressure's weighted by eps.  Reading: the pressure inside the solid,
    tied to the rest only through links of order eps_min and damped by the
    Kozeny-Carman drag, relaxes orders of magnitude more slowly than in the
    pore space while it barely moves the flow, so its change is measured
    with the fluid fraction as weight.
    """
    shp = _shape(prm)
    axes = _axes(prm)
    method = int(prm["method"])
    M = int(prm.get("flow_subiters", 1))
    qs_rtol = float(prm.get("qs_rtol", 0.0))
    dtau = float(prm.get("qs_dtau", 0.0)) if M > 1 else 0.0
    if not dtau > 0.0:
        dtau = dt
    eps_n = state["eps"]
    eps, excess = solid_update(eps_n, state["R"], dt, prm)
    eps_store = eps_n if M == 1 else eps
    u_it, p_it, c_it, R_it = state["u"], state["p"], state["c"], state["R"]
    qs_iters, du, dp, dc = 0, float("nan"), float("nan"), float("nan")
    for m in range(M):
        # S2
        ustar = [x.copy() for x in u_it]
        for a in axes:
            A, b, unk = momentum_system(a, eps, p_it, u_it[a], dtau, prm, u_all=u_it)
            ustar[a][unk] = _solve(A, b, True, solver, rtol)
        # S3
        A, b = pressure_system(eps, ustar, R_it, dtau, prm)
        phi = _solve(A, b, True, solver, rtol).reshape(shp)
        u = project(ustar, phi, eps, dtau, prm)
        p = p_it + phi
        # S5/S6
        lam = float("nan")
        if method == VOS_IVOS:
            faces = ivos_faces(eps, c_it, prm)
            A, b = transport_system(eps_store, eps, c_it, u, prm, dtau, faces=faces)
            c = _solve(A, b, False, solver, rtol).reshape(shp)
            R, Rf = ivos_rates(eps, c, faces, prm)
        else:
            lam = prm["lam"] if method == VOS_PSI else vos_lambda(eps, prm)
            kr = vos_coefficient(eps, prm, lam)
            A, b = transport_system(eps_store, eps, c_it, u, prm, dtau, kr=kr)
            c = _solve(A, b, True, solver, rtol).reshape(shp)
            R = kr * c
            Rf = R.copy()
        qs_iters = m + 1
        if M > 1:
            du_num = sum(float(np.sum((u[a] - u_it[a]) ** 2)) for a in axes)
            du_den = sum(float(np.sum(u[a] ** 2)) for a in axes)
            du = float(np.sqrt(du_num / du_den)) if du_den > 0 else 0.0
            dcn, dcd = float(np.sum((c - c_it) ** 2)), float(np.sum(c ** 2))
            dc = float(np.sqrt(dcn / dcd)) if dcd > 0 else 0.0
            dpn, dpd = float(np.sum(eps * phi ** 2)), float(np.sum(eps * p ** 2))
            dp = float(np.sqrt(dpn / dpd)) if dpd > 0 else 0.0
        prev_c = c_it
        u_it, p_it, c_it, R_it = u, p, c, R
        if M > 1 and qs_rtol > 0 and du <= qs_rtol and dp <= qs_rtol and dc <= qs_rtol:
            break
    new = dict(eps=eps, c=c, p=p, u=u, R=R, Rf=Rf, t=state["t"] + dt,
               step=state["step"] + 1)
    stats = diagnostics(dict(state, c=prev_c), new, prm)
    stats.update(lam=lam, clamp_excess=excess, qs_iters=qs_iters, qs_du=du, qs_dp=dp, qs_dc=dc)
    return new, stats


def run(eps_s, prm, dts, solver="direct", rtol=1e-13):
    st = init_state(eps_s, prm)
    stats = []
    for dt in dts:
        st, s = step(st, dt, prm, solver=solver, rtol=rtol)
        stats.append(s)
    return st, stats


def diagnostics(prev, new, prm):
    """Global FP64 diagnostics of a step from ``prev`` (fields at t^n) to
    ``new`` (t^{n+1}).

    * porosity: mean eps^{n+1} (the total porosity phi of Sec. 2.5);
    * reactant = sum eps c V, sum_R = sum R V, sum_Rf = sum R_f V;
    * q_in, q_out: volumetric flow through the inlet and outlet faces,
      sum u_f A_f with A_f = dx^(d-1) (Q_i of Sec. 2.5 at the inlet);
    * flux_in, flux_out: reactant carried through the inlet and outlet
      faces during the step: inlet u_f c_in plus the diffusive flux
      2 D eps_P (c_in - c_P^{n+1}) / dx of the Dirichlet ghost, outlet
      u_f c_P^n (the explicit convective flux), times A_f.  With them the
      integral form of Eq. concentrationDBS over a step reads
      sum(eps c V)^{n+1} - sum(eps c V)^n = dt (flux_in - flux_out - zeta sum_Rf);
    * umax = max over all faces of |u_f| / eps_f (interior faces: mean of
      the two cells; boundary faces: the adjacent cell) and rmax = max |V_m R|,
      the two quantities the time-step limit of App. D is built from.
    """
    shp = _shape(prm)
    dim = int(prm["dim"])
    dx, D = prm["dx"], prm["D"]
    V = dx ** dim
    A = dx ** (dim - 1)
    eps, c, u = new["eps"], new["c"], new["u"]
    nx = shp[2]
    q_in = float(np.sum(u[0][_sl(0, 0, 1)]) * A)
    q_out = float(np.sum(u[0][_sl(0, nx, nx + 1)]) * A)
    e0 = eps[_sl(0, 0, 1)]
    fin = u[0][_sl(0, 0, 1)] * prm["c_in"] + 2.0 * D * e0 * (prm["c_in"] - c[_sl(0, 0, 1)]) / dx
    fout = u[0][_sl(0, nx, nx + 1)] * prev["c"][_sl(0, nx - 1, nx)]
    return dict(porosity=float(np.mean(eps)), reactant=float(np.sum(eps * c) * V),
                sum_R=float(np.sum(new["R"]) * V), sum_Rf=float(np.sum(new["Rf"]) * V),
                q_in=q_in, q_out=q_out, flux_in=float(np.sum(fin) * A), flux_out=float(np.sum(fout) * A),
                umax=interstitial_speed_max(new, prm), rmax=float(np.max(np.abs(prm["Vm"] * new["R"]))))


def upscaled(state, prm):
    """Darcy-scale characterisation of the domain (Sec. 2.5).

    * phi: total porosity, mean eps;
    * U_D = Q_i / A_i: inlet flow rate over inlet area (sum over the inlet
      faces of u_f A_f, over ny nz A_f);
    * K = nu U_D L_D / dP.  Reading: the pressure is stored at cell centres
      with a zero-gradient inlet condition, so dP is the mean pressure of the
      first cell column (i = 0) minus the outlet face value 0 and L_D is the
      distance between them, (nx - 1/2) dx (for uniform Darcy flow this
      gives K = k of Eq. perm exactly);
    * a = (1/V_Omega) int_Gamma dS, with the surface area density of the
      micro-continuum |grad eps| (the integral VoS-psi' normalises by,
      Sec. 2.4; centred gradient): a = mean |grad eps|;
    * alpha = (1/a) int_Gamma c dS / int_Omega_f c dV with
      int_Gamma c dS = sum c |grad eps| V and int_Omega_f c dV = sum eps c V;
    * reference length L = sqrt(f K / phi), f = 12 in 2D (channel size of a
      bundle of straight channels, BM2) and f = 8 in 3D (throat radius of a
      capillary bundle, BM3); reference velocity U = U_D / phi; with them
      Pe = U L / D, Da = k_c / U, Ki = Da Pe (Sec. 2.5).
    Quantities whose denominator vanishes are NaN."""
    shp = _shape(prm)
    dim = int(prm["dim"])
    dx = prm["dx"]
    nz, ny, nx = shp
    eps, c, p = state["eps"], state["c"], state["p"]
    A = dx ** (dim - 1)
    V = dx ** dim
    phi = float(np.mean(eps))
    Q = float(np.sum(state["u"][0][_sl(0, 0, 1)]) * A)
    Ai = ny * nz * A
    UD = Q / Ai
    dP = float(np.mean(p[_sl(0, 0, 1)]))
    LD = (nx - 0.5) * dx
    nan = float("nan")
    K = prm["nu"] * UD * LD / dP if dP != 0.0 else nan
    g = central_gradient(eps, dx, _axes(prm))
    mag = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    a = float(np.sum(mag) * V / (eps.size * V))
    cs = float(np.sum(c * mag) * V)
    cv = float(np.sum(eps * c) * V)
    alpha = (cs / cv) / a if (a != 0.0 and cv != 0.0) else nan
    f = 12.0 if dim == 2 else 8.0
    Lr = float(np.sqrt(f * K / phi)) if K == K and K > 0 else nan
    Ur = UD / phi
    Pe = Ur * Lr / prm["D"] if prm["D"] > 0 else nan
    Da = prm["kc"] / Ur if Ur != 0 else nan
    return dict(phi=phi, Q_in=Q, A_in=Ai, U_D=UD, dP=dP, L_D=LD, K=K, a=a, alpha=alpha,
                L_ref=Lr, U_ref=Ur, Pe=Pe, Da=Da, Ki=Da * Pe)


def interstitial_speed_max(state, prm):
    """max over all faces of |u_f| / eps_f: eps_f is the mean of the two cells
    of an interior face and the adjacent cell of a boundary face."""
    shp = _shape(prm)
    eps = state["eps"]
    umax = 0.0
    for a in _axes(prm):
        n = shp[_nax(a)]
        ef = np.zeros_like(state["u"][a])
        ef[_sl(a, 1, n)] = face_average(eps, a)
        ef[_sl(a, 0, 1)] = eps[_sl(a, 0, 1)]
        ef[_sl(a, n, n + 1)] = eps[_sl(a, n - 1, n)]
        umax = max(umax, float(np.max(np.abs(state["u"][a]) / ef)))
    return umax


def suggest_dt(state, prm, cfl, deps_max):
    """min(cfl dx / max_f |u_f|/eps_f, deps_max / max |V_m R|)  (App. D:
    the time step is limited by the largest change of eps per step, here
    eps changes by dt V_m R (Eq. mbs); reading: the convective CFL uses the
    interstitial speed |u_f|/eps_f).  +inf when neither limit applies."""
    umax = interstitial_speed_max(state, prm)
    rmax = float(np.max(np.abs(prm["Vm"] * state["R"])))
    dt1 = cfl * prm["dx"] / umax if umax > 0 else np.inf
    dt2 = deps_max / rmax if rmax > 0 else np.inf
    return min(dt1, dt2)
