"""Pins of the CPU oracle against closed forms, invariants and the paper's
identities (no GPU).  Each test names the passage it checks.

These pin the oracle to something other than itself: discrete-exact
closed-form profiles (Poiseuille, Brinkman, Darcy, 1D diffusion-reaction),
exact identities of the method (Sec. 2.3 conservative term, Sec. 2.4
global area, Eq. mbs mass balance), and limiting cases (sharp interface,
front speed of Eq. Ws).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import vos_oracle as O
from paper_2204_07019_gb300 import inputs as I


def _run_to_steady(es, prm, dt, max_steps=600, tol_u=1e-13):
    st = O.init_state(es, prm)
    for _ in range(max_steps):
        u0 = st["u"][0].copy()
        p0 = st["p"].copy()
        st, _ = O.step(st, dt, prm)
        du = np.abs(st["u"][0] - u0).max()
        dp = np.abs(st["p"] - p0).max()
        if du < tol_u and dp < 1e-12 * max(1.0, np.abs(st["p"]).max()):
            return st
    raise AssertionError("no steady state")


# ---------------------------------------------------------------- closures

def test_kozeny_carman_values():
    """Eq. perm: k = k0 eps^3/(1-eps)^2, stored as its inverse."""
    k0 = 2.5e-3
    assert O.kozeny_carman_kinv(np.array(1.0), k0) == 0.0
    assert O.kozeny_carman_kinv(np.array(0.5), k0) == pytest.approx(0.25 / (k0 * 0.125), rel=1e-15)
    e = 0.3
    assert 1.0 / O.kozeny_carman_kinv(np.array(e), k0) == pytest.approx(k0 * e ** 3 / (1 - e) ** 2, rel=1e-14)


def test_van_leer_limiter_values():
    """van Leer (1974) limiter: psi(0)=0, psi(1)=1, psi(3)=3/2, psi(1/3)=1/2,
    psi(r<0)=0, psi -> 2, symmetry psi(1/r) = psi(r)/r, TVD region."""
    psi = O.van_leer_psi
    assert psi(np.array(0.0)) == 0.0
    assert psi(np.array(1.0)) == 1.0
    assert psi(np.array(3.0)) == pytest.approx(1.5, rel=1e-15)
    assert psi(np.array(1.0 / 3.0)) == pytest.approx(0.5, rel=1e-15)
    assert psi(np.array(-2.0)) == 0.0
    assert psi(np.array(1e12)) == pytest.approx(2.0, rel=1e-11)
    r = np.geomspace(1e-3, 1e3, 61)
    assert np.allclose(psi(1.0 / r), psi(r) / r, rtol=1e-14)
    assert np.all(psi(r) <= np.minimum(2 * r, 2.0) + 1e-15)


def test_van_leer_harmonic_mean_form():
    """van Leer's limited correction is half the harmonic mean of the two
    one-sided differences (ref. 1974-vanLeer): with a = c_U - c_UU and
    b = c_D - c_U, w (c_D - c_U) = a b / (a + b) when a and b have one sign
    and 0 otherwise, so the face value stays between c_U and c_D."""
    rng = np.random.default_rng(5)
    cUU, cU, cD = rng.uniform(-1.0, 1.0, (3, 20000))
    a, b = cU - cUU, cD - cU
    corr = O.van_leer_weight(cUU, cU, cD, np.ones(cU.shape, dtype=bool)) * b
    same = a * b > 0
    assert 0.3 < same.mean() < 0.7
    np.testing.assert_allclose(corr[same], (a * b / (a + b))[same], rtol=1e-13, atol=0)
    assert np.all(corr[~same] == 0.0)
    cf = cU + corr
    assert np.all(cf >= np.minimum(cU, cD) - 1e-15) and np.all(cf <= np.maximum(cU, cD) + 1e-15)


def test_van_leer_linear_profile_exact():
    """A second-order TVD scheme reconstructs a linear profile exactly
    (r = 1 -> c_f = midpoint), both flow directions; first face upwind."""
    nx = 12
    prm = I.make_params((1, 1, nx), Pe=1, Da=0, L=1, method="psi")
    c = (3.0 + 0.5 * np.arange(nx))[None, None, :]
    for sgn in (1.0, -1.0):
        pos = np.full((1, 1, nx - 1), sgn > 0)
        cUU, cU, cD, h = O._upwind_triplets(c, 0, pos)
        cf = cU + O.van_leer_weight(cUU, cU, cD, h) * (cD - cU)
        mid = 0.5 * (c[..., :-1] + c[..., 1:])
        inner = slice(1, nx - 1) if sgn > 0 else slice(0, nx - 2)
        assert np.allclose(cf[..., inner], mid[..., inner], rtol=0, atol=1e-14)
        edge = 0 if sgn > 0 else nx - 2
        assert cf[0, 0, edge] == cU[0, 0, edge]


def test_advection_tvd_no_new_extrema():
    """Explicit van Leer advection of a step at CFL 0.5 creates no new
    extrema (TVD property of the limiter, ref. 1974-vanLeer)."""
    nx = 64
    prm = I.make_params((1, 1, nx), Pe=1, Da=0, L=1, method="psi", wall_mask=0)
    u = [np.ones((1, 1, nx + 1)), np.zeros((1, 2, nx)), np.zeros((0,))]
    c = np.zeros((1, 1, nx))
    c[..., :20] = 1.0
    for _ in range(40):
        c = c - 0.5 * O.advection_divergence(c, u, prm)
        assert c.min() >= -1e-15 and c.max() <= 1.0 + 1e-15


# ---------------------------------------------------------------- flow

def test_poiseuille_discrete_exact():
    """Sec. 2.2 DBS in pure fluid reduces to Stokes: fully developed channel
    flow.  With no-slip ghosts u_{-1} = -u_0 the discrete profile is exactly
    u_j ~ y_j (H - y_j) + dx^2/4, y_j = (j + 1/2) dx, mean = u_in."""
    for ny in (6, 9):
        nx = 14 * ny
        es = np.zeros((1, ny, nx))
        prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0,
                            c_in=0.0, kc=0.0, u_in=1.3)
        st = _run_to_steady(es, prm, dt=1.0)
        y = np.arange(ny) + 0.5
        f = y * (ny - y) + 0.25
        ref = 1.3 * f / f.mean()
        col = st["u"][0][0, :, nx // 2]
        assert np.max(np.abs(col - ref)) < 1e-11
        # pressure gradient of the developed flow: nu u'' = dp/dx
        G = -(st["p"][0, :, nx // 2 + 1] - st["p"][0, :, nx // 2])
        assert np.allclose(G, 1.3 * 2.0 * 1.0 / f.mean(), rtol=1e-9)


def test_brinkman_channel_discrete_exact():
    """Eq. momentumDBS with uniform eps0 < 1 and no-slip walls (steady, 1D):
    nu u'' - nu eps0 k^-1 u = -eps0 G.  Discrete solution
    u_j = u_p (1 - A cosh(theta (j - c))), cosh theta = 1 + eps0 k^-1 dx^2 / 2,
    c = (n-1)/2, A from the no-slip ghost; k^-1 from Eq. perm."""
    ny, nx = 8, 112
    eps0, k0 = 0.5, 1.0
    es = np.full((1, ny, nx), 1.0 - eps0)
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0, c_in=0.0,
                        kc=0.0, k0=k0)
    st = _run_to_steady(es, prm, dt=1.0)
    kinv = (1 - eps0) ** 2 / (k0 * eps0 ** 3)
    th = math.acosh(1.0 + eps0 * kinv / 2.0)
    cc = (ny - 1) / 2.0
    A = 2.0 / (math.cosh(th * (cc + 1)) + math.cosh(th * cc))
    j = np.arange(ny)
    f = 1.0 - A * np.cosh(th * (j - cc))
    ref = f / f.mean()
    col = st["u"][0][0, :, nx // 2]
    assert np.max(np.abs(col - ref)) < 1e-11


def test_darcy_limit_exact():
    """Uniform eps0, free-slip sides: plug flow u = u_in and Darcy's law
    dp/dx = -nu k^-1 u_in with k from Eq. perm (Sec. 2.2)."""
    ny, nx = 4, 24
    eps0, k0, nu, uin = 0.6, 0.5, 0.7, 0.9
    es = np.full((1, ny, nx), 1.0 - eps0)
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=nu, c_in=0.0,
                        kc=0.0, k0=k0, u_in=uin, wall_mask=0)
    st = _run_to_steady(es, prm, dt=1.0)
    kinv = (1 - eps0) ** 2 / (k0 * eps0 ** 3)
    assert np.allclose(st["u"][0], uin, rtol=1e-12)
    dpdx = np.diff(st["p"][0], axis=1)
    assert np.allclose(dpdx, -nu * kinv * uin, rtol=1e-10)
    # outlet Dirichlet p = 0 on the boundary face: p_last = -dp/dx * dx/2
    assert np.allclose(st["p"][0, :, -1], nu * kinv * uin * 0.5, rtol=1e-10)


def test_projection_divergence_equals_source():
    """Eq. contDBS: div u^{n+1} = R V_m (1 - rho_s/rho) after the projection,
    and 0 for rho_s = rho (Eq. contDBSQS)."""
    es = I.calcite_post_2d(48, 16, 16.0, 8.0, 4.0)
    for rr in (1.0, 2.5):
        prm = I.make_params(es.shape, Pe=1, Da=1.0, L=8, method="ivos", rho_ratio=rr,
                            Vm=0.05)
        st = O.init_state(es, prm)
        for _ in range(3):
            R = st["R"].copy()
            st, _ = O.step(st, 0.5, prm)
            div = O.divergence(st["u"], prm)
            s = R * prm["Vm"] * (1.0 - rr)
            assert np.max(np.abs(div - s)) < 1e-10


def test_pressure_operator_laplacian_and_spd():
    """For eps = 1 the pressure operator is the 5-point Laplacian: applied to
    phi = x^2 + 3 y^2 it returns -8/dx^2 ... at interior cells, i.e. -lap(phi).
    It is symmetric positive definite (Dirichlet outlet)."""
    ny, nx = 7, 9
    es = np.zeros((1, ny, nx))
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi")
    eps = np.ones((1, ny, nx))
    us = O.init_state(es, prm)["u"]
    A, _ = O.pressure_system(eps, us, np.zeros_like(eps), 1.0, prm)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    phi = (x[None, :] ** 2 + 3 * y[:, None] ** 2)[None]
    r = (A @ phi.ravel()).reshape(phi.shape)
    assert np.allclose(r[0, 1:-1, 1:-1], -8.0, atol=1e-11)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > 0


# ---------------------------------------------------------------- transport

def test_diffusion_reaction_1d_discrete_exact():
    """Steady 1D diffusion with a first-order sink (Eq. concentrationDBS with
    R_f = kappa c, u = 0): the discrete solution is c_i = a r^i + b r^-i,
    r + 1/r = 2 + kappa dx^2 / (eps D), with the inlet Dirichlet ghost
    2 c_in - c_0 and a zero-gradient outlet."""
    nx = 30
    eps0, D, kappa, cin = 0.8, 2.0, 0.15, 1.0
    es = np.full((1, 1, nx), 1 - eps0)
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", D=D, u_in=0.0,
                        c_in=cin, wall_mask=0)
    eps = np.full((1, 1, nx), eps0)
    u = [np.zeros((1, 1, nx + 1)), np.zeros((1, 2, nx)), np.zeros((0,))]
    A, b = O.transport_system(eps, eps, np.zeros_like(eps), u, prm, 1e30,
                              kr=np.full_like(eps, kappa))
    import scipy.sparse.linalg as spla
    c = spla.spsolve(A.tocsc(), b)
    a = eps0 * D
    t = 2.0 + kappa / a
    r = (t + math.sqrt(t * t - 4)) / 2.0
    # unknowns (alpha, beta): outlet ghost c_n = c_{n-1}; inlet ghost c_-1 = 2cin - c_0
    M = np.array([[r ** nx - r ** (nx - 1), r ** -nx - r ** -(nx - 1)],
                  [1.0 / r + 1.0, r + 1.0]])
    al, be = np.linalg.solve(M, [0.0, 2 * cin])
    ref = al * r ** np.arange(nx) + be * r ** -np.arange(nx)
    assert np.max(np.abs(c - ref)) < 1e-12


def _small_case(method, seed=3, shape=(1, 12, 40), Pe=2.0, Da=0.5):
    es = np.zeros(shape)
    es2 = I.calcite_post_2d(shape[2], shape[1], 14.0, shape[1] / 2, 4.0)
    es[:] = es2
    prm = I.make_params(shape, Pe=Pe, Da=Da, L=8, method=method, Vm=0.05)
    return es, prm


@pytest.mark.parametrize("method", ["psi", "psi_prime", "ivos"])
def test_reactant_mass_balance(method):
    """Eq. concentrationDBS in integral form over one step: change of
    sum(eps c) V = dt (inflow - outflow - zeta sum(R_f) V) (up to the direct
    solver's rounding)."""
    es, prm = _small_case(method)
    st = O.init_state(es, prm)
    dx, D = prm["dx"], prm["D"]
    for n in range(4):
        dt = 0.4
        st1, s = O.step(st, dt, prm)
        before = np.sum(st["eps"] * st["c"])
        after = np.sum(st1["eps"] * st1["c"])
        inflow = np.sum(st1["u"][0][..., 0] * prm["c_in"]) \
            + np.sum(2 * D * st1["eps"][..., 0] * (prm["c_in"] - st1["c"][..., 0]) / dx)
        outflow = np.sum(st1["u"][0][..., -1] * st["c"][..., -1])
        sink = prm["zeta"] * np.sum(st1["Rf"])
        lhs = after - before
        rhs = dt * (inflow - outflow - sink)
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(before), abs(after))
        st = st1


@pytest.mark.parametrize("method", ["psi", "psi_prime", "ivos"])
def test_no_reaction_degenerate(method):
    """Da = 0 (k_c = 0): every rate is exactly zero and the solid does not
    change, whatever the reactive-surface form; the reactant is only
    transported, so with c = 0 inside and c_in = 1 at the inlet it stays in
    [0, c_in] (explicit TVD advection at CFL <= 1/2, implicit M-matrix
    diffusion)."""
    es = I.calcite_post_2d(40, 20, 14.0, 10.0, 5.0)
    prm = I.make_params(es.shape, Pe=5.0, Da=0.0, L=10.0, method=method)
    st = O.init_state(es, prm)
    eps0 = st["eps"].copy()
    for _ in range(4):
        st, _ = O.step(st, 0.2, prm)
        assert np.all(st["R"] == 0.0) and np.all(st["Rf"] == 0.0)
        np.testing.assert_array_equal(st["eps"], eps0)
        assert st["c"].min() >= -1e-12 and st["c"].max() <= prm["c_in"] + 1e-12
    assert st["c"][..., 0].mean() > 0.05  # the reactant did enter


def test_solid_mass_balance():
    """Eq. mbs: sum(eps^{n+1} - eps^n) V = dt V_m sum(R^n) V - clamp excess."""
    es, prm = _small_case("ivos", Da=5.0)
    prm["Vm"] = 20.0
    st = O.init_state(es, prm)
    for n in range(5):
        st1, s = O.step(st, 0.5, prm)
        lhs = np.sum(st1["eps"] - st["eps"])
        rhs = 0.5 * prm["Vm"] * np.sum(st["R"]) - s["clamp_excess"]
        assert abs(lhs - rhs) < 1e-12 * max(1.0, np.sum(st["eps"]))
        st = st1
    assert s["clamp_excess"] != 0.0  # the clamp was exercised


# ---------------------------------------------------------------- reaction

def test_ivos_sharp_interface():
    """Sec. 2.3: between a fluid cell P (eps = 1) and a solid cell N
    (eps ~ 0) the reactant is consumed in P (R_f,P = k_c c_P / dx) and the
    solid dissolves in N (R_N = k_c c_P / dx (1 - eps_N)), R_P = 0."""
    nx = 4
    prm = I.make_params((1, 1, nx), Pe=1, Da=0.7, L=1, method="ivos")
    em = prm["eps_min"]
    eps = np.array([1.0, 1.0, em, em])[None, None]
    c = np.array([0.6, 0.6, 0.1, 0.1])[None, None]
    faces = O.ivos_faces(eps, c, prm)
    R, Rf = O.ivos_rates(eps, c, faces, prm)
    na = (1 - em) / ((1 - em) + 1e-8)
    F = 0.7 * 0.6 * na
    assert np.allclose(R[0, 0], [0.0, 0.0, F * (1 - em), 0.0], rtol=1e-15, atol=1e-18)
    assert np.allclose(Rf[0, 0], [0.0, F, -em * F, 0.0], rtol=1e-15, atol=1e-18)
    assert abs(F - 0.7 * 0.6) < 1e-7


@pytest.mark.parametrize("dim", [2, 3])
def test_ivos_conservative_term_sums_to_zero(dim):
    """Sec. 2.3: sum of -div(eps Phi) over the domain vanishes, so
    sum R = sum R_f (= sum eps div Phi) for any eps, c."""
    shape = (1, 17, 23) if dim == 2 else (7, 9, 11)
    prm = I.make_params(shape, Pe=1, Da=1.3, L=1, method="ivos")
    eps = I.random_field(shape, 1, 1e-4, 1.0, smooth=1)
    c = I.random_field(shape, 2, 0.0, 1.0)
    faces = O.ivos_faces(eps, I.random_field(shape, 3), prm)
    R, Rf = O.ivos_rates(eps, c, faces, prm)
    assert abs(R.sum() - Rf.sum()) < 1e-13 * np.abs(Rf).sum()
    assert np.abs(R - Rf).max() > 1e-3  # the local split is non-trivial


def test_ivos_smooth_limit_converges():
    """Sec. 2.3: R = -Phi . grad eps = k_c c |grad eps| for smooth fields;
    the discrete iVoS rate converges to it under refinement."""
    errs = []
    for n in (32, 64, 128):
        dx = 1.0 / n
        prm = I.make_params((1, n, n), Pe=1, Da=1.0, L=1, method="ivos", dx=dx)
        x = (np.arange(n) + 0.5) * dx
        X, Y = np.meshgrid(x, x)
        eps = (0.5 + 0.3 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y))[None]
        c = (1.0 + 0.5 * X * Y)[None]
        gx = 0.3 * 2 * np.pi * np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
        gy = -0.3 * np.pi * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
        exact = 1.0 * c[0] * np.hypot(gx, gy)
        faces = O.ivos_faces(eps, c, prm)
        R, _ = O.ivos_rates(eps, c, faces, prm)
        m = slice(n // 8, n - n // 8)
        errs.append(np.mean(np.abs(R[0][m, m] - exact[m, m])))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]


def test_vos_psi_prime_conserves_area():
    """Sec. 2.4: with lambda(eps) = int|grad eps| / int|grad eps| eps(1-eps)
    the localised area sum psi' |grad eps| equals sum |grad eps|."""
    for shape in ((1, 20, 30), (6, 8, 10)):
        prm = I.make_params(shape, Pe=1, Da=1.0, L=1, method="psi_prime")
        eps = I.random_field(shape, 5, 1e-4, 1.0, smooth=1)
        lam = O.vos_lambda(eps, prm)
        a_psi = O.vos_coefficient(eps, prm, lam).sum() / prm["kc"]
        g = O.central_gradient(eps, 1.0, O._axes(prm))
        assert a_psi == pytest.approx(np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2).sum(), rel=1e-13)
    # degenerate: uniform eps -> lambda = 4
    assert O.vos_lambda(np.full((1, 4, 5), 0.3), I.make_params((1, 4, 5), 1, 1, 1)) == 4.0


def test_vos_psi_lambda_in_paper_range_calcite_post():
    """Sec. 3.1 reports lambda between 8 and 16 for the calcite post; the
    calcite-post stand-in geometry falls in that range (informative)."""
    es = I.calcite_post_2d()
    prm = I.make_params(es.shape, Pe=1, Da=0.1, L=32, method="psi_prime")
    eps = np.maximum(1 - es, prm["eps_min"])
    assert 8.0 <= O.vos_lambda(eps, prm) <= 16.0


def test_front_speed_reaction_limited():
    """Eq. Ws: the interface moves at M_ws R / rho_s.  Reaction-limited
    (Ki << 1, c = c_in): a flat solid layer under iVoS gains fluid at
    d eps/dt = V_m k_c c_in (1 - eps_min) / dx in its interface cells, i.e. a
    cell holding 1 - eps_min of solid clears in dx / (V_m k_c c_in)."""
    ny, nx = 6, 8
    es = np.zeros((1, ny, nx))
    es[0, :2, :] = 1.0
    prm = I.make_params(es.shape, Pe=1, Da=0.01, L=1, method="ivos", D=1e4, u_in=0.0,
                        Vm=0.5, wall_mask=0)
    st = O.init_state(es, prm)
    st["c"][:] = prm["c_in"]
    st, _ = O.step(st, 1.0, prm)
    e0 = st["eps"].copy()
    st, _ = O.step(st, 1.0, prm)
    rate = (st["eps"] - e0)[0, 1, :]
    expect = prm["Vm"] * prm["kc"] * prm["c_in"] * (1 - prm["eps_min"]) / prm["dx"]
    assert np.allclose(rate, expect, rtol=1e-5)
    assert np.allclose((st["eps"] - e0)[0, 0, :], 0.0, atol=1e-12)


def test_poiseuille_3d_plates_discrete_exact():
    """3D: no-slip plates at y = 0, H and free-slip z sides give the same
    discrete plane-Poiseuille profile, uniform in z (w = 0)."""
    nz, ny, nx = 3, 6, 84
    es = np.zeros((nz, ny, nx))
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0, c_in=0.0,
                        kc=0.0, wall_mask=I.WALL_YM | I.WALL_YP)
    st = _run_to_steady(es, prm, dt=1.0)
    y = np.arange(ny) + 0.5
    f = y * (ny - y) + 0.25
    ref = f / f.mean()
    for k in range(nz):
        assert np.max(np.abs(st["u"][0][k, :, nx // 2] - ref)) < 1e-11
    assert np.max(np.abs(st["u"][2])) < 1e-12


def test_reactant_mass_balance_3d():
    """Integral balance of Eq. concentrationDBS over one step, 3D, iVoS."""
    shape = (6, 7, 16)
    es = I.sphere_rock_3d(shape, seed=2, median_r=2.5, sigma=0.2, target_porosity=0.6,
                          start_solid=0.5, band=2, margin=3.0)
    prm = I.make_params(shape, Pe=2.0, Da=0.5, L=4, method="ivos", Vm=0.05)
    st = O.init_state(es, prm)
    D, dx = prm["D"], prm["dx"]
    for _ in range(3):
        st1, _ = O.step(st, 0.3, prm)
        inflow = np.sum(st1["u"][0][..., 0] * prm["c_in"]) \
            + np.sum(2 * D * st1["eps"][..., 0] * (prm["c_in"] - st1["c"][..., 0]) / dx)
        outflow = np.sum(st1["u"][0][..., -1] * st["c"][..., -1])
        lhs = np.sum(st1["eps"] * st1["c"]) - np.sum(st["eps"] * st["c"])
        rhs = 0.3 * (inflow - outflow - np.sum(st1["Rf"]))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, np.sum(st1["eps"] * st1["c"]))
        st = st1


# ---------------------------------------------------------------- time step and diagnostics

def _dt_state(prm, eps, u0, R):
    shp = (int(prm["nz"]), int(prm["ny"]), int(prm["nx"]))
    u = [np.asarray(u0, dtype=float).reshape(shp[0], shp[1], shp[2] + 1),
         np.zeros((shp[0], shp[1] + 1, shp[2])), np.zeros((0,))]
    return dict(eps=np.asarray(eps, dtype=float).reshape(shp), u=u, R=np.asarray(R, dtype=float).reshape(shp))


def test_suggest_dt_closed_forms():
    """App. D: dt is limited by the largest change of eps in a step, which by
    Eq. mbs is dt V_m |R|, and (reading) by the interstitial CFL number
    |u_f| dt / (eps_f dx).  Hand-built fields whose binding term is known:
    the face porosity of an interior face is the mean of its two cells (a
    cell-based eps would give a different number), |R| enters with V_m and
    its sign does not matter, and the smaller of the two limits wins."""
    prm = I.make_params((1, 1, 4), Pe=1, Da=1, L=1, Vm=0.5, dx=0.25)
    eps = [0.2, 0.6, 1.0, 1.0]
    # faces 0..4: inlet 0.1 / eps 0.2 = 0.5; interior face 1: 0.4 / mean(0.2, 0.6) = 1.0;
    # outlet 0.5 / eps 1.0 = 0.5
    u = [0.1, 0.4, 0.0, 0.0, 0.5]
    st = _dt_state(prm, eps, u, [0.0, 0.0, 0.0, 0.0])
    assert O.suggest_dt(st, prm, 0.5, 0.005) == pytest.approx(0.5 * 0.25 / 1.0, rel=1e-15)
    # the rate limit alone: max |Vm R| = 0.5 * 5 = 2.5 (a negative rate binds)
    st = _dt_state(prm, eps, np.zeros(5), [0.0, 3.0, 0.0, -5.0])
    assert O.suggest_dt(st, prm, 0.5, 0.005) == pytest.approx(0.005 / 2.5, rel=1e-15)
    # both: the smaller limit
    st = _dt_state(prm, eps, u, [0.0, 3.0, 0.0, -5.0])
    assert O.suggest_dt(st, prm, 0.5, 0.005) == pytest.approx(min(0.125, 0.002), rel=1e-15)
    # nothing moves: no limit
    st = _dt_state(prm, eps, np.zeros(5), np.zeros(4))
    assert O.suggest_dt(st, prm, 0.5, 0.005) == np.inf
    # uniform flow through pure fluid in 3D: dt = cfl dx / U along every axis
    shp = (3, 4, 5)
    prm3 = I.make_params(shp, Pe=1, Da=1, L=1)
    u3 = [np.full((3, 4, 6), 2.0), np.zeros((3, 5, 5)), np.full((4, 4, 5), -4.0)]
    st3 = dict(eps=np.ones(shp), u=u3, R=np.zeros(shp))
    assert O.suggest_dt(st3, prm3, 0.5, 0.005) == pytest.approx(0.5 / 4.0, rel=1e-15)


@pytest.mark.parametrize("method", ["psi", "ivos"])
def test_step_diagnostics_balance(method):
    """The step's flux diagnostics close the integral balances: with
    rho_s = rho the flow is divergence-free (Eq. contDBSQS), so q_out = q_in
    = u_in x inlet area; the reactant content changes by
    dt (flux_in - flux_out - zeta sum R_f) (Eq. concentrationDBS integrated
    over the domain); umax and rmax give back suggest_dt."""
    es, prm = _small_case(method)
    st = O.init_state(es, prm)
    ny = es.shape[1]
    for _ in range(3):
        dt = 0.4
        st1, s = O.step(st, dt, prm)
        assert s["q_in"] == pytest.approx(prm["u_in"] * ny * prm["dx"], rel=1e-14)
        assert s["q_out"] == pytest.approx(s["q_in"], rel=1e-9)
        before = np.sum(st["eps"] * st["c"]) * prm["dx"] ** 2
        lhs = s["reactant"] - before
        rhs = dt * (s["flux_in"] - s["flux_out"] - prm["zeta"] * s["sum_Rf"])
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(before))
        assert s["umax"] > 0 and s["rmax"] > 0
        dt_ref = min(0.5 * prm["dx"] / s["umax"], 0.005 / s["rmax"])
        assert O.suggest_dt(st1, prm, 0.5, 0.005) == pytest.approx(dt_ref, rel=1e-15)
        st = st1


def test_vos_psi_rate_on_linear_ramp():
    """Eq. RfVoSpsi with lambda = 4 (Sec. 2.4): R = k_c c 4 eps (1 - eps) |grad eps|
    with the centred gradient.  On eps = a + b x + g y the centred gradient
    is exact in interior cells, |grad eps| = sqrt(b^2 + g^2); in the first
    and last column the zero-gradient ghost halves the x component."""
    ny, nx, dx = 9, 12, 0.5
    prm = I.make_params((1, ny, nx), Pe=1, Da=0.7, L=1, method="psi", dx=dx)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    b, g = 0.05, -0.03
    eps = (0.2 + b * x[None, :] + g * y[:, None] + 0.2)[None]
    c = (1.0 + 0.1 * x[None, :] * y[:, None])[None]
    kr = O.vos_coefficient(eps, prm, 4.0)
    R = kr * c
    gx = np.full((ny, nx), b)
    gx[:, 0] = gx[:, -1] = b / 2
    gy = np.full((ny, nx), g)
    gy[0, :] = gy[-1, :] = g / 2
    ref = 0.7 * c[0] * 4.0 * eps[0] * (1 - eps[0]) * np.sqrt(gx ** 2 + gy ** 2)
    np.testing.assert_allclose(R[0], ref, rtol=1e-13, atol=0)
    # the fitted lambda of VoS-psi' replaces the 4, nothing else changes
    lam = O.vos_lambda(eps, prm)
    np.testing.assert_allclose(O.vos_coefficient(eps, prm, lam), kr * lam / 4.0, rtol=1e-14)


# ---------------------------------------------------------------- upscaled properties (Sec. 2.5)

def test_upscaled_permeability_poiseuille():
    """Sec. 2.5: K = nu U_D L_D / dP.  Plane Poiseuille flow between no-slip
    plates H apart has K = H^2/12; the discrete developed profile
    y(H - y) + dx^2/4 (no-slip ghost) gives exactly K = H^2/12 + dx^2/6.  The
    plug inlet adds a fixed entrance loss to dP, so the whole-domain K
    approaches that value as the channel lengthens (error ~ 1/L) and the
    difference of the pressure drops of two lengths is the developed
    gradient exactly.  The reference length sqrt(12 K / phi) of BM2 is then
    the channel width up to the O(dx^2) term."""
    for ny in (6, 10):
        kdev = ny ** 2 / 12.0 + 1.0 / 6.0
        ups = []
        for mult in (12, 24):
            nx = mult * ny
            es = np.zeros((1, ny, nx))
            prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0, c_in=0.0, kc=0.0, u_in=0.7)
            st = _run_to_steady(es, prm, dt=1.0)
            up = O.upscaled(st, prm)
            assert up["U_D"] == pytest.approx(0.7, rel=1e-14)
            assert up["phi"] == 1.0
            assert up["L_D"] == (nx - 0.5) * prm["dx"]
            assert up["K"] == pytest.approx(prm["nu"] * up["U_D"] * up["L_D"] / up["dP"], rel=1e-15)
            ups.append(up)
        G = (ups[1]["dP"] - ups[0]["dP"]) / (ups[1]["L_D"] - ups[0]["L_D"])
        assert 1.0 * 0.7 / G == pytest.approx(kdev, rel=1e-9)
        e1, e2 = kdev - ups[0]["K"], kdev - ups[1]["K"]
        assert 0 < e2 < 0.6 * e1 and e1 < 0.05 * kdev
        assert ups[1]["L_ref"] == pytest.approx(np.sqrt(12.0 * ups[1]["K"]), rel=1e-14)


def test_upscaled_permeability_darcy():
    """Uniform eps0 with free-slip sides: Darcy flow, K = k = k0 eps^3/(1-eps)^2
    (Eq. perm) exactly; in 3D the reference length is sqrt(8 K / phi)."""
    eps0, k0, nu = 0.6, 0.5, 0.7
    for shape in ((1, 4, 24), (3, 4, 20)):
        es = np.full(shape, 1.0 - eps0)
        prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=nu, c_in=0.0, kc=0.0, k0=k0,
                            u_in=0.9, wall_mask=0)
        st = _run_to_steady(es, prm, dt=1.0)
        up = O.upscaled(st, prm)
        k = k0 * eps0 ** 3 / (1 - eps0) ** 2
        assert up["K"] == pytest.approx(k, rel=1e-10)
        f = 12.0 if shape[0] == 1 else 8.0
        assert up["L_ref"] == pytest.approx(np.sqrt(f * k / eps0), rel=1e-10)
        assert up["U_ref"] == pytest.approx(0.9 / eps0, rel=1e-14)


def test_upscaled_surface_area_and_alpha():
    """Sec. 2.5 a = (1/V) int_Gamma dS with |grad eps| as the surface density:
    across a flat solid layer (any monotone ramp) the centred-gradient sum
    telescopes to the jump of eps, so a = (1 - eps_min) A_perp / V_Omega per
    interface.  With a uniform concentration alpha = 1/phi (the surface sees
    the same c as the fluid volume)."""
    ny, nx = 10, 30
    es = np.zeros((1, ny, nx))
    es[0, :, 12:] = 1.0
    es[0, :, 11] = 0.37  # partial ramp cell
    prm = I.make_params(es.shape, Pe=1, Da=1, L=1, dx=0.5)
    st = O.init_state(es, prm)
    st["c"][:] = 0.8
    up = O.upscaled(st, prm)
    dx = prm["dx"]
    area = (1.0 - prm["eps_min"]) * ny * dx
    assert up["a"] == pytest.approx(area / (nx * ny * dx * dx), rel=1e-13)
    assert up["alpha"] == pytest.approx(1.0 / up["phi"], rel=1e-13)
    # a concentration vanishing on the surface cells lowers alpha
    st["c"][0, :, 9:13] = 0.0
    assert O.upscaled(st, prm)["alpha"] < 1e-12


def _printed_tol(value, digits):
    """Half a unit in the last significant digit of a printed value."""
    e = math.floor(math.log10(abs(value)))
    return 0.5 * 10.0 ** (e - digits + 1)


def test_upscaled_reference_numbers_of_benchmark3():
    """Sec. 3.3 worked example (tests/golden/bm3_ketton_reference_numbers.json):
    from Table param3, the 1.7 mm sample radius, K = 16 D and phi = 0.173 the
    paper obtains U = U_D / phi = 5.3e-3 m/s, L = sqrt(8 K / phi) = 27 um,
    Pe = U L / D = 190 and Da = k_c / U = 4.4e-2.  A state with that porosity,
    the Darcy velocity Q_i / (pi r^2) through the inlet and the Darcy pressure
    profile of K gives these numbers back through the oracle to the printed
    digits (12 for 8 in the length, U_D for U or Ki for Da each miss)."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bm3_ketton_reference_numbers.json")))
    inp, out, dig = g["inputs"], g["printed"], g["printed_significant_digits"]
    darcy = 9.869233e-13
    K0 = inp["K0_darcy"] * darcy
    UD = inp["Q_i_m3_s"] / (math.pi * inp["sample_radius_m"] ** 2)
    nz, ny, nx, dx = 3, 4, 10, 2.0e-5
    prm = dict(dim=3, nx=nx, ny=ny, nz=nz, dx=dx, nu=inp["nu_m2_s"], D=inp["D_m2_s"], kc=inp["k_c_m_s"])
    eps = np.full((nz, ny, nx), inp["phi0"])
    u = [np.full((nz, ny, nx + 1), UD), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))]
    # Darcy's law in a uniform medium of permeability K0, outlet face at p = 0
    xc = (np.arange(nx) + 0.5) * dx
    p = np.broadcast_to(inp["nu_m2_s"] * UD / K0 * (nx * dx - xc), (nz, ny, nx)).copy()
    st = dict(eps=eps, c=np.ones_like(eps), p=p, u=u)
    up = O.upscaled(st, prm)
    assert up["K"] == pytest.approx(K0, rel=1e-12)
    for key, name in (("U_ref", "U_m_s"), ("L_ref", "L_m"), ("Pe", "Pe"), ("Da", "Da")):
        assert abs(up[key] - out[name]) <= _printed_tol(out[name], dig[name]), (key, up[key], out[name])


# ---------------------------------------------------------------- quasi-static variant (App. A, App. B)

def test_quasi_static_step_reaches_poiseuille_and_darcy():
    """App. B: with flow_subiters > 1 one step iterates flow and transport
    to a steady state with eps frozen.  From rest, a single call reaches the
    discrete-exact plane-Poiseuille profile (no-slip ghost) and the Darcy
    plug flow with dp/dx = -nu k^-1 u_in (Eq. perm)."""
    ny, nx = 6, 84
    es = np.zeros((1, ny, nx))
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0, c_in=0.0, kc=0.0,
                        flow_subiters=2000, qs_rtol=1e-14)
    st, s = O.step(O.init_state(es, prm), 1.0, prm)
    assert 1 < s["qs_iters"] < 2000 and s["qs_du"] <= 1e-14
    y = np.arange(ny) + 0.5
    f = y * (ny - y) + 0.25
    assert np.max(np.abs(st["u"][0][0, :, nx // 2] - f / f.mean())) < 1e-11
    eps0, k0, nu, uin = 0.6, 0.5, 0.7, 0.9
    es = np.full((1, 4, 24), 1.0 - eps0)
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=nu, c_in=0.0, kc=0.0, k0=k0, u_in=uin,
                        wall_mask=0, flow_subiters=2000, qs_rtol=1e-14)
    st, s = O.step(O.init_state(es, prm), 1.0, prm)
    kinv = (1 - eps0) ** 2 / (k0 * eps0 ** 3)
    assert np.allclose(st["u"][0], uin, rtol=1e-12)
    assert np.allclose(np.diff(st["p"][0], axis=1), -nu * kinv * uin, rtol=1e-10)


def _smooth_porous(method, **over):
    """A porous field without solid cells (eps in [0.55, 0.95]): no near-null
    pressure modes, so the quasi-static sub-iterations converge quickly."""
    ny, nx = 10, 30
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    eps = 0.75 + 0.2 * np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    prm = I.make_params((1, ny, nx), Pe=2.0, Da=2.0, L=8, method=method, Vm=0.0, Sc=1.0, k0=0.5)
    prm.update(over)
    return (1.0 - eps)[None], prm


@pytest.mark.parametrize("method", ["ivos", "psi"])
def test_quasi_static_fixed_point_solves_steady_transport(method):
    """App. A, Eq. concentrationDBSQS: at the converged sub-iteration the
    concentration satisfies div(c u) - div(eps D grad c) + zeta R_f = 0 (the
    pseudo-time storage terms cancel), checked by assembling the transport
    operator with an infinite time step; the flow is divergence-free
    (Eq. contDBSQS)."""
    es, prm = _smooth_porous(method, flow_subiters=3000, qs_rtol=1e-12, qs_dtau=0.5)
    st, s = O.step(O.init_state(es, prm), 1.0, prm)
    assert s["qs_iters"] < 3000 and max(s["qs_du"], s["qs_dp"], s["qs_dc"]) <= 1e-12
    eps, c, u = st["eps"], st["c"], st["u"]
    if method == "ivos":
        A, b = O.transport_system(eps, eps, c, u, prm, 1e300, faces=O.ivos_faces(eps, c, prm))
    else:
        kr = O.vos_coefficient(eps, prm, prm["lam"])
        A, b = O.transport_system(eps, eps, c, u, prm, 1e300, kr=kr)
    res = A @ c.ravel() - b
    scale = np.abs(O.advection_divergence(c, u, prm)).max()
    assert np.abs(res).max() < 1e-9 * scale
    assert np.abs(O.divergence(u, prm)).max() < 1e-10
    # the sink is active: the reactant does not just pass through
    assert s["sum_Rf"] > 1e-3 * s["flux_in"]


def test_quasi_static_result_independent_of_pseudo_step():
    """The converged quasi-static flow and concentration do not depend on
    the pseudo time step of the sub-iterations (eps frozen: V_m = 0)."""
    es, prm = _smooth_porous("ivos", flow_subiters=4000, qs_rtol=1e-13)
    out = []
    for dtau in (0.5, 2.0):
        prm["qs_dtau"] = dtau
        out.append(O.step(O.init_state(es, prm), 1.0, prm)[0])
    a, b = out
    for n in ("c", "p", "R"):
        assert np.linalg.norm(a[n] - b[n]) <= 1e-9 * np.linalg.norm(b[n]), n
    assert np.linalg.norm(a["u"][0] - b["u"][0]) <= 1e-9 * np.linalg.norm(b["u"][0])


def test_quasi_static_single_subiteration_is_the_transient_step():
    """flow_subiters = 1 is the transient step: identical fields."""
    es, prm = _small_case("ivos")
    st = O.init_state(es, prm)
    a, _ = O.step(st, 0.4, prm)
    p2 = dict(prm, flow_subiters=1, qs_rtol=1e-3, qs_dtau=0.1)
    b, _ = O.step(st, 0.4, p2)
    for n in ("eps", "c", "p", "R", "Rf"):
        assert np.array_equal(a[n], b[n]), n


# ---------------------------------------------------------------- inertia term of Eq. momentumDBS

def test_inertia_hand_worked_1d():
    """div(u u / eps) on a single row (free slip, eps = 1), u on the x-faces
    1, 2, 3, 4: cell-centre fluxes U phi with U the cell mean and phi the van
    Leer value (first cell upwind, r = 1 elsewhere: phi = 1, 2.5, 3.5), the
    outlet face's control volume losing u_3 phi_3 = 16 past the outlet."""
    prm = I.make_params((1, 1, 3), Pe=1, Da=0, L=1, wall_mask=0, inertia=1)
    u = [np.array([1.0, 2.0, 3.0, 4.0]).reshape(1, 1, 4), np.zeros((1, 2, 3)), np.zeros((0,))]
    N = O.inertia(u, np.ones((1, 1, 3)), prm)
    F = [1.5 * 1.0, 2.5 * 2.5, 3.5 * 3.5]
    np.testing.assert_allclose(N[0][0, 0, 1:], [F[1] - F[0], F[2] - F[1], 16.0 - F[2]], rtol=1e-15)
    assert np.all(N[1] == 0.0)


def test_inertia_uniform_flow_vanishes():
    """Uniform flow through a uniform porous medium carries no net momentum
    into any control volume: N = 0 (2D and 3D, free-slip sides)."""
    for shape in ((1, 5, 9), (4, 5, 9)):
        prm = I.make_params(shape, Pe=1, Da=0, L=1, wall_mask=0, inertia=1)
        nz, ny, nx = shape
        u = [np.full((nz, ny, nx + 1), 1.7), np.zeros((nz, ny + 1, nx)),
             np.zeros((nz + 1, ny, nx)) if nz > 1 else np.zeros((0,))]
        N = O.inertia(u, np.full(shape, 0.4), prm)
        assert np.abs(N[0][..., 1:]).max() < 1e-12


def test_inertia_interior_fluxes_telescope():
    """Finite-volume conservation: summed over every face of a component,
    the fluxes through interior control-volume faces cancel and only the
    outlet terms remain -- u_n phi_n for the x-component, and for y/z the
    outlet-plane edges, U (the outlet u averaged onto the face) times the
    last column's phi (random fields, 2D and 3D, dx = 1)."""
    for shape in ((1, 7, 11), (5, 6, 8)):
        nz, ny, nx = shape
        prm = I.make_params(shape, Pe=1, Da=0, L=1, inertia=1)
        rng = np.random.default_rng(3)
        u = [rng.normal(size=(nz, ny, nx + 1)), rng.normal(size=(nz, ny + 1, nx)),
             rng.normal(size=(nz + 1, ny, nx)) if nz > 1 else np.zeros((0,))]
        eps = rng.uniform(0.2, 1.0, size=shape)
        N = O.inertia(u, eps, prm)
        ux = u[0][..., nx]
        for a in O._axes(prm):
            phi = u[a] / O.face_porosity(eps, a, prm)
            if a == 0:
                out = np.sum(ux * phi[..., nx])
            elif a == 1:
                out = np.sum(0.5 * (ux[:, :-1] + ux[:, 1:]) * phi[:, 1:-1, nx - 1])
            else:
                out = np.sum(0.5 * (ux[:-1] + ux[1:]) * phi[1:-1, :, nx - 1])
            assert N[a].sum() == pytest.approx(out, rel=1e-12, abs=1e-12), a
            assert np.abs(N[a]).max() > 1.0  # the interior terms are not trivially zero


def test_inertia_leaves_developed_poiseuille_unchanged():
    """Developed channel flow has u . grad u = 0: with the inertia term on,
    the steady profile away from the entrance is still the discrete
    Poiseuille profile (Sec. 2.2 Stokes limit)."""
    ny, nx = 6, 84
    es = np.zeros((1, ny, nx))
    prm = I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=1.0, c_in=0.0, kc=0.0, inertia=1)
    st = _run_to_steady(es, prm, dt=0.5, max_steps=1500)
    y = np.arange(ny) + 0.5
    f = y * (ny - y) + 0.25
    col = st["u"][0][0, :, 3 * nx // 4]
    assert np.max(np.abs(col - f / f.mean())) < 1e-9
    # and the inertia term changed the entrance region (it is active)
    prm0 = dict(prm, inertia=0)
    st0 = _run_to_steady(es, prm0, dt=0.5, max_steps=1500)
    assert np.max(np.abs(st["p"] - st0["p"])) > 1e-3
