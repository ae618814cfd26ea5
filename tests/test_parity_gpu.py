"""GPU path vs the FP64 CPU oracle on the same seeded inputs.

FP64 path: every GPU solve to a relative residual of 1e-11 (the oracle
solves directly), so both compute the unique discrete solution; the bar is
a relative L2 difference <= 1e-9 per field after several steps.  The rates
R, R_f are linear in c but are taken where c may be many orders of
magnitude below c_in (an arriving front), so they are compared against the
rate scale k_c c_in / dx (absolute L2 over the grid) unless the case starts
from a concentration field that already covers the reactive surface.
Mixed path (FP32 inner solves, FP64 refinement, FP64 fields): at the same
tight tolerance the refinement must recover FP64 accuracy (<= 1e-9); at the
production tolerance 1e-8 the measured difference is bounded per field.
"""
import numpy as np
import pytest

from oracle import vos_oracle as O
from paper_2204_07019_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("eps", "c", "u", "v", "w", "p", "R", "Rf")


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07019_gb300 import build_lib, vos
    build_lib.build()
    vos.load_library()
    return vos


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    return d / nb if nb > 0 else d


def oracle_fields(st):
    f = dict(eps=st["eps"], c=st["c"], p=st["p"], R=st["R"], Rf=st["Rf"], u=st["u"][0], v=st["u"][1])
    if st["u"][2].size:
        f["w"] = st["u"][2]
    return f


def run_gpu(V, es, prm, dts, init=None):
    h = V.vos_create(es, prm)
    try:
        if init:
            V.vos_set_fields(h, **init)
        for dt in dts:
            rc = V.vos_step(h, dt)
            assert rc == 0, V.vos_get_stats(h)
        return V.vos_fields(h), V.vos_get_stats(h)
    finally:
        V.vos_destroy(h)


def tight(prm, precision=0):
    prm = dict(prm)
    prm.update(p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000, precision=precision)
    return prm


def compare(V, es, prm, dts, tol, fields=FIELDS, init=None):
    """Run both sides from the same initial state; per-field relative L2.
    Without ``init`` the rates are measured against the scale k_c c_in / dx."""
    st = O.init_state(es, prm)
    if init:
        for k, v in init.items():
            st[k] = np.asarray(v, dtype=np.float64).reshape(st[k].shape).copy()
    for dt in dts:
        st, _ = O.step(st, dt, prm)
    ref = oracle_fields(st)
    got, stats = run_gpu(V, es, prm, dts, init=init)
    errs = {}
    rscale = prm["kc"] * prm["c_in"] / prm["dx"] * np.sqrt(np.asarray(ref["c"]).size)
    for n in fields:
        if n not in ref:
            continue
        if n in ("R", "Rf") and not init:
            errs[n] = np.linalg.norm(got[n] - ref[n]) / max(rscale, 1e-300)
        else:
            errs[n] = rel_l2(got[n], ref[n])
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, (bad, errs, stats)
    return errs, stats


def c_start(es, prm):
    """A concentration field covering the whole domain (c_in decaying along x)."""
    nz, ny, nx = es.shape
    x = (np.arange(nx) + 0.5) / nx
    return {"c": np.broadcast_to(prm["c_in"] * (1.0 - 0.5 * x), es.shape).copy()}


@pytest.mark.parametrize("method", ["ivos", "psi", "psi_prime"])
def test_calcite_post_fp64(V, method):
    """Calcite-post channel (256 x 64, disc R = 16), Pe = 1, Da = 0.1, with a
    larger V_m so that eps changes measurably over 5 steps."""
    es = I.calcite_post_2d()
    prm = tight(I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method=method, Vm=0.5))
    compare(V, es, prm, [0.25] * 5, 1e-9, init=c_start(es, prm))


def test_calcite_post_front_arrival_fp64(V):
    """Same channel from c = 0: the acid front reaches the post during the
    run (rates compared on the k_c c_in / dx scale)."""
    es = I.calcite_post_2d()
    prm = tight(I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method="ivos", Vm=0.5))
    compare(V, es, prm, [0.5] * 6, 1e-9)


def test_ragged_micromodel_2d_fp64(V):
    """Ragged 2D size (77 x 45, not a multiple of the 32-wide tiles), seeded
    discs, iVoS with strong reaction."""
    es = I.disc_micromodel_2d(77, 45, seed=4, rmin=3, rmax=7, target_porosity=0.7)
    prm = tight(I.make_params(es.shape, Pe=10.0, Da=1.0, L=10.0, method="ivos", Vm=0.2))
    compare(V, es, prm, [0.2] * 4, 1e-9, init=c_start(es, prm))


@pytest.mark.parametrize("method", ["ivos", "psi_prime"])
def test_rock_3d_fp64(V, method):
    """3D overlapping-sphere rock on a ragged 37 x 21 x 19 grid."""
    es = I.sphere_rock_3d((19, 21, 37), seed=1, median_r=3.0, sigma=0.3, target_porosity=0.45,
                          start_solid=0.6, band=2, margin=3.0)
    prm = tight(I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method=method, Vm=0.2))
    compare(V, es, prm, [0.2] * 3, 1e-9, init=c_start(es, prm))


def test_edge_all_fluid_and_free_slip_source(V):
    """All-fluid channel with free-slip sides and a dissolution source in the
    continuity equation (rho_s/rho = 2.5) seeded by a solid block."""
    es = np.zeros((1, 12, 40))
    es[0, 4:8, 10:14] = 1.0
    prm = tight(I.make_params(es.shape, Pe=2.0, Da=2.0, L=4.0, method="ivos", Vm=0.5, rho_ratio=2.5,
                              wall_mask=0))
    compare(V, es, prm, [0.3] * 4, 1e-9, init=c_start(es, prm))


def test_edge_single_row_channel(V):
    """ny = 1: no v unknowns; 1D transport along the channel, VoS-psi."""
    es = np.zeros((1, 1, 50))
    es[0, 0, 20:30] = 0.6
    prm = tight(I.make_params(es.shape, Pe=5.0, Da=1.0, L=4.0, method="psi", Vm=0.5, wall_mask=0))
    compare(V, es, prm, [0.3] * 4, 1e-9, fields=("eps", "c", "u", "p", "R", "Rf"), init=c_start(es, prm))


def test_edge_thin_3d(V):
    """3D with nz = 2 (one coarsening step in z only), walls on all sides."""
    es = I.sphere_rock_3d((2, 14, 30), seed=3, median_r=2.5, sigma=0.2, target_porosity=0.6,
                          start_solid=0.5, band=2, margin=3.0)
    prm = tight(I.make_params(es.shape, Pe=3.0, Da=0.5, L=5.0, method="ivos", Vm=0.3))
    compare(V, es, prm, [0.25] * 3, 1e-9, init=c_start(es, prm))


def test_mixed_precision_tight_recovers_fp64(V):
    """Mixed path (FP32 multigrid / Krylov, FP64 refinement) at rtol 1e-11
    reaches the FP64 discrete solution."""
    es = I.calcite_post_2d(128, 48, 40.0, 24.0, 10.0)
    prm = tight(I.make_params(es.shape, Pe=1.0, Da=0.5, L=20.0, method="ivos", Vm=0.5), precision=1)
    compare(V, es, prm, [0.25] * 4, 1e-9, init=c_start(es, prm))


@pytest.mark.parametrize("precision", [0, 1])
def test_production_tolerance_bound(V, precision):
    """At the production tolerances (p, u: 1e-8; c: 1e-10) the FP64 and mixed
    paths stay within 1e-5 relative L2 of the oracle's exact solves on every
    field (measured bound; solver-tolerance limited)."""
    es = I.calcite_post_2d(128, 48, 40.0, 24.0, 10.0)
    prm = I.make_params(es.shape, Pe=1.0, Da=0.5, L=20.0, method="ivos", Vm=0.5, precision=precision)
    errs, stats = compare(V, es, prm, [0.25] * 4, 1e-5, init=c_start(es, prm))
    assert stats["res_p"] <= 1e-8 and stats["res_c"] <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_dominated_momentum(V, precision):
    """Small dt (2 d nu dt / dx^2 <= 30): the momentum solves take the
    diagonally preconditioned CG path; same bar as the multigrid path."""
    es = I.sphere_rock_3d((16, 18, 34), seed=2, median_r=3.0, sigma=0.3, target_porosity=0.5,
                          start_solid=0.6, band=2, margin=3.0)
    prm = tight(I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=2.0), precision=precision)
    assert 2 * 3 * prm["nu"] * 0.005 <= 30
    compare(V, es, prm, [0.005] * 3, 1e-9, init=c_start(es, prm))


@pytest.mark.parametrize("precision,dt", [(0, 0.2), (1, 0.2), (1, 0.005)])
def test_graph_mode_equals_eager(V, precision, dt):
    """The step replayed as one CUDA graph (device-side refinement and
    Krylov loops) gives exactly the fields of the eager launch sequence."""
    es = I.sphere_rock_3d((14, 18, 30), seed=4, median_r=3.0, sigma=0.3, target_porosity=0.5,
                          start_solid=0.6, band=2, margin=3.0)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.3, precision=precision)
    init = c_start(es, prm)
    out = {}
    try:
        for mode in (0, 1):
            V.vos_set_launch_mode(mode)
            got, stats = run_gpu(V, es, prm, [dt] * 3, init=init)
            out[mode] = (got, stats)
    finally:
        V.vos_set_launch_mode(1)
    for n in ("eps", "c", "u", "v", "w", "p", "R", "Rf"):
        assert np.array_equal(out[0][0][n], out[1][0][n]), n
    assert out[0][1]["iters_p"] == out[1][1]["iters_p"]
    assert out[0][1]["iters_u"] == out[1][1]["iters_u"]


@pytest.mark.parametrize("shape3", [False, True])
def test_inertia_term_fp64(V, shape3):
    """Inertia term of Eq. momentumDBS kept (inertia = 1) at Re = Pe/Sc = 10,
    where it moves the flow: FP64 parity with the oracle's explicit van Leer
    form, 2D calcite post and 3D rock, iVoS."""
    if shape3:
        es = I.sphere_rock_3d((14, 16, 30), seed=6, median_r=3.0, sigma=0.3, target_porosity=0.5,
                              start_solid=0.6, band=2, margin=3.0)
        kw = dict(L=6.0)
    else:
        es = I.calcite_post_2d(96, 32, 30.0, 16.0, 8.0)
        kw = dict(L=16.0)
    prm = tight(I.make_params(es.shape, Pe=10.0, Da=1.0, method="ivos", Vm=0.2, Sc=1.0, inertia=1, **kw))
    compare(V, es, prm, [0.1] * 4, 1e-9, init=c_start(es, prm))
    # the term matters at this Reynolds number: the flow without it differs
    st1 = O.init_state(es, prm)
    p0 = dict(prm, inertia=0)
    st0 = O.init_state(es, p0)
    for _ in range(2):
        st1, _ = O.step(st1, 0.1, prm)
        st0, _ = O.step(st0, 0.1, p0)
    assert rel_l2(st1["u"][0], st0["u"][0]) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_warm_started_solves_same_solution(V, precision):
    """Starting the pressure correction from the previous step's correction
    and the momentum solves from 2 u^n - u^{n-1} (VOS_PRECOND_P_WARM |
    VOS_PRECOND_U_EXTRAP) changes the iteration counts only: the fields stay
    within the FP64 parity bar of the oracle, graph and eager launches alike."""
    es = I.sphere_rock_3d((14, 18, 30), seed=4, median_r=3.0, sigma=0.3, target_porosity=0.5,
                          start_solid=0.6, band=2, margin=3.0)
    prm = tight(I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.3,
                              precond=V.PRECOND_P_WARM | V.PRECOND_U_EXTRAP), precision=precision)
    compare(V, es, prm, [0.05] * 4, 1e-9, init=c_start(es, prm))
    try:
        V.vos_set_launch_mode(0)
        compare(V, es, prm, [0.05] * 4, 1e-9, init=c_start(es, prm))
    finally:
        V.vos_set_launch_mode(1)
