"""Step diagnostics (S7), the time-step limit and the non-convergence path
on the GPU, against the oracle.

Two checks per step:
* exact reductions: the oracle's diagnostics and time-step limit evaluated
  on the GPU's own fields (before and after the step) equal what the GPU
  reduced (sums to 1e-12 relative, maxima to 1e-14: the GPU's quotient
  |u_f| / eps_f is within 2 ulp of the IEEE one);
* parity: an independent oracle run from the same state gives the same
  statistics within the field tolerance of the FP64 parity tests.
"""
import numpy as np
import pytest

from oracle import vos_oracle as O
from paper_2204_07019_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SUMS = ("porosity", "reactant", "sum_R", "sum_Rf", "q_in", "q_out", "flux_in", "flux_out")


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07019_gb300 import build_lib, vos
    build_lib.build()
    vos.load_library()
    return vos


def _tight(prm, precision=0):
    prm = dict(prm)
    prm.update(p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000, precision=precision)
    return prm


def _c_start(es, prm):
    nz, ny, nx = es.shape
    x = (np.arange(nx) + 0.5) / nx
    return np.broadcast_to(prm["c_in"] * (1.0 - 0.5 * x), es.shape).copy()


def _gpu_state(V, h, prm):
    f = V.vos_fields(h)
    u = [f["u"], f["v"], f.get("w", np.zeros((0,)))]
    return dict(eps=f["eps"], c=f["c"], p=f["p"], u=u, R=f["R"], Rf=f["Rf"])


def _case(name, method):
    if name == "calcite":
        es = I.calcite_post_2d()
        prm = I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method=method, Vm=0.5)
        return es, prm, [0.25] * 3
    es = I.sphere_rock_3d((19, 21, 37), seed=1, median_r=3.0, sigma=0.3, target_porosity=0.45,
                          start_solid=0.6, band=2, margin=3.0)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method=method, Vm=2.0)
    return es, prm, [0.2] * 3


@pytest.mark.parametrize("name,method,precision", [
    ("calcite", "ivos", 0), ("calcite", "psi", 0), ("calcite", "psi_prime", 0),
    ("rock", "ivos", 0), ("rock", "psi_prime", 0), ("rock", "ivos", 1)])
def test_step_stats_and_dt_against_oracle(V, name, method, precision):
    es, prm, dts = _case(name, method)
    prm = _tight(prm, precision)
    c0 = _c_start(es, prm)
    ost = O.init_state(es, prm)
    ost["c"] = c0.copy()
    h = V.vos_create(es, prm)
    try:
        V.vos_set_fields(h, c=c0)
        prev = _gpu_state(V, h, prm)
        for dt in dts:
            assert V.vos_step(h, dt) == 0
            s = V.vos_get_stats(h)
            new = _gpu_state(V, h, prm)
            # exact reductions on the GPU's own fields
            d = O.diagnostics(prev, new, prm)
            for k in SUMS:
                assert s[k] == pytest.approx(d[k], rel=1e-12, abs=1e-13 * abs(d["q_in"]) + 1e-300), k
            for k in ("umax", "rmax"):
                assert s[k] == pytest.approx(d[k], rel=1e-14, abs=0), k
            _, excess = O.solid_update(prev["eps"], prev["R"], dt, prm)
            assert abs(s["clamp_excess"] - excess) <= 1e-12 * np.sum(new["eps"]) * prm["dx"] ** prm["dim"]
            if method == "psi_prime":
                assert s["lambda"] == pytest.approx(O.vos_lambda(new["eps"], prm), rel=1e-13)
            elif method == "psi":
                assert s["lambda"] == prm["lam"]
            else:
                assert np.isnan(s["lambda"])
            for cfl, dem in ((0.5, 0.005), (1e6, 1e-4)):
                assert V.vos_suggest_dt(h, cfl, dem) == pytest.approx(O.suggest_dt(new, prm, cfl, dem),
                                                                      rel=1e-15)
            # parity with an independent oracle step
            ost, od = O.step(ost, dt, prm)
            for k in SUMS + ("umax", "rmax"):
                scale = abs(od[k]) if k not in ("sum_R", "sum_Rf") else max(abs(od["sum_Rf"]), 1e-300)
                assert abs(s[k] - od[k]) <= 1e-8 * max(scale, 1e-12), (k, s[k], od[k])
            if method == "psi_prime":
                assert s["lambda"] == pytest.approx(od["lam"], rel=1e-9)
            assert V.vos_suggest_dt(h, 0.5, 0.005) == pytest.approx(O.suggest_dt(ost, prm, 0.5, 0.005), rel=1e-8)
            # the flux terms close the reactant balance of the step
            before = np.sum(prev["eps"] * prev["c"]) * prm["dx"] ** prm["dim"]
            lhs = s["reactant"] - before
            rhs = dt * (s["flux_in"] - s["flux_out"] - prm["zeta"] * s["sum_Rf"])
            assert abs(lhs - rhs) <= 1e-8 * max(1.0, abs(before))
            prev = new
    finally:
        V.vos_destroy(h)


@pytest.mark.parametrize("graphs", [1, 0])
def test_max_iter_reports_nonconvergence_and_applies_step(V, graphs):
    """max_iter = 1 cannot reach the tolerances: vos_step returns
    VOS_ENOCONV, the stats carry the status and the step is still applied
    (eps updated, the velocity moved from its initial state, all finite)."""
    es = I.calcite_post_2d(96, 32, 30.0, 16.0, 8.0)
    prm = I.make_params(es.shape, Pe=1.0, Da=0.5, L=16.0, method="ivos", Vm=0.5, max_iter=1)
    try:
        V.vos_set_launch_mode(graphs)
        h = V.vos_create(es, prm)
        try:
            V.vos_set_fields(h, c=_c_start(es, prm))
            f0 = V.vos_fields(h)
            assert V.vos_step(h, 0.25) == V.VOS_ENOCONV
            assert "max_iter" in V.vos_last_error(h)
            s = V.vos_get_stats(h)
            assert s["status"] == V.VOS_ENOCONV and s["step"] == 1
            assert s["iters_p"] <= 1 * max(s["outer_p"], 1) + 1
            f1 = V.vos_fields(h)
            for n, a in f1.items():
                assert np.all(np.isfinite(a)), n
            assert not np.array_equal(f1["u"], f0["u"])
            assert not np.array_equal(f1["c"], f0["c"])
            # a later step with the same handle still runs
            assert V.vos_step(h, 0.25) == V.VOS_ENOCONV
        finally:
            V.vos_destroy(h)
    finally:
        V.vos_set_launch_mode(1)


@pytest.mark.parametrize("name,method", [("calcite", "ivos"), ("rock", "psi_prime")])
def test_upscaled_properties_against_oracle(V, name, method):
    """vos_upscaled equals the oracle's Sec. 2.5 properties evaluated on the
    GPU's own fields (FP64 sums, 1e-12)."""
    es, prm, dts = _case(name, method)
    prm = _tight(prm)
    h = V.vos_create(es, prm)
    try:
        V.vos_set_fields(h, c=_c_start(es, prm))
        for dt in dts:
            V.vos_step(h, dt)
        got = V.vos_upscaled(h)
        ref = O.upscaled(_gpu_state(V, h, prm), prm)
        for k, v in ref.items():
            assert got[k] == pytest.approx(v, rel=1e-12), k
        assert 0 < got["phi"] < 1 and got["K"] > 0 and got["a"] > 0 and got["alpha"] > 0
    finally:
        V.vos_destroy(h)


def test_upscaled_darcy_permeability_on_gpu(V):
    """Uniform eps0, free-slip sides, run to a steady state on the GPU: the
    measured K is the Kozeny-Carman k of Eq. perm (Sec. 2.5 definition)."""
    eps0, k0, nu = 0.6, 0.5, 0.7
    es = np.full((4, 6, 28), 1.0 - eps0)
    prm = _tight(I.make_params(es.shape, Pe=1, Da=0, L=1, method="psi", nu=nu, c_in=0.0, kc=0.0, k0=k0,
                               u_in=0.9, wall_mask=0))
    h = V.vos_create(es, prm)
    try:
        for _ in range(60):
            V.vos_step(h, 1.0)
        up = V.vos_upscaled(h)
        assert up["K"] == pytest.approx(k0 * eps0 ** 3 / (1 - eps0) ** 2, rel=1e-8)
        assert up["U_D"] == pytest.approx(0.9, rel=1e-14)
    finally:
        V.vos_destroy(h)
