"""Quasi-static steps (flow_subiters > 1; App. A, App. B) on the GPU against
the oracle: a fixed number of sub-iterations (qs_rtol = 0) gives the same
fields as the oracle's loop to the FP64 parity bar; converged steps reach
the same quasi-static state; and the calcite-post channel runs at the
paper's time-step rule (App. D: the largest change of eps per step is
0.005)."""
import numpy as np
import pytest

from oracle import vos_oracle as O
from paper_2204_07019_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07019_gb300 import build_lib, vos
    build_lib.build()
    vos.load_library()
    return vos


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def _compare(V, es, prm, dts, tol, c0=None):
    st = O.init_state(es, prm)
    if c0 is not None:
        st["c"] = c0.copy()
    ostats = []
    for dt in dts:
        st, s = O.step(st, dt, prm)
        ostats.append(s)
    h = V.vos_create(es, prm)
    try:
        if c0 is not None:
            V.vos_set_fields(h, c=c0)
        for dt in dts:
            V.vos_step(h, dt)
        got = V.vos_fields(h)
        gs = V.vos_get_stats(h)
    finally:
        V.vos_destroy(h)
    ref = dict(eps=st["eps"], c=st["c"], p=st["p"], u=st["u"][0], v=st["u"][1], R=st["R"], Rf=st["Rf"])
    errs = {n: _rel(got[n], r) for n, r in ref.items()}
    assert all(e <= tol for e in errs.values()), errs
    return gs, ostats[-1]


@pytest.mark.parametrize("method,precision", [("ivos", 0), ("psi_prime", 0), ("ivos", 1)])
def test_five_subiterations_match_oracle(V, method, precision):
    es = I.calcite_post_2d(128, 48, 40.0, 24.0, 10.0)
    prm = I.make_params(es.shape, Pe=1.0, Da=0.5, L=20.0, method=method, Vm=0.5, precision=precision,
                        p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000,
                        flow_subiters=5, qs_rtol=0.0, qs_dtau=0.2)
    nz, ny, nx = es.shape
    x = (np.arange(nx) + 0.5) / nx
    c0 = np.broadcast_to(1.0 - 0.5 * x, es.shape).copy()
    gs, os_ = _compare(V, es, prm, [1.0, 1.0], 1e-9, c0=c0)
    assert gs["qs_iters"] == 5 == os_["qs_iters"]
    for k in ("qs_du", "qs_dp", "qs_dc"):
        assert gs[k] == pytest.approx(os_[k], rel=1e-6, abs=1e-14), k


def test_converged_quasi_static_state_matches_oracle(V):
    """Smooth porous field (no solid cells), iterated to qs_rtol = 1e-11 on
    both sides: the same quasi-static flow and concentration."""
    ny, nx = 10, 30
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    eps = 0.75 + 0.2 * np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    es = (1.0 - eps)[None]
    prm = I.make_params(es.shape, Pe=2.0, Da=2.0, L=8, method="ivos", Vm=0.0, Sc=1.0, k0=0.5,
                        p_rtol=1e-12, u_rtol=1e-12, c_rtol=1e-12, max_iter=4000,
                        flow_subiters=3000, qs_rtol=1e-11, qs_dtau=0.5)
    gs, os_ = _compare(V, es, prm, [1.0], 1e-8)
    assert gs["status"] == 0 and gs["qs_iters"] < 3000
    assert max(gs["qs_du"], gs["qs_dp"], gs["qs_dc"]) <= 1e-11


def test_calcite_post_at_the_paper_time_step_rule(V):
    """The calcite-post channel (256 x 64, Pe = 1, Da = 0.1, iVoS) in
    quasi-static steps whose length follows App. D: dt = 0.005 / max|Vm R|,
    so no cell's eps moves by more than 0.005 in a step, and the solid mass
    balance (Eq. mbs) holds over each step."""
    es = I.calcite_post_2d()
    prm = I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method="ivos", flow_subiters=60, qs_rtol=0.0,
                        qs_dtau=0.25)
    h = V.vos_create(es, prm)
    try:
        V.vos_step(h, 1.0)  # from rest: the reactant enters, R becomes positive
        for _ in range(3):
            dt = V.vos_suggest_dt(h, 1e30, 0.005)
            assert np.isfinite(dt) and dt > 1.0
            f0 = V.vos_fields(h, ("eps", "R"))
            V.vos_step(h, dt)
            s = V.vos_get_stats(h)
            f1 = V.vos_fields(h, ("eps",))
            deps = f1["eps"] - f0["eps"]
            assert np.abs(deps).max() <= 0.005 * (1 + 1e-12)
            assert np.abs(deps).max() >= 0.005 * (1 - 1e-9) or s["clamp_excess"] > 0
            lhs = deps.sum() * prm["dx"] ** 2
            rhs = dt * prm["Vm"] * f0["R"].sum() * prm["dx"] ** 2 - s["clamp_excess"]
            assert abs(lhs - rhs) <= 1e-10 * max(abs(rhs), 1e-30)
            assert s["qs_iters"] == 60 and np.isfinite(s["qs_du"])
    finally:
        V.vos_destroy(h)
