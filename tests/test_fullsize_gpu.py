"""Checks at the benchmark sizes.

* 256^3 rock (the benchmark workload, mixed precision at the production
  tolerances): the oracle cannot solve 16.7M-unknown 3D systems, so the
  checks are the ones that hold at any size -- the S1 update cell by cell
  (Eq. mbs), the iVoS rates recomputed by the oracle's functions from the
  GPU's eps^{n+1}, c^n and c^{n+1} (Eq. RfiVoS), the conservative term
  summing to zero, the reactant balance over the step, the discrete
  divergence after projection, and the solver residuals.
* 1024 x 512 disc micromodel: one FP64 step element by element against the
  oracle's direct solves.
"""
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


def _state_from(f):
    st = dict(eps=f["eps"], c=f["c"], p=f["p"], R=f["R"], Rf=f["Rf"], u=[f["u"], f["v"], f.get("w", np.zeros((0,)))])
    return st


def test_rock256_properties(V):
    es = I.sphere_rock_3d(256, seed=0)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=24.0, method="ivos", precision=1,
                        p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=2000)
    h = V.vos_create(es, prm)
    try:
        nz, ny, nx = es.shape
        x = (np.arange(nx) + 0.5) / nx
        V.vos_set_fields(h, c=np.broadcast_to(1.0 - 0.5 * x, es.shape).copy())
        V.vos_step(h, 0.5)
        dt = V.vos_suggest_dt(h, 0.5, 0.005)
        V.vos_step(h, dt)
        f0 = V.vos_fields(h)
        assert V.vos_step(h, dt) == 0
        f1 = V.vos_fields(h)
        s = V.vos_get_stats(h)
    finally:
        V.vos_destroy(h)
    assert s["res_p"] <= 1e-8 and max(s["res_u"]) <= 1e-8 and s["res_c"] <= 1e-10
    # S1 (Eq. mbs), cell by cell
    e_ref = np.clip(f0["eps"] + dt * prm["Vm"] * f0["R"], prm["eps_min"], 1.0)
    assert np.max(np.abs(f1["eps"] - e_ref)) <= 1e-15
    # iVoS rates from the GPU's eps^{n+1}, c^n, c^{n+1} (oracle functions)
    faces = O.ivos_faces(f1["eps"], f0["c"], prm)
    R, Rf = O.ivos_rates(f1["eps"], f1["c"], faces, prm)
    scale = prm["kc"] * prm["c_in"] / prm["dx"] * np.sqrt(R.size)
    assert np.linalg.norm(f1["R"] - R) <= 1e-12 * scale
    assert np.linalg.norm(f1["Rf"] - Rf) <= 1e-12 * scale
    assert abs(f1["R"].sum() - f1["Rf"].sum()) <= 1e-12 * np.abs(f1["Rf"]).sum()
    # reactant balance over the step (concentration solved to 1e-10)
    D, dx = prm["D"], prm["dx"]
    inflow = np.sum(f1["u"][..., 0] * prm["c_in"]) + np.sum(2 * D * f1["eps"][..., 0] * (prm["c_in"] - f1["c"][..., 0]) / dx)
    outflow = np.sum(f1["u"][..., -1] * f0["c"][..., -1])
    lhs = np.sum(f1["eps"] * f1["c"]) - np.sum(f0["eps"] * f0["c"])
    rhs = dt * (inflow - outflow - np.sum(f1["Rf"]))
    assert abs(lhs - rhs) <= 1e-6 * (abs(dt * inflow) + abs(dt * outflow) + 1e-300)
    # projection: divergence-free velocity (rho_s = rho), relative to the inflow rate
    st = _state_from(f1)
    div = O.divergence(st["u"], prm)
    assert np.abs(div).max() <= 1e-6 * prm["u_in"] / dx


def test_micromodel_1024x512_one_step_fp64(V):
    es = I.disc_micromodel_2d(1024, 512, seed=0)
    prm = I.make_params(es.shape, Pe=100.0, Da=1.0, L=40.0, method="ivos", precision=0, Vm=0.5,
                        p_rtol=1e-10, u_rtol=1e-10, c_rtol=1e-10, max_iter=4000)
    nz, ny, nx = es.shape
    x = (np.arange(nx) + 0.5) / nx
    c0 = np.broadcast_to(1.0 - 0.5 * x, es.shape).copy()
    h = V.vos_create(es, prm)
    try:
        V.vos_set_fields(h, c=c0)
        assert V.vos_step(h, 0.2) == 0
        got = V.vos_fields(h)
    finally:
        V.vos_destroy(h)
    st = O.init_state(es, prm)
    st["c"] = c0.copy()
    st, _ = O.step(st, 0.2, prm)
    ref = dict(eps=st["eps"], c=st["c"], p=st["p"], u=st["u"][0], v=st["u"][1], R=st["R"], Rf=st["Rf"])
    for n, r in ref.items():
        err = np.linalg.norm(got[n] - r) / max(np.linalg.norm(r), 1e-300)
        assert err <= 1e-9, (n, err)
