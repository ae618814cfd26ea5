"""Floating-cluster deflation of the pressure solve on the GPU.

The deflation is a preconditioner term: it must leave the converged step
unchanged (parity with the FP64 oracle on a rock with pore pockets), cut the
pressure iterations on such a rock, and follow the geometry when eps is set
through vos_set_fields (new labels, new captured graph).
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


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def pocket_rock(shape, seed, n):
    """Overlapping-sphere rock with n isolated pores: a 6x6x6 solid block
    with a 2x2x2 pore pocket at its centre, planted at random places that do
    not overlap (away from the outlet column).  Each pocket and its ring of
    solid cells touch the pore network only through solid cells."""
    es = I.sphere_rock_3d(shape, seed=seed, median_r=3.0, sigma=0.3, target_porosity=0.45,
                          start_solid=0.6, band=2, margin=3.0)
    rng = np.random.default_rng(seed)
    nz, ny, nx = es.shape
    used = np.zeros(es.shape, dtype=bool)
    placed = 0
    for _ in range(5000):
        k, j, i = int(rng.integers(0, nz - 5)), int(rng.integers(0, ny - 5)), int(rng.integers(0, nx - 7))
        if used[k:k + 6, j:j + 6, i:i + 6].any():
            continue
        es[k:k + 6, j:j + 6, i:i + 6] = 1.0
        es[k + 2:k + 4, j + 2:j + 4, i + 2:i + 4] = 0.0
        used[max(k - 1, 0):k + 7, max(j - 1, 0):j + 7, max(i - 1, 0):i + 7] = True
        placed += 1
        if placed == n:
            break
    assert placed == n
    return es


def clusters(V, es, prm):
    _, k, m = V.vos_floating_clusters(np.maximum(1.0 - es, prm["eps_min"]), prm)
    return k, m


def run(V, es, prm, dts, init):
    h = V.vos_create(es, prm)
    try:
        V.vos_set_fields(h, **init)
        for dt in dts:
            assert V.vos_step(h, dt) == 0, V.vos_get_stats(h)
            yield V.vos_get_stats(h)
        yield V.vos_fields(h)
    finally:
        V.vos_destroy(h)


def c_start(es, prm):
    nz, ny, nx = es.shape
    x = (np.arange(nx) + 0.5) / nx
    return {"c": np.broadcast_to(prm["c_in"] * (1.0 - 0.5 * x), es.shape).copy()}


def test_pocket_rock_fp64_parity(V):
    """With pockets deflated, the FP64 step still matches the oracle."""
    es = pocket_rock((20, 22, 38), seed=5, n=4)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.2)
    prm.update(p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000, precision=0)
    k, _ = clusters(V, es, prm)
    assert k >= 4
    init = c_start(es, prm)
    st = O.init_state(es, prm)
    st["c"] = init["c"].copy()
    dts = [0.2] * 3
    for dt in dts:
        st, _ = O.step(st, dt, prm)
    *_, got = run(V, es, prm, dts, init)
    ref = dict(eps=st["eps"], c=st["c"], p=st["p"], R=st["R"], Rf=st["Rf"], u=st["u"][0], v=st["u"][1], w=st["u"][2])
    errs = {n: rel_l2(got[n], ref[n]) for n in ref}
    assert max(errs.values()) <= 1e-9, errs


@pytest.mark.parametrize("precision", [0, 1])
def test_deflation_cuts_pressure_iterations(V, precision):
    """Same rock, same steps, with and without deflation: the fields agree
    to the solve tolerance and the pressure solve needs fewer iterations."""
    es = pocket_rock((28, 30, 48), seed=6, n=8)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.2, precision=precision)
    k, _ = clusters(V, es, prm)
    assert k >= 8
    init = c_start(es, prm)
    out = {}
    for flag in (0, V.PRECOND_NO_DEFLATION):
        p = dict(prm, precond=flag)
        res = list(run(V, es, p, [0.2] * 3, init))
        out[flag] = (sum(s["iters_p"] for s in res[:-1]), res[-1])
    it_d, f_d = out[0]
    it_n, f_n = out[V.PRECOND_NO_DEFLATION]
    assert it_d < it_n, (it_d, it_n)
    for n in ("u", "v", "w", "c"):
        assert rel_l2(f_d[n], f_n[n]) <= 1e-5, n


def test_set_fields_eps_relabels(V):
    """A handle created on one geometry and given another through
    vos_set_fields steps exactly like a handle created on the second one
    (labels recomputed, graph captured again)."""
    es1 = I.sphere_rock_3d((18, 20, 34), seed=8, median_r=3.0, sigma=0.3, target_porosity=0.5,
                           start_solid=0.6, band=2, margin=3.0)
    es2 = pocket_rock((18, 20, 34), seed=9, n=3)
    prm = I.make_params(es2.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.2, precision=1)
    assert clusters(V, es2, prm)[0] >= 3
    ha = V.vos_create(es1, prm)
    hb = V.vos_create(es2, prm)
    try:
        assert V.vos_step(ha, 0.2) == 0  # captures a graph for geometry 1
        V.vos_set_fields(ha, **V.vos_fields(hb))
        for _ in range(2):
            assert V.vos_step(ha, 0.2) == 0
            assert V.vos_step(hb, 0.2) == 0
        fa, fb = V.vos_fields(ha), V.vos_fields(hb)
        for n in ("eps", "c", "u", "v", "w", "p", "R", "Rf"):
            assert np.array_equal(fa[n], fb[n]), n
        assert V.vos_get_stats(ha)["iters_p"] == V.vos_get_stats(hb)["iters_p"]
    finally:
        V.vos_destroy(ha)
        V.vos_destroy(hb)
