"""Batched micromodels (vos_batch_*): several instances of uneven sizes and
parameters stepped together on their own streams give exactly the results
of stepping each one alone (the kernels and reductions are deterministic),
and agree with the CPU oracle."""
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


def _cases():
    out = []
    for k, (nx, ny, Pe, Da, meth) in enumerate([(96, 40, 3.0, 0.5, "ivos"), (61, 77, 40.0, 5.0, "ivos"),
                                                 (130, 33, 1.5, 0.05, "psi_prime"), (70, 70, 10.0, 1.0, "psi")]):
        es = I.disc_micromodel_2d(nx, ny, seed=100 + k, rmin=3, rmax=8, target_porosity=0.7)
        prm = I.make_params(es.shape, Pe=Pe, Da=Da, L=10.0, method=meth, Vm=0.3, precision=k % 2,
                            p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000)
        out.append((es, prm))
    return out


def test_batch_equals_single_runs_and_oracle(V):
    cases = _cases()
    dts = [0.2, 0.15, 0.25, 0.2]
    b = V.vos_batch_create([c[0] for c in cases], [c[1] for c in cases], nthreads=3)
    try:
        for _ in range(3):
            assert V.vos_batch_step(b, dts) == 0
        got = [V.vos_fields(h) for h in b.handles]
    finally:
        V.vos_batch_destroy(b)
    for (es, prm), dt, g in zip(cases, dts, got):
        h = V.vos_create(es, prm)
        try:
            for _ in range(3):
                V.vos_step(h, dt)
            ref = V.vos_fields(h)
        finally:
            V.vos_destroy(h)
        for n in ("eps", "c", "u", "v", "p", "R", "Rf"):
            assert np.array_equal(g[n], ref[n]), n
        st, _ = O.run(es, prm, [dt] * 3)
        for n, r in (("eps", st["eps"]), ("c", st["c"]), ("u", st["u"][0]), ("p", st["p"])):
            err = np.linalg.norm(g[n] - r) / max(np.linalg.norm(r), 1e-300)
            assert err <= 1e-9, (n, err)


def test_batch_rejects_bad_dt(V):
    es, prm = _cases()[0]
    b = V.vos_batch_create([es], [prm])
    try:
        with pytest.raises(V.VosError):
            V.vos_batch_step(b, [0.0])
    finally:
        V.vos_batch_destroy(b)
