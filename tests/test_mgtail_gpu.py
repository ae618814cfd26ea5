"""The cluster-resident coarse multigrid cycle (one launch of one 8-CTA
thread-block cluster for every level of at most 32^3 cells, data in
distributed shared memory) against the one-launch-per-operation cycle:
the same arithmetic per cell in the same order, so whole time steps give
bit-identical fields and iteration counts, for symmetric (PCG) and
non-symmetric (BiCGStab, iVoS transport) hierarchies, FP32 and FP64, 2D and
3D, graph and eager launches."""
import numpy as np
import pytest

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


def _run(V, es, prm, dts, tail, graphs=1, count_tail=False):
    V.vos_set_coarse_cycle(tail)
    V.vos_set_launch_mode(graphs)
    try:
        h = V.vos_create(es, prm)
    finally:
        V.vos_set_coarse_cycle(0)
    try:
        nz, ny, nx = es.shape
        x = (np.arange(nx) + 0.5) / nx
        V.vos_set_fields(h, c=np.broadcast_to(1.0 - 0.5 * x, es.shape).copy())
        its = []
        ntail = None
        for k, dt in enumerate(dts):
            if count_tail and k == len(dts) - 1:
                V.vos_prof_reset()
                V.vos_prof_enable("mg_tail")
            V.vos_step(h, dt)
            if count_tail and k == len(dts) - 1:
                rep = V.vos_prof_report()
                V.vos_prof_enable(None)
                V.vos_prof_reset()
                ntail = sum(v[0] for k2, v in rep.items() if k2.startswith("mg_tail"))
            s = V.vos_get_stats(h)
            its.append((tuple(s["iters_u"]), s["iters_p"], s["iters_c"]))
        return V.vos_fields(h), its, ntail
    finally:
        V.vos_set_launch_mode(1)
        V.vos_destroy(h)


CASES = {
    "rock_ivos_mixed": (lambda: I.sphere_rock_3d((40, 44, 66), seed=3, median_r=3.5, sigma=0.3,
                                                 target_porosity=0.4, start_solid=0.6, band=2, margin=3.0),
                        dict(Pe=10.0, Da=1.0, L=7.0, method="ivos", Vm=0.3, precision=1), 0.01),
    "rock_psi_fp64": (lambda: I.sphere_rock_3d((34, 30, 50), seed=7, median_r=3.0, sigma=0.3,
                                               target_porosity=0.45, start_solid=0.6, band=2, margin=3.0),
                      dict(Pe=5.0, Da=0.5, L=6.0, method="psi", Vm=0.3, precision=0), 0.01),
    "micromodel_ivos_mixed": (lambda: I.disc_micromodel_2d(300, 170, seed=2, rmin=5, rmax=12,
                                                           target_porosity=0.6),
                              dict(Pe=20.0, Da=2.0, L=16.0, method="ivos", Vm=0.3, precision=1), 0.05),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("graphs", [1, 0])
def test_coarse_cycle_bit_identical(V, case, graphs):
    make, kw, dt = CASES[case]
    es = make()
    prm = I.make_params(es.shape, **kw)
    dts = [dt] * 3
    on, its_on, ntail = _run(V, es, prm, dts, 1, graphs, count_tail=True)
    off, its_off, _ = _run(V, es, prm, dts, 0, graphs)
    assert ntail and ntail > 0, "the cluster-resident cycle did not run"
    assert its_on == its_off
    for n in on:
        assert np.array_equal(on[n], off[n]), n
