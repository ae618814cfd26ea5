"""Fused FP32 Krylov forms of the mixed path.  The two-kernel diagonally
preconditioned CG (the momentum solves at small 2 d nu dt / dx^2: direction
update fused with the matrix-vector product, x/r update fused with the
preconditioner and the dot products) gives the four-kernel form's results
bit for bit.  The MG-PCG form fused with the V-cycle's first and last fine
sweeps (pressure) agrees with the separate kernels to the solve tolerance.
Both match the FP64 oracle.  Shapes cover the four-cells-per-thread kernel (v, w with nx
a multiple of 4), the one-cell kernel (u: nx + 1 faces; nx = 30) and 2D
boxes; both launch modes (graph replay, eager)."""
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


def _geometry(shape):
    if shape[0] == 1:
        return I.disc_micromodel_2d(shape[2], shape[1], seed=4, rmin=5, rmax=10, target_porosity=0.6)
    return I.sphere_rock_3d(shape, seed=7, median_r=3.0, sigma=0.3, target_porosity=0.45, start_solid=0.6, band=2,
                            margin=3.0)


def _run(V, es, prm, dts, fused, graphs):
    V.vos_set_fused_pcg(fused)
    V.vos_set_launch_mode(graphs)
    try:
        h = V.vos_create(es, prm)
        try:
            its = []
            for dt in dts:
                assert V.vos_step(h, dt) == 0
                s = V.vos_get_stats(h)
                its.append(sum(s["iters_u"]))
                assert max(s["res_u"]) <= prm["u_rtol"], s["res_u"]
            return V.vos_fields(h), its
        finally:
            V.vos_destroy(h)
    finally:
        V.vos_set_fused_pcg(V.FUSED_ALL)
        V.vos_set_launch_mode(1)


@pytest.mark.parametrize("shape", [(16, 20, 32), (10, 14, 30), (1, 48, 64)])
@pytest.mark.parametrize("graphs", [1, 0])
def test_fused_diag_pcg(V, shape, graphs):
    es = _geometry(shape)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.5, precision=1,
                        p_rtol=1e-11, u_rtol=1e-11, c_rtol=1e-11, max_iter=4000)
    prm["precond"] = int(prm.get("precond", 0)) | V.PRECOND_MOM_DIAG
    dts = [2e-3, 2e-3, 2e-3]  # 2 d nu dt / dx^2 = 7.2 (3D), 4.8 (2D): the diagonal regime
    # momentum: two kernels against four, the pressure form fixed
    f1, it1 = _run(V, es, prm, dts, V.FUSED_DIAG_PCG, graphs)
    f0, it0 = _run(V, es, prm, dts, 0, graphs)
    assert it1 == it0
    for n in f0:
        assert np.array_equal(f1[n], f0[n]), n
    # pressure: MG-PCG fused with the V-cycle sweeps, to the solve tolerance
    f3, _ = _run(V, es, prm, dts, V.FUSED_DIAG_PCG | V.FUSED_MG_PCG, graphs)
    for n in ("u", "v", "w", "p", "c", "eps"):
        if n == "w" and shape[0] == 1:
            continue
        ref = np.linalg.norm(f1[n])
        assert np.linalg.norm(f3[n] - f1[n]) <= 1e-9 * max(ref, 1e-300), n
    # and the FP64 oracle's exact solves
    st = O.init_state(es, prm)
    for dt in dts:
        st, _ = O.step(st, dt, prm)
    ref = dict(u=st["u"][0], v=st["u"][1], p=st["p"], c=st["c"])
    if shape[0] > 1:
        ref["w"] = st["u"][2]
    for f in (f1, f3):
        for n, r in ref.items():
            assert np.linalg.norm(f[n] - r) <= 1e-9 * max(np.linalg.norm(r), 1e-300), n


def test_fused_pcg_mask_checked(V):
    with pytest.raises(V.VosError):
        V.vos_set_fused_pcg(8)


@pytest.mark.parametrize("shape", [(16, 20, 32), (1, 48, 64)])
@pytest.mark.parametrize("graphs", [1, 0])
def test_df_residual(V, shape, graphs):
    """Refinement residual in double-FP32 after the first pass (symmetric
    solves to 1e-8): the solves reach their tolerance and the fields agree
    with the FP64-residual path and the FP64 oracle at that tolerance."""
    es = _geometry(shape)
    prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=6.0, method="ivos", Vm=0.5, precision=1,
                        p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=4000)
    dts = [0.05, 0.05, 0.05]
    f_df, it_df = _run(V, es, prm, dts, V.FUSED_ALL, graphs)
    f_64, it_64 = _run(V, es, prm, dts, V.FUSED_DIAG_PCG | V.FUSED_MG_PCG, graphs)
    for a, b in zip(it_df, it_64):
        assert abs(a - b) <= max(4, 0.1 * b), (it_df, it_64)
    st = O.init_state(es, prm)
    for dt in dts:
        st, _ = O.step(st, dt, prm)
    ref = dict(u=st["u"][0], v=st["u"][1], p=st["p"], c=st["c"])
    if shape[0] > 1:
        ref["w"] = st["u"][2]
    for n, r in ref.items():
        rn = max(np.linalg.norm(r), 1e-300)
        e_df = np.linalg.norm(f_df[n] - r) / rn
        e_64 = np.linalg.norm(f_64[n] - r) / rn
        assert e_df <= 2e-8 and np.linalg.norm(f_df[n] - f_64[n]) / rn <= 2e-8, (n, e_df, e_64)
