"""The allocation-free time-step limit (vos_suggest_dt_noalloc).

Some callers cannot let a library allocate device memory (hosts that own
the whole GPU pool, or loops that must not trigger the synchronisation of a
cudaMalloc/cudaFree).  For them the library offers one entry point whose
scratch is a fixed device array.  This test calls it through the C ABI on
fields a simulation holds on the device and checks it against the
allocating vos_suggest_dt on the same fields, twice in a row (the shared
scratch keeps the previous call's contents, so a second call must not see
them), and checks that a grid above its fixed capacity is refused.

The file is named so that pytest collects it last.
"""
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


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_noalloc_matches_suggest_dt_twice(V, case):
    if case == "2d":
        es = I.calcite_post_2d(200, 48, 60.0, 24.0, 10.0)
        prm = I.make_params(es.shape, Pe=1.0, Da=1.0, L=20.0, method="ivos", Vm=0.5)
    else:
        es = I.sphere_rock_3d((20, 24, 40), seed=5, median_r=3.0, sigma=0.3, target_porosity=0.5,
                              start_solid=0.6, band=2, margin=3.0)
        prm = I.make_params(es.shape, Pe=5.0, Da=1.0, L=6.0, method="ivos", Vm=0.5)
    h = V.vos_create(es, prm)
    try:
        nz, ny, nx = es.shape
        x = (np.arange(nx) + 0.5) / nx
        V.vos_set_fields(h, c=np.broadcast_to(1.0 - 0.5 * x, es.shape).copy())
        for _ in range(2):
            V.vos_step(h, 0.2)
        f = V.vos_device_fields_get(h)
        ref = V.vos_suggest_dt(h, 0.5, 0.005)
        for _ in range(2):
            got = V.vos_suggest_dt_noalloc(prm, f["eps"], f["u"], f["v"], f["w"], f["R"], 0.5, 0.005)
            assert np.isfinite(got) and got > 0
            assert abs(got - ref) <= 1e-9 * abs(ref)
        # the Delta-eps limit alone (tiny cfl makes the other term irrelevant)
        ref2 = V.vos_suggest_dt(h, 1e6, 1e-4)
        got2 = V.vos_suggest_dt_noalloc(prm, f["eps"], f["u"], f["v"], f["w"], f["R"], 1e6, 1e-4)
        assert got2 == ref2 or abs(got2 - ref2) <= 1e-9 * abs(ref2)
    finally:
        V.vos_destroy(h)


def test_noalloc_single_row_without_v_and_on_a_side_stream(V):
    """ny == 1: every v face is a wall face, so v may be NULL; the result
    equals vos_suggest_dt (which reads the zero wall faces).  Also run on a
    non-default torch stream, twice in a row."""
    import torch
    es = np.zeros((1, 1, 64))
    es[0, 0, 20:30] = 0.7
    prm = I.make_params(es.shape, Pe=1.0, Da=1.0, L=8.0, method="ivos", Vm=0.5, wall_mask=0)
    h = V.vos_create(es, prm)
    try:
        V.vos_set_fields(h, c=np.linspace(1.0, 0.2, 64).reshape(es.shape))
        for _ in range(2):
            V.vos_step(h, 0.2)
        f = V.vos_device_fields_get(h)
        ref = V.vos_suggest_dt(h, 0.5, 0.005)
        side = torch.cuda.Stream()
        torch.cuda.synchronize()
        for _ in range(2):
            got = V.vos_suggest_dt_noalloc(prm, f["eps"], f["u"], None, None, f["R"], 0.5, 0.005, stream=side)
            assert np.isfinite(got) and got > 0
            assert abs(got - ref) <= 1e-9 * abs(ref)
    finally:
        V.vos_destroy(h)


def test_noalloc_rejects_grids_beyond_its_scratch(V):
    prm = I.make_params((257, 256, 256), Pe=1.0, Da=1.0, L=1.0)
    with pytest.raises(V.VosError) as ei:
        V.vos_suggest_dt_noalloc(prm, 1, 1, 1, 1, 1)
    assert ei.value.code == V.VOS_EINVAL
    assert "16777216" in str(ei.value)
