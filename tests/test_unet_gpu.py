"""Tensor-core (tcgen05) kernels of the learned preconditioner against the
FP64 U-Net oracle.

Operands are BF16 on the GPU; the oracle takes the same BF16 values in
FP64, so an FP32-accumulated result differs from it only by FP32 rounding of
the sum (<= K * 2^-24 relative for K <= 27 * 96 products): the bar is 1e-5
relative L2 and 2e-5 relative max.  BF16 outputs are compared to the
oracle's value rounded to BF16 within one BF16 step.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07019_gb300 import build_lib, vos
    build_lib.build()
    vos.load_library()
    return torch, vos


def _bf16_dev(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda().contiguous()


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape,cin,cout", [
    ((5, 7, 9), 8, 16), ((4, 6, 10), 16, 16), ((6, 5, 11), 16, 32), ((3, 8, 8), 32, 64),
    ((4, 4, 12), 96, 32), ((5, 6, 7), 48, 16), ((4, 4, 8), 64, 64), ((3, 5, 9), 16, 48),
    ((2, 3, 40), 32, 96), ((16, 16, 16), 16, 16)])
def test_conv3d_fp32_out(env, shape, cin, cout):
    torch, V = env
    g = np.random.default_rng(cin * 1000 + cout)
    nv = int(np.prod(shape))
    xd = _bf16_dev(torch, g.standard_normal((nv, cin)))
    wd = _bf16_dev(torch, g.standard_normal((cout, 27, cin)) * 0.2)
    bd = torch.tensor(g.standard_normal(cout), dtype=torch.float32, device="cuda")
    y = torch.empty((nv, cout), dtype=torch.float32, device="cuda")
    V.vos_conv3d_bf16(xd, shape, cin, wd, bd, cout, y_f32=y)
    x = _f64(xd).reshape(shape + (cin,))
    W = _f64(wd).reshape(cout, 3, 3, 3, cin)
    ref = U.conv3(x, W, bd.cpu().numpy().astype(np.float64)).reshape(nv, cout)
    got = y.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-5, rel
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_conv3d_bf16_relu_out(env):
    torch, V = env
    g = np.random.default_rng(3)
    shape, cin, cout = (6, 9, 13), 16, 32
    nv = int(np.prod(shape))
    xd = _bf16_dev(torch, g.standard_normal((nv, cin)))
    wd = _bf16_dev(torch, g.standard_normal((cout, 27, cin)) * 0.2)
    bd = torch.tensor(g.standard_normal(cout), dtype=torch.float32, device="cuda")
    yb = torch.empty((nv, cout), dtype=torch.bfloat16, device="cuda")
    yf = torch.empty((nv, cout), dtype=torch.float32, device="cuda")
    V.vos_conv3d_bf16(xd, shape, cin, wd, bd, cout, relu=True, y_f32=yf, y_bf16=yb)
    ref = np.maximum(U.conv3(_f64(xd).reshape(shape + (cin,)), _f64(wd).reshape(cout, 3, 3, 3, cin),
                             bd.cpu().numpy().astype(np.float64)), 0.0).reshape(nv, cout)
    got_f = yf.cpu().numpy().astype(np.float64)
    assert (got_f >= 0).all()
    assert np.linalg.norm(got_f - ref) <= 1e-5 * np.linalg.norm(ref)
    # the BF16 output is the FP32 result rounded to nearest even
    np.testing.assert_array_equal(_f64(yb), U.bf16(got_f))
    step = np.abs(U.bf16(ref)) * 2.0 ** -7 + 1e-30
    assert (np.abs(_f64(yb) - U.bf16(ref)) <= step).all()


def test_conv3d_rejects_bad_shapes(env):
    torch, V = env
    x = torch.zeros((64, 12), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((16, 27, 12), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((64, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VosError):
        V.vos_conv3d_bf16(x, (4, 4, 4), 12, w, None, 16, y_f32=y)
