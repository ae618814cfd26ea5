"""Pins of the U-Net oracle (CPU).

Each operation is checked against something other than itself: the conv
against scipy.ndimage.correlate, backward passes against adjoint identities
and finite differences, the BF16 rounding against torch's bfloat16
conversion and hand-worked ties.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi
import scipy.sparse as sp

from oracle import unet_oracle as U


def rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3_matches_scipy_correlate():
    g = rng(1)
    x = g.standard_normal((5, 6, 7, 3))
    W = g.standard_normal((4, 3, 3, 3, 3))
    b = g.standard_normal(4)
    y = U.conv3(x, W, b)
    for o in range(4):
        ref = b[o] + sum(ndi.correlate(x[..., i], W[o, ..., i], mode="constant", cval=0.0) for i in range(3))
        np.testing.assert_allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_conv3_delta_kernel_is_identity_and_shift():
    x = rng(2).standard_normal((4, 5, 6, 2))
    W = np.zeros((2, 3, 3, 3, 2))
    W[0, 1, 1, 1, 0] = 1.0
    W[1, 1, 1, 2, 1] = 1.0  # reads x at +1 along x
    y = U.conv3(x, W, np.zeros(2))
    np.testing.assert_array_equal(y[..., 0], x[..., 0])
    np.testing.assert_array_equal(y[..., 1][:, :, :-1], x[..., 1][:, :, 1:])
    np.testing.assert_array_equal(y[..., 1][:, :, -1], 0.0)


def test_conv3_backward_adjoints():
    g = rng(3)
    x = g.standard_normal((4, 5, 6, 3))
    W = g.standard_normal((2, 3, 3, 3, 3))
    dy = g.standard_normal((4, 5, 6, 2))
    y0 = U.conv3(x, W, np.zeros(2))
    dx, dW, db = U.conv3_backward(x, W, dy)
    s = np.sum(y0 * dy)
    assert np.isclose(s, np.sum(x * dx), rtol=1e-12)   # linear in x
    assert np.isclose(s, np.sum(W * dW), rtol=1e-12)   # linear in W
    np.testing.assert_allclose(db, dy.reshape(-1, 2).sum(0), rtol=1e-12)


def test_pool_up_adjoints():
    g = rng(4)
    x = g.standard_normal((4, 6, 8, 3))
    yc = g.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(U.pool(x) * yc), np.sum(x * U.pool_backward(yc)), rtol=1e-12)
    assert np.isclose(np.sum(U.up(yc) * x), np.sum(yc * U.up_backward(x)), rtol=1e-12)
    np.testing.assert_allclose(U.pool(U.up(yc)), yc, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(U.pool(np.ones_like(x)), 1.0)


def _laplace(shape):
    """A small SPD operator on the box (7-point, Dirichlet) for the loss."""
    nz, ny, nx = shape
    def d1(n):
        return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = lambda n: sp.identity(n)
    return (sp.kron(sp.kron(d1(nz), I(ny)), I(nx)) + sp.kron(sp.kron(I(nz), d1(ny)), I(nx))
            + sp.kron(sp.kron(I(nz), I(ny)), d1(nx))).tocsr()


def _loss(P, r_hat, eps, A):
    z, _ = U.forward(P, r_hat, eps)
    return U.loss_and_grad_z(A, z, r_hat)[0]


def test_network_gradient_finite_differences():
    shape = (4, 8, 8)
    g = rng(5)
    P = U.init_params(7)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * g.standard_normal(P[k].shape)
    r_hat = U.normalise(g.standard_normal(shape))
    eps = g.uniform(1e-4, 1.0, shape)
    A = _laplace(shape)
    z, C = U.forward(P, r_hat, eps)
    L, dz = U.loss_and_grad_z(A, z, r_hat)
    G = U.backward(P, C, dz)
    h = 1e-6
    for key in ("enc1a.W", "enc2b.W", "enc3a.W", "enc3b.b", "dec2a.W", "dec1b.W", "head.W", "head.b"):
        flat = P[key].reshape(-1)
        for idx in g.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = _loss(P, r_hat, eps, A)
            flat[idx] = old - h
            lm = _loss(P, r_hat, eps, A)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (key, idx, fd, an)


def test_loss_gradient_finite_differences():
    shape = (3, 4, 5)
    g = rng(6)
    A = _laplace(shape)
    z = g.standard_normal(shape)
    r_hat = g.standard_normal(shape)
    L, dz = U.loss_and_grad_z(A, z, r_hat)
    res = A @ z.ravel() - r_hat.ravel()
    assert np.isclose(L, res @ res / (r_hat.ravel() @ r_hat.ravel()))
    h = 1e-6
    for idx in range(0, z.size, 7):
        zp = z.copy().reshape(-1)
        zp[idx] += h
        zm = z.copy().reshape(-1)
        zm[idx] -= h
        fd = (U.loss_and_grad_z(A, zp.reshape(shape), r_hat)[0] - U.loss_and_grad_z(A, zm.reshape(shape), r_hat)[0]) / (2 * h)
        assert abs(fd - dz.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding():
    # spacing of bfloat16 at 1 is 2^-7; ties go to the even mantissa
    assert U.bf16(1.0) == 1.0
    assert U.bf16(1.0 + 2.0 ** -8) == 1.0
    assert U.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert U.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert U.bf16(-2.5) == -2.5
    torch = pytest.importorskip("torch")
    x = rng(8).standard_normal(10000) * 10.0 ** rng(9).uniform(-6, 6, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.bf16(x), ref)


def test_bf16_emulation_close_to_fp64():
    shape = (4, 8, 8)
    g = rng(10)
    P = U.init_params(11)
    r_hat = U.normalise(g.standard_normal(shape))
    eps = g.uniform(1e-4, 1.0, shape)
    z64, _ = U.forward(P, r_hat, eps)
    z16, _ = U.forward(P, r_hat, eps, bf16_emulation=True)
    rel = np.linalg.norm(z16 - z64) / np.linalg.norm(z64)
    assert 0 < rel < 0.05
