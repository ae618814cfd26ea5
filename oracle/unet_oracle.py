"""FP64 CPU oracle of the learned pressure preconditioner (a 3-level U-Net).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA path.

The paper has no learned component: it mentions machine learning only as a
route to upscaling.  This network is the build's preconditioner for the
pressure correction (Eq. contDBS).  What it computes is fixed here, in plain
numpy, as the definition the CUDA kernels are checked against:

* Tensors are channels-last, shape (nz, ny, nx, C), float64.
* conv3 (3x3x3, zero padding, stride 1):
  y[v, o] = b[o] + sum over taps t = (dz, dy, dx) in {-1, 0, 1}^3 and input
  channels i of W[o, dz+1, dy+1, dx+1, i] x[v + t, i], with x = 0 outside the box.
  Each tap is one matrix product (a library primitive) of the shifted input
  with W[:, tap, :]^T.
* pool: 2x2x2 average (box sides even).  up: nearest-neighbour x2.
* Network (inputs r_hat = r / rms(r) and eps, 2 channels):
    e1 = relu(conv3(relu(conv3([r_hat, eps]; 2 -> 16)); 16 -> 16))
    e2 = relu(conv3(relu(conv3(pool(e1); 16 -> 32)); 32 -> 32))
    e3 = relu(conv3(relu(conv3(pool(e2); 32 -> 64)); 64 -> 64))
    d2 = relu(conv3(relu(conv3([up(e3), e2]; 96 -> 32)); 32 -> 32))
    d1 = relu(conv3(relu(conv3([up(d2), e1]; 48 -> 16)); 16 -> 16))
    z  = h . d1 + h0   (1x1x1 head, 16 -> 1, no activation)
  ([a, b] is channel concatenation, a first.)
* Training loss for one residual r of the pressure operator A (SPD):
  L = |A z - r_hat|^2 / |r_hat|^2.
* Optional BF16 emulation (``bf16=True``): inputs, conv weights and the
  output of every conv and pool are rounded to bfloat16 (round to nearest
  even), as the tensor-core path stores them; accumulation stays FP64.

Backward passes are written out by hand (the chain rule per operation) and
pinned in the tests by finite differences and adjoint identities.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

# (name, C_in, C_out) of the ten 3x3x3 convs, in forward order
LAYERS = [
    ("enc1a", 2, 16), ("enc1b", 16, 16),
    ("enc2a", 16, 32), ("enc2b", 32, 32),
    ("enc3a", 32, 64), ("enc3b", 64, 64),
    ("dec2a", 96, 32), ("dec2b", 32, 32),
    ("dec1a", 48, 16), ("dec1b", 16, 16),
]


def bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), via FP32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, t):
    """xs[v] = x[v + t] with zeros outside the box (x: (nz, ny, nx, C))."""
    out = np.zeros_like(x)
    src = []
    dst = []
    for ax, d in enumerate(t):
        n = x.shape[ax]
        if d >= 0:
            src.append(slice(d, n))
            dst.append(slice(0, n - d))
        else:
            src.append(slice(0, n + d))
            dst.append(slice(-d, n))
    out[tuple(dst)] = x[tuple(src)]
    return out


def conv3(x, W, b):
    """3x3x3 zero-padded convolution (cross-correlation), W: (Co, 3, 3, 3, Ci)."""
    y = np.broadcast_to(b, x.shape[:3] + (W.shape[0],)).copy()
    for t in TAPS:
        y += _shift(x, t) @ W[:, t[0] + 1, t[1] + 1, t[2] + 1, :].T
    return y


def conv3_backward(x, W, dy):
    """Gradients of sum(dy * conv3(x, W, b)) w.r.t. x, W and b.

    dx[v] = sum_t W[:, t]^T dy[v - t] (the shifts taken the other way),
    dW[:, t, :] = dy^T shift(x, t), db = sum over voxels of dy."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in TAPS:
        wt = W[:, t[0] + 1, t[1] + 1, t[2] + 1, :]
        dx += _shift(dy, (-t[0], -t[1], -t[2])) @ wt
        dW[:, t[0] + 1, t[1] + 1, t[2] + 1, :] = dy.reshape(-1, dy.shape[-1]).T @ _shift(x, t).reshape(-1, x.shape[-1])
    db = dy.reshape(-1, dy.shape[-1]).sum(axis=0)
    return dx, dW, db


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def pool_backward(dy):
    return up(dy) / 8.0


def up(x):
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def up_backward(dy):
    nz, ny, nx, c = dy.shape
    return dy.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def init_params(seed):
    """He-normal weights, zero biases (the GPU side takes the same arrays)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co in LAYERS:
        P[name + ".W"] = rng.standard_normal((co, 3, 3, 3, ci)) * np.sqrt(2.0 / (27 * ci))
        P[name + ".b"] = np.zeros(co)
    P["head.W"] = rng.standard_normal(16) * np.sqrt(1.0 / 16)
    P["head.b"] = np.zeros(1)
    return P


def normalise(r):
    """r_hat = r / rms(r) (0 for r = 0)."""
    rms = np.sqrt(np.mean(np.square(r)))
    return r / rms if rms > 0 else np.zeros_like(r)


def forward(P, r_hat, eps, bf16_emulation=False):
    """Network output z (nz, ny, nx) and the cache for backward."""
    rnd = bf16 if bf16_emulation else (lambda a: a)
    C = {}

    def cv(name, x):
        W = rnd(P[name + ".W"])
        pre = conv3(x, W, P[name + ".b"])
        out = rnd(np.maximum(pre, 0.0))
        C[name] = (x, W, pre)
        return out

    x0 = rnd(np.stack([r_hat, eps], axis=-1))
    e1 = cv("enc1b", cv("enc1a", x0))
    p1 = rnd(pool(e1))
    e2 = cv("enc2b", cv("enc2a", p1))
    p2 = rnd(pool(e2))
    e3 = cv("enc3b", cv("enc3a", p2))
    c2 = np.concatenate([up(e3), e2], axis=-1)
    d2 = cv("dec2b", cv("dec2a", c2))
    c1 = np.concatenate([up(d2), e1], axis=-1)
    d1 = cv("dec1b", cv("dec1a", c1))
    z = d1 @ P["head.W"] + P["head.b"][0]
    C["d1"] = d1
    return z, C


def backward(P, C, dz, bf16_emulation=False):
    """Gradients of sum(dz * z) for every parameter (same keys as P).

    With BF16 emulation the upstream gradient of each conv is rounded to
    BF16 before the data-gradient convolution and the weight-gradient
    contraction (the tensor-core path takes BF16 operands for both); the
    bias gradient sums it unrounded."""
    rnd = bf16 if bf16_emulation else (lambda a: a)
    G = {}
    G["head.W"] = C["d1"].reshape(-1, 16).T @ dz.ravel()
    G["head.b"] = np.array([dz.sum()])
    g = dz[..., None] * P["head.W"]

    def cvb(name, g_out, need_dx=True):
        x, W, pre = C[name]
        g_pre = g_out * (pre > 0.0)
        dx, dW, _ = conv3_backward(x, W, rnd(g_pre))
        G[name + ".W"] = dW
        G[name + ".b"] = g_pre.reshape(-1, g_pre.shape[-1]).sum(axis=0)
        return dx if need_dx else None

    g = cvb("dec1a", cvb("dec1b", g))
    g_up_d2, g_e1 = g[..., :32], g[..., 32:]
    g = cvb("dec2a", cvb("dec2b", up_backward(g_up_d2)))
    g_up_e3, g_e2 = g[..., :64], g[..., 64:]
    g = cvb("enc3a", cvb("enc3b", up_backward(g_up_e3)))
    g_e2 = g_e2 + pool_backward(g)
    g = cvb("enc2a", cvb("enc2b", g_e2))
    g_e1 = g_e1 + pool_backward(g)
    cvb("enc1a", cvb("enc1b", g_e1), need_dx=False)
    return G


def loss_and_grad_z(A, z, r_hat):
    """L = |A z - r_hat|^2 / |r_hat|^2 and dL/dz = 2 A (A z - r_hat) / |r_hat|^2
    (A symmetric, a scipy sparse matrix over the flattened box)."""
    rn = float(np.dot(r_hat.ravel(), r_hat.ravel()))
    res = A @ z.ravel() - r_hat.ravel()
    L = float(np.dot(res, res)) / rn
    dz = (2.0 / rn) * (A @ res)
    return L, dz.reshape(z.shape)
