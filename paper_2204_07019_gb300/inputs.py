"""Seeded synthetic inputs: solid-fraction fields and non-dimensional parameters.

This module is shared by the CUDA path, the tests and the CPU oracle.  It
holds only input generation (geometry rasterisation and the mapping from
(Pe, Da) to physical parameters); none of the method's arithmetic lives here.

Geometry recipes (the paper's image data -- calcite post, BM2 micromodel,
Ketton micro-CT -- are not available, so these stand in for them, keeping
only their shapes, sizes and porosities):

* ``calcite_post_2d``: one disc in a channel (benchmark 1 analogue, Sec. 3.1).
* ``disc_micromodel_2d``: polydisperse non-overlapping discs placed by seeded
  random sequential addition to a target porosity (benchmark 2 analogue,
  Sec. 3.2).
* ``sphere_rock_3d``: union of overlapping spheres with lognormal radii,
  shifted ("eroded") by a signed-distance threshold to a target porosity and
  checked to percolate inlet->outlet (benchmark 3 analogue, Sec. 3.3).

All fields are returned as float64 arrays of shape (nz, ny, nx) (nz = 1 in
2D), x fastest, holding the solid fraction eps_s in [0, 1] with a one-cell
linear ramp at interfaces.

Parameters follow the dimensionless groups of Sec. 2.5: Pe = U L / D,
Da = k_c / U, beta = c_in M_ws / (zeta rho_s).  We take U = u_in = 1,
dx = 1, Sc = nu / D = 1000, k0 = 1e-4 dx^2, V_m c_in = 1e-3, zeta = 1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "PARAM_DEFAULTS", "make_params", "calcite_post_2d", "disc_micromodel_2d",
    "sphere_rock_3d", "batched_micromodels", "random_field", "porosity",
]

# Method ids (match include/vos.h)
VOS_PSI, VOS_PSI_PRIME, VOS_IVOS = 0, 1, 2
METHOD_IDS = {"psi": VOS_PSI, "psi_prime": VOS_PSI_PRIME, "ivos": VOS_IVOS}

# Boundary-side bits for wall_mask (match include/vos.h)
WALL_YM, WALL_YP, WALL_ZM, WALL_ZP = 1, 2, 4, 8

PARAM_DEFAULTS = dict(
    dim=2, nx=0, ny=0, nz=1, dx=1.0,
    nu=1.0, D=1.0, kc=0.0, k0=1e-4, Vm=1e-3, zeta=1.0, rho_ratio=1.0,
    c_in=1.0, u_in=1.0, eps_min=1e-4, lam=4.0,
    method=VOS_IVOS, precision=0, precond=0,
    p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10,
    max_iter=500, flow_subiters=1, qs_rtol=0.0, qs_dtau=0.0, inertia=0,
    wall_mask=WALL_YM | WALL_YP | WALL_ZM | WALL_ZP,
)


def make_params(shape, Pe, Da, L, method="ivos", Sc=1000.0, **over):
    """Map (Pe, Da, reference length L) to the parameter dict.

    With U = u_in = 1 and dx = 1: D = U L / Pe, k_c = Da U, nu = Sc D.
    ``shape`` is (nz, ny, nx); nz == 1 selects 2D.
    """
    nz, ny, nx = shape
    p = dict(PARAM_DEFAULTS)
    D = 1.0 * L / Pe
    p.update(dim=2 if nz == 1 else 3, nx=nx, ny=ny, nz=nz, D=D, kc=Da * 1.0,
             nu=Sc * D, method=METHOD_IDS[method] if isinstance(method, str) else method)
    p.update(over)
    return p


def porosity(eps_s):
    return float(1.0 - np.mean(eps_s))


def _disc_ramp(shape2, cx, cy, R):
    """eps_s of one disc, cell centres at (i+1/2, j+1/2): clamp(R + 1/2 - r, 0, 1)."""
    ny, nx = shape2
    y = np.arange(ny)[:, None] + 0.5
    x = np.arange(nx)[None, :] + 0.5
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return np.clip(R + 0.5 - r, 0.0, 1.0)


def calcite_post_2d(nx=256, ny=64, cx=64.0, cy=32.0, R=16.0):
    """Single disc of radius R centred at (cx, cy) with a 1-cell linear ramp."""
    return _disc_ramp((ny, nx), cx, cy, R)[None, :, :].astype(np.float64)


def disc_micromodel_2d(nx=1024, ny=512, seed=0, rmin=8.0, rmax=32.0,
                       target_porosity=0.60, band=2, gap=1.0, max_tries=200000):
    """Polydisperse non-overlapping discs by seeded random sequential addition.

    Radii ~ U[rmin, rmax]; centres uniform such that discs stay inside
    x in [band, nx - band] and y in [0, ny]; any two discs keep a gap >= ``gap``
    cells.  Discs are added until the porosity (1 - mean eps_s) reaches the
    target.  Returns eps_s of shape (1, ny, nx).
    """
    rng = np.random.default_rng(seed)
    es = np.zeros((ny, nx))
    cxs, cys, rs = [], [], []
    tries = 0
    while porosity(es) > target_porosity and tries < max_tries:
        tries += 1
        R = rng.uniform(rmin, rmax)
        lo_x, hi_x = band + R + 1.0, nx - band - R - 1.0
        lo_y, hi_y = R + 1.0, ny - R - 1.0
        if hi_x <= lo_x or hi_y <= lo_y:
            continue
        cx = rng.uniform(lo_x, hi_x)
        cy = rng.uniform(lo_y, hi_y)
        if cxs:
            d = np.hypot(np.asarray(cxs) - cx, np.asarray(cys) - cy)
            if np.any(d < np.asarray(rs) + R + gap + 1.0):
                continue
        cxs.append(cx); cys.append(cy); rs.append(R)
        x0, x1 = max(int(cx - R - 2), 0), min(int(cx + R + 3), nx)
        y0, y1 = max(int(cy - R - 2), 0), min(int(cy + R + 3), ny)
        sub = _disc_ramp((y1 - y0, x1 - x0), cx - x0, cy - y0, R)
        es[y0:y1, x0:x1] = np.maximum(es[y0:y1, x0:x1], sub)
    return es[None, :, :].astype(np.float64)


def _sphere_sdf(shape, centres, radii, margin):
    """max_i (R_i - |x - c_i|) clipped below at -margin (positive inside solid)."""
    nz, ny, nx = shape
    sdf = np.full(shape, -float(margin))
    for (cz, cy, cx), R in zip(centres, radii):
        h = R + margin + 1.0
        z0, z1 = max(int(cz - h), 0), min(int(cz + h) + 1, nz)
        y0, y1 = max(int(cy - h), 0), min(int(cy + h) + 1, ny)
        x0, x1 = max(int(cx - h), 0), min(int(cx + h) + 1, nx)
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        z = np.arange(z0, z1)[:, None, None] + 0.5
        y = np.arange(y0, y1)[None, :, None] + 0.5
        x = np.arange(x0, x1)[None, None, :] + 0.5
        d = R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        np.maximum(sdf[z0:z1, y0:y1, x0:x1], d, out=sdf[z0:z1, y0:y1, x0:x1])
    return sdf


def _percolates_x(pore):
    from scipy import ndimage
    lab, _ = ndimage.label(pore)
    a = np.unique(lab[:, :, 0]); b = np.unique(lab[:, :, -1])
    common = np.intersect1d(a[a > 0], b[b > 0])
    return common.size > 0


def sphere_rock_3d(n=256, seed=0, median_r=12.0, sigma=0.3, target_porosity=0.20,
                   start_solid=0.8, band=2, margin=4.0, max_reseed=8):
    """Overlapping-sphere rock, shifted to the target porosity, percolating in x.

    Solid = union of spheres with lognormal radii (median ``median_r``,
    log-sd ``sigma``), centres uniform, added until the solid fraction of the
    union reaches ``start_solid``.  The union's signed distance s(x) is then
    shifted by t (bisection) so that eps_s = clamp(s - t + 1/2, 0, 1) gives
    the target porosity in the rock; ``band`` fluid layers are kept at the
    inlet and outlet.  Reseeds (seed + 7919 k) until the pore space
    (eps_s < 1/2, 6-connected) joins inlet and outlet.
    Returns eps_s of shape (n, n, n) (or ``n`` a (nz, ny, nx) tuple).
    """
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    nz, ny, nx = shape
    vol = float(nz * ny * nx)
    for k in range(max_reseed):
        rng = np.random.default_rng(seed + 7919 * k)
        mean_v = 4.0 / 3.0 * math.pi * median_r ** 3 * math.exp(4.5 * sigma * sigma)
        n_sph = int(math.ceil(-math.log(1.0 - start_solid) * vol / mean_v * 1.05))
        radii = median_r * np.exp(sigma * rng.standard_normal(n_sph))
        centres = np.stack([rng.uniform(0, nz, n_sph), rng.uniform(0, ny, n_sph),
                            rng.uniform(0, nx, n_sph)], axis=1)
        sdf = _sphere_sdf(shape, centres, radii, margin)
        rock = (slice(None), slice(None), slice(band, nx - band))

        def phi_of(t):
            return 1.0 - float(np.mean(np.clip(sdf[rock] - t + 0.5, 0.0, 1.0)))

        lo, hi = -margin + 1.0, margin - 1.0
        if phi_of(hi) < target_porosity or phi_of(lo) > target_porosity:
            continue
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if phi_of(mid) < target_porosity:
                lo = mid
            else:
                hi = mid
        t = 0.5 * (lo + hi)
        es = np.clip(sdf - t + 0.5, 0.0, 1.0)
        es[:, :, :band] = 0.0
        es[:, :, nx - band:] = 0.0
        if _percolates_x(es < 0.5):
            return es.astype(np.float64)
    raise RuntimeError("sphere_rock_3d: no percolating sample found")


def batched_micromodels(count=64, seed=0, lo=128, hi=768):
    """List of (eps_s, Pe, Da) for the batched micromodel workload.

    Side lengths i.i.d. uniform integers in [lo, hi]; discs as in
    ``disc_micromodel_2d`` (porosity 0.6); Pe log-uniform in [1, 100],
    Da log-uniform in [0.01, 100].
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        nx, ny = (int(v) for v in rng.integers(lo, hi + 1, size=2))
        Pe = float(10 ** rng.uniform(0.0, 2.0))
        Da = float(10 ** rng.uniform(-2.0, 2.0))
        es = disc_micromodel_2d(nx, ny, seed=seed * 1000 + b + 1)
        out.append((es, Pe, Da))
    return out


def random_field(shape, seed, lo=0.0, hi=1.0, smooth=0):
    """Seeded uniform random field in [lo, hi] of the given (nz, ny, nx) shape,
    optionally box-smoothed ``smooth`` times (for gradient-rich test inputs)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(lo, hi, size=shape)
    for _ in range(smooth):
        g = f.copy()
        for ax in range(3):
            if f.shape[ax] > 2:
                g = g + np.roll(f, 1, ax) + np.roll(f, -1, ax)
        f = g / (1 + 2 * sum(1 for a in range(3) if f.shape[a] > 2))
    return f.astype(np.float64)
