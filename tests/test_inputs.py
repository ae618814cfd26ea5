"""Seeded synthetic inputs, the stand-ins for the paper's image data: each
generator is deterministic for its seed and meets the recipe it states
(shapes, porosities, fluid bands at inlet and outlet, percolation, parameter
mapping)."""
import math

import numpy as np
from scipy import ndimage

from paper_2204_07019_gb300 import inputs as I


def test_calcite_post_area_and_centre():
    es = I.calcite_post_2d(256, 64, 64.0, 32.0, 16.0)
    assert es.shape == (1, 64, 256) and es.min() >= 0.0 and es.max() <= 1.0
    # the one-cell linear ramp integrates to about the disc area pi R^2
    assert abs(es.sum() - math.pi * 16.0 ** 2) < 0.01 * math.pi * 16.0 ** 2
    y, x = np.nonzero(es[0] > 0.5)
    assert abs(x.mean() + 0.5 - 64.0) < 0.1 and abs(y.mean() + 0.5 - 32.0) < 0.1


def test_disc_micromodel_recipe():
    kw = dict(rmin=4.0, rmax=12.0)
    es = I.disc_micromodel_2d(256, 128, seed=4, **kw)
    assert es.shape == (1, 128, 256)
    # discs are added until the porosity reaches 0.60; the last disc may
    # overshoot by at most its own area
    assert 0.60 - math.pi * 12.5 ** 2 / es.size <= I.porosity(es) <= 0.60
    assert np.all(es[..., :2] == 0.0) and np.all(es[..., -2:] == 0.0)
    # non-overlapping discs with a gap: every solid component is one disc
    lab, k = ndimage.label(es[0] > 0.0)
    areas = np.bincount(lab.ravel())[1:]
    assert k > 10 and areas.min() >= 0.8 * math.pi * 3.5 ** 2 and areas.max() <= 1.1 * math.pi * 12.5 ** 2
    np.testing.assert_array_equal(es, I.disc_micromodel_2d(256, 128, seed=4, **kw))
    assert not np.array_equal(es, I.disc_micromodel_2d(256, 128, seed=5, **kw))


def test_sphere_rock_recipe():
    kw = dict(median_r=5.0, target_porosity=0.3)
    es = I.sphere_rock_3d(48, seed=2, **kw)
    assert es.shape == (48, 48, 48) and es.min() >= 0.0 and es.max() <= 1.0
    assert abs((1.0 - es[:, :, 2:-2].mean()) - 0.3) < 1e-6  # the shift is bisected to the target
    assert np.all(es[..., :2] == 0.0) and np.all(es[..., -2:] == 0.0)
    lab, _ = ndimage.label(es < 0.5)
    joined = np.intersect1d(np.unique(lab[..., 0]), np.unique(lab[..., -1]))
    assert joined[joined > 0].size > 0  # the pore space joins inlet and outlet
    np.testing.assert_array_equal(es, I.sphere_rock_3d(48, seed=2, **kw))


def test_batched_micromodels_recipe():
    """The 64-instance batch workload: sides in [128, 768], porosity 0.60
    (reached to within the last disc), Pe in [1, 100], Da in [0.01, 100];
    the first instances do not depend on the batch size."""
    items = I.batched_micromodels()
    assert len(items) == 64
    for es, Pe, Da in items:
        _, ny, nx = es.shape
        assert 128 <= nx <= 768 and 128 <= ny <= 768
        assert 1.0 <= Pe <= 100.0 and 0.01 <= Da <= 100.0
        assert 0.58 <= I.porosity(es) <= 0.60
    for (a, pa, da), (b, pb, db) in zip(items[:2], I.batched_micromodels(count=2)):
        np.testing.assert_array_equal(a, b)
        assert (pa, da) == (pb, db)


def test_make_params_mapping():
    p = I.make_params((1, 20, 40), Pe=8.0, Da=0.5, L=16.0, method="psi_prime")
    assert p["dim"] == 2 and (p["nx"], p["ny"], p["nz"]) == (40, 20, 1)
    assert p["D"] == 16.0 / 8.0 and p["kc"] == 0.5 and p["nu"] == 1000.0 * p["D"]
    q = I.make_params((6, 7, 9), Pe=1.0, Da=1.0, L=1.0, precision=1)
    assert q["dim"] == 3 and q["precision"] == 1
