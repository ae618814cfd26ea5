"""Host logic of the floating-cluster deflation of the pressure solve.

The labels that ``vos_floating_clusters`` returns (the clusters the pressure
preconditioner deflates) are checked against an independent construction
with scipy's connected components on the graph of strong faces of the
pressure operator (face porosity 0.5 (eps_a + eps_b) >= 0.01, Sec. 2.2's
arithmetic face mean), keeping components of >= 2 cells that contain no
outlet cell.  No GPU is needed.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_2204_07019_gb300 import inputs as I
from paper_2204_07019_gb300 import vos as V

THETA = 0.01


def expected_labels(eps):
    """Cluster labels from scipy, numbered by each cluster's smallest cell."""
    shape = eps.shape
    n = eps.size
    idx = np.arange(n).reshape(shape)
    rows, cols = [], []
    for ax in range(eps.ndim):
        a = [slice(None)] * eps.ndim
        b = [slice(None)] * eps.ndim
        a[ax] = slice(0, -1)
        b[ax] = slice(1, None)
        strong = 0.5 * (eps[tuple(a)] + eps[tuple(b)]) >= THETA
        rows.append(idx[tuple(a)][strong])
        cols.append(idx[tuple(b)][strong])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    g = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    comp = comp.reshape(shape)
    sizes = np.bincount(comp.ravel())
    outlet = set(np.unique(comp[..., -1]).tolist())
    first = {}
    for cell, q in enumerate(comp.ravel()):
        if sizes[q] >= 2 and q not in outlet and q not in first:
            first[q] = len(first)
    lab = np.full(n, -1, dtype=np.int32)
    for cell, q in enumerate(comp.ravel()):
        if q in first:
            lab[cell] = first[q]
    return lab.reshape(shape), len(first)


def _prm(shape):
    full = (1,) * (3 - len(shape)) + tuple(shape)
    return I.make_params(full, Pe=10.0, Da=1.0, L=8.0, method="ivos")


def test_hand_made_pocket_2d():
    """A 3x2 pore pocket inside solid is one cluster, and so is a single pore
    cell with its solid ring; the channel that reaches the outlet is not."""
    eps = np.full((10, 12), 1e-4)
    eps[1, :] = 1.0          # channel to the outlet column: anchored
    eps[5:7, 3:6] = 1.0      # pocket (3 x 2 pore cells)
    eps[8, 9] = 1.0          # single pore cell: its solid ring joins it
    lab, k, m = V.vos_floating_clusters(eps, _prm(eps.shape))
    ref, kr = expected_labels(eps)
    assert k == kr == 2
    np.testing.assert_array_equal(lab, ref)
    # the pocket cluster holds the 6 pore cells and their 10 edge neighbours
    pocket = lab[5, 3]
    assert pocket >= 0 and (lab == pocket).sum() == 6 + 10
    assert (lab[1, :] == -1).all()
    assert m == (lab >= 0).sum()


def test_all_pore_and_all_solid():
    for val, k_expected in ((1.0, 0), (1e-4, 0)):
        eps = np.full((6, 7, 9), val)
        lab, k, m = V.vos_floating_clusters(eps, _prm(eps.shape))
        assert k == k_expected and m == 0 and (lab == -1).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_connected_components_rock(seed):
    es = I.sphere_rock_3d(40, seed=seed, median_r=3.0)
    eps = np.maximum(1.0 - es, 1e-4)
    lab, k, m = V.vos_floating_clusters(eps, _prm(eps.shape))
    ref, kr = expected_labels(eps)
    assert k == kr
    np.testing.assert_array_equal(lab, ref)
    assert m == (ref >= 0).sum()


def test_matches_connected_components_random_2d():
    rng = np.random.default_rng(7)
    eps = np.where(rng.random((48, 64)) < 0.45, 1.0, 1e-4)
    eps[rng.random(eps.shape) < 0.05] = 0.015  # partially dissolved cells near the threshold
    lab, k, m = V.vos_floating_clusters(eps, _prm(eps.shape))
    ref, kr = expected_labels(eps)
    assert k == kr and k > 0
    np.testing.assert_array_equal(lab, ref)


def test_rejects_bad_arguments():
    eps = np.ones((4, 5))
    with pytest.raises(ValueError):
        V.vos_floating_clusters(np.ones(7), _prm(eps.shape))
    bad = dict(_prm(eps.shape))
    bad["precond"] = 6
    with pytest.raises(V.VosError):
        V.vos_floating_clusters(eps, bad)
