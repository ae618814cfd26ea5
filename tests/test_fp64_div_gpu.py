"""The FP64 quotient of the physics kernels against IEEE division.

The kernels replace IEEE division by a Newton-Raphson refinement of the
hardware reciprocal estimate (FP64 instructions are their bottleneck).  The
quotient must stay within a couple of ulp of a/d over the range the kernels
use, and fall back to the IEEE quotient outside it.  The IEEE column is
checked against numpy's division first, so the harness itself is pinned.
"""
import numpy as np
import pytest

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


def _ulps(q, ref):
    return np.abs(q - ref) / np.spacing(np.abs(ref))


def test_quotient_within_two_ulp(V):
    rng = np.random.default_rng(11)
    n = 1 << 20
    # magnitudes over most of the FP64 range, both signs, quotient normal
    ea = rng.uniform(-280, 280, n)
    ed = ea - rng.uniform(-280, 280, n)
    ed = np.clip(ed, -299, 299)
    a = rng.choice([-1.0, 1.0], n) * 10.0 ** ea * rng.uniform(1, 10, n)
    d = rng.choice([-1.0, 1.0], n) * 10.0 ** ed * rng.uniform(1, 10, n)
    # plus the ranges the physics meets: O(1) differences, diagonals, k0 eps^3
    a[:4096] = rng.uniform(-1, 1, 4096)
    d[:4096] = rng.uniform(1e-6, 2, 4096)
    qf, qi = V.vos_fp64_div_check(a, d)
    np.testing.assert_array_equal(qi, a / d)
    ref = a / d
    ok = np.isfinite(ref) & (np.abs(ref) > 1e-300)
    assert ok.sum() > n // 2
    assert _ulps(qf[ok], ref[ok]).max() <= 2.0


def test_exact_cases_and_zero_numerator(V):
    """Exactly representable quotients come out exact; a zero numerator gives
    a zero (its sign is not kept: the quotient step adds +0 to -0)."""
    a = np.array([1.0, 3.0, -6.0, 0.0, -0.0, 2.5, 1.0])
    d = np.array([1.0, 3.0, 2.0, 7.0, 7.0, 0.5, 4.0])
    qf, _ = V.vos_fp64_div_check(a, d)
    np.testing.assert_array_equal(qf, a / d)


def test_out_of_range_takes_ieee(V):
    d = np.array([0.0, -0.0, 5e-324, 1e-305, 2.0 ** -1001, 2.0 ** 1001, 1e305, np.inf, -np.inf, np.nan])
    a = np.full(d.shape, 3.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = a / d
    qf, qi = V.vos_fp64_div_check(a, d)
    np.testing.assert_array_equal(qf, qi)
    np.testing.assert_array_equal(qi, ref)
