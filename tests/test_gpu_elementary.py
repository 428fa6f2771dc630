"""The device FP64 log and exp (table-driven, used by the solver) against numpy's: within
2 ulp on wide ranges, near 1 for the logarithm, and IEEE special values; and the guesses'
-Phi^{-1} against mpmath."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import api  # noqa: E402
from gpu_helpers import to_dev, to_np  # noqa: E402

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref):
    fin = np.isfinite(ref) & (ref != 0)
    return np.abs(got[fin] - ref[fin]) / np.spacing(np.abs(ref[fin]))


def test_log_fp64():
    rng = np.random.default_rng(1)
    v = np.concatenate([10.0 ** rng.uniform(-307, 308, 200_000), 1 + rng.uniform(-1e-2, 1e-2, 100_000),
                        1 + rng.uniform(-1e-14, 1e-14, 10_000), rng.uniform(0.0, 3.0, 100_000)])
    got = to_np(api.elementary("log", to_dev(v)))
    ref = np.log(v)
    assert _ulp_err(got, ref).max() <= 2.0
    assert np.all(got[v == 1.0] == 0.0)
    special = np.array([0.0, -0.0, -1.0, np.inf, np.nan, 4.9e-324, 1e-310, -np.inf])
    got = to_np(api.elementary("log", to_dev(special)))
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.log(special)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    m = ~np.isnan(ref)
    assert np.allclose(got[m], ref[m], rtol=4e-16, atol=0)


def test_exp_fp64():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-707.99, 707.99, 200_000), rng.uniform(-1, 1, 100_000),
                        rng.uniform(-1e-10, 1e-10, 10_000)])
    got = to_np(api.elementary("exp", to_dev(x)))
    assert _ulp_err(got, np.exp(x)).max() <= 2.0
    special = np.array([0.0, -0.0, 708.0, 709.7, 710.0, -708.0, -740.0, -745.0, -746.0, np.inf, -np.inf, np.nan])
    got = to_np(api.elementary("exp", to_dev(special)))
    with np.errstate(over="ignore"):
        ref = np.exp(special)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    m = ~np.isnan(ref)
    # beyond |v| = 708 the library exponential answers; in the subnormal range it may round
    # differently from the host's by a few units of the smallest subnormal
    assert np.allclose(got[m], ref[m], rtol=4e-16, atol=1e-322)


def test_neg_ncdfinv_of_the_guesses():
    """-Phi^{-1}(G) of the lower- and upper-region guesses: the float inverse normal CDF from 1e-37
    on (seed accuracy), the library's FP64 normcdfinv below; against 50-digit mpmath and scipy."""
    mp = pytest.importorskip("mpmath")
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    G = np.concatenate([np.logspace(-300, np.log10(0.5), 400), np.logspace(-37, np.log10(0.5), 600),
                        [0.5, np.nextafter(0.5, 0), 0.49999, 1e-37, np.nextafter(1e-37, 0)]])
    got = to_np(api.elementary("neg_ncdfinv", to_dev(G)))
    with mp.workdps(50):
        # the root of erfc(y / sqrt 2) / 2 = G (no cancellation in the tail), from scipy's value
        ref = np.array([float(mp.findroot(lambda y: mp.erfc(y / mp.sqrt(2)) / 2 - mp.mpf(float(g)), -special.ndtri(g)))
                        for g in G])
    err = np.abs(got - ref)
    # float branch: a few float ulps of y, plus the rounding of G to float near y = 0
    assert np.all(err <= 2e-6 * np.abs(ref) + 1e-7), (err / np.maximum(np.abs(ref), 1e-300)).max()
    # the library branch below 1e-37 is FP64-accurate
    lo = G < 1e-37
    assert np.all(err[lo] <= 1e-14 * np.abs(ref[lo]))
    assert abs(got[G == 0.5][0]) < 1e-7
    # dense sample against scipy
    g2 = np.exp(rng.uniform(np.log(1e-37), np.log(0.5), 200_000))
    got2 = to_np(api.elementary("neg_ncdfinv", to_dev(g2)))
    ref2 = -special.ndtri(g2)
    assert np.all(np.abs(got2 - ref2) <= 2e-6 * np.abs(ref2) + 1e-7)


def test_seed_cube_root():
    """The guesses' cube root: float cube root of the mantissa scaled into [1, 8), exponent added
    as an integer, ~1e-7 relative over the whole positive normal range; library cbrt elsewhere."""
    rng = np.random.default_rng(5)
    v = np.concatenate([10.0 ** rng.uniform(-307.5, 308, 500_000), rng.uniform(0.5, 8.0, 100_000),
                        [1.0, 8.0, 27.0, 2.0 ** -1022, 2.0 ** 1023, 0.125]])
    got = to_np(api.elementary("cbrt", to_dev(v)))
    ref = np.cbrt(v)
    assert np.all(np.abs(got - ref) <= 2.5e-7 * ref)
    special = np.array([0.0, 5e-324, 1e-310, np.inf])
    got = to_np(api.elementary("cbrt", to_dev(special)))
    assert np.allclose(got, np.cbrt(special), rtol=1e-15, atol=0)


def test_fast_reciprocal():
    """The solver's quotients off the rounding-critical path: 1/x from the hardware estimate and
    two Newton-Raphson steps, within 1 ulp of the IEEE reciprocal over the whole normal range,
    and the IEEE result itself for zero, subnormal, huge, infinite and NaN x."""
    rng = np.random.default_rng(4)
    e = rng.integers(-1021, 1022, 2_000_000)
    m = rng.uniform(1.0, 2.0, e.size)
    x = np.ldexp(m, e) * np.where(rng.random(e.size) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, [1.0, -1.0, 2.0 ** -1022, 0.75, 3.0, np.nextafter(2.0, 0)]])
    got = to_np(api.elementary("rcp", to_dev(x)))
    ref = 1.0 / x
    assert _ulp_err(got, ref).max() <= 1.0
    special = np.array([0.0, -0.0, 5e-324, -1e-310, 2.0 ** 1022, 1e308, np.inf, -np.inf, np.nan])
    got = to_np(api.elementary("rcp", to_dev(special)))
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / special
    assert np.array_equal(got, ref, equal_nan=True)
