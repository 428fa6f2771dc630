"""The device FP64 log and exp (table-driven, used by the solver) against numpy's: within
2 ulp on wide ranges, near 1 for the logarithm, and IEEE special values."""
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
