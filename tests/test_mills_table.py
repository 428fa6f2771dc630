"""The FP64 Mills-ratio table behind Y = Phi/phi (csrc/mills_table.inc), checked on the CPU.

The device code evaluates M(w) = Y(-w) = Phi(-w)/phi(w) for 0 <= w < 128 as the degree-9
polynomial of the interval picked by the bit pattern of w (interval 0 = [0, 1/16); from 1/16
on, 16 equal parts per binade), in tau = w * scale + offset, by Horner's rule in double; this
test repeats the index arithmetic on the bit patterns and the evaluation in numpy and compares
with Phi(-w)/phi(w) in 50-digit mpmath (the normal tail over the density: no cancellation), and
checks the asymptotic series used from 128 on.
"""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_17065_gb300", "csrc",
                   "mills_table.inc")
N_INTERVALS = 1 + 16 * 11  # [0, 1/16), then 16 parts of each binade 2^-4 .. 2^7


def table():
    text = open(INC).read()
    rows = re.findall(r"\{([^{}]+)\}", text.split("=", 1)[1])
    return np.array([[float(v) for v in r.split(",")] for r in rows])


def interval_index(w):
    """The device's index: the biased exponent and top four mantissa bits, less those of 1/16, plus one."""
    bits = np.asarray(w, dtype=np.float64).view(np.uint64) & np.uint64(0x7fffffffffffffff)
    raw = (bits >> np.uint64(48)).astype(np.int64)
    return np.maximum(raw - ((1023 - 4) << 4) + 1, 0)


def eval_table(C, w):
    c = C[interval_index(w)]
    tau = w * c[:, 10] + c[:, 11]
    v = c[:, 9].copy()
    for k in range(8, -1, -1):
        v = v * tau + c[:, k]
    return v, tau


def mills_ref(w):
    with mp.workdps(50):
        return np.array([float(mp.ncdf(-mp.mpf(x)) / mp.npdf(mp.mpf(x))) for x in w])


def test_interval_index_and_bounds():
    C = table()
    assert C.shape == (N_INTERVALS, 12)
    # the index of each interval's left end is that interval, and tau runs over [-1, 1) on it
    lo = np.concatenate([[0.0], [2.0 ** e * (1 + m / 16) for e in range(-4, 7) for m in range(16)]])
    assert np.array_equal(interval_index(lo), np.arange(N_INTERVALS))
    assert np.array_equal(interval_index(np.nextafter(lo[1:], 0)), np.arange(N_INTERVALS - 1))
    assert interval_index(np.array([np.nextafter(128.0, 0)]))[0] == N_INTERVALS - 1
    w = np.concatenate([lo, np.nextafter(lo[1:], 0), [np.nextafter(128.0, 0), 5e-324, 1e-300, -0.0]])
    _, tau = eval_table(C, np.abs(w))
    assert np.all(tau >= -1.0) and np.all(tau <= 1.0)
    # scale is a power of two and offset an integer: tau = w scale + offset rounds once
    assert np.all(np.frexp(C[:, 10])[0] == 0.5) and np.all(C[:, 11] == np.round(C[:, 11]))


def test_table_matches_the_mills_ratio_to_a_few_ulp():
    C = table()
    rng = np.random.default_rng(0)
    w = np.concatenate([np.linspace(0, 128, 4001)[:-1], rng.uniform(0, 128, 2000),
                        np.exp(rng.uniform(-12, np.log(128), 2000)),
                        [0.0, 1.0 / 16, np.nextafter(1.0 / 16, 0), np.nextafter(128.0, 0), 1e-300]])
    w = w[w < 128]
    got, _ = eval_table(C, w)
    ref = mills_ref(w)
    assert np.max(np.abs(got - ref) / ref) < 4e-16


def test_table_is_sqrt_pi_over_2_erfcx():
    """M(w) = sqrt(pi/2) erfcx(w / sqrt 2): the same function as the textbook erfcx (scipy)."""
    sps = pytest.importorskip("scipy.special")
    C = table()
    w = np.linspace(0.0, 127.9, 20001)
    got, _ = eval_table(C, w)
    ref = np.sqrt(np.pi / 2) * sps.erfcx(w / np.sqrt(2))
    assert np.max(np.abs(got - ref) / ref) < 2e-15


def test_asymptotic_series_beyond_128():
    coef = [1.0, -1.0, 3.0, -15.0, 105.0, -945.0, 10395.0, -135135.0, 2027025.0]
    for w in [128.0, 128.5, 300.0, 1e3, 1e8]:
        q = 1.0 / (w * w)
        s = 0.0
        for cc in reversed(coef):
            s = s * q + cc
        got = s / w
        ref = mills_ref([w])[0]
        assert abs(got - ref) / ref < 4e-16
