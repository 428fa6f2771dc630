"""The FP64 erfcx table behind the Mills ratio (csrc/erfcx_table.inc), checked on the CPU.

The device code evaluates, for 0 <= a < 64, the degree-9 polynomial of the
interval picked by the bit pattern of a (interval 0 = [0, 1/16); from 1/16 on,
16 equal parts per binade), in tau = a * scale + offset, by Horner's rule in
double; this test repeats the index arithmetic on the bit patterns and the
evaluation in numpy and compares with erfcx in 50-digit mpmath, and checks the
asymptotic series used from 64 on.
"""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_17065_gb300", "csrc",
                   "erfcx_table.inc")


def table():
    text = open(INC).read()
    rows = re.findall(r"\{([^{}]+)\}", text.split("=", 1)[1])
    return np.array([[float(v) for v in r.split(",")] for r in rows])


def interval_index(a):
    """The device's index: the biased exponent and top four mantissa bits, less those of 1/16, plus one."""
    bits = np.asarray(a, dtype=np.float64).view(np.uint64) & np.uint64(0x7fffffffffffffff)
    raw = (bits >> np.uint64(48)).astype(np.int64)
    return np.maximum(raw - ((1023 - 4) << 4) + 1, 0)


def eval_table(C, a):
    c = C[interval_index(a)]
    tau = a * c[:, 10] + c[:, 11]
    v = c[:, 9].copy()
    for k in range(8, -1, -1):
        v = v * tau + c[:, k]
    return v, tau


def test_interval_index_and_bounds():
    C = table()
    assert C.shape == (161, 12)
    # the index of each interval's left end is that interval, and tau runs over [-1, 1) on it
    lo = np.concatenate([[0.0], [2.0 ** e * (1 + m / 16) for e in range(-4, 6) for m in range(16)]])
    assert np.array_equal(interval_index(lo), np.arange(161))
    assert np.array_equal(interval_index(np.nextafter(lo[1:], 0)), np.arange(160))
    assert interval_index(np.array([np.nextafter(64.0, 0)]))[0] == 160
    a = np.concatenate([lo, np.nextafter(lo[1:], 0), [np.nextafter(64.0, 0), 5e-324, 1e-300, -0.0]])
    _, tau = eval_table(C, np.abs(a))
    assert np.all(tau >= -1.0) and np.all(tau <= 1.0)
    # scale is a power of two and offset an integer: tau = a scale + offset rounds once
    assert np.all(np.frexp(C[:, 10])[0] == 0.5) and np.all(C[:, 11] == np.round(C[:, 11]))


def test_table_matches_erfcx_to_a_few_ulp():
    C = table()
    rng = np.random.default_rng(0)
    a = np.concatenate([np.linspace(0, 64, 4001)[:-1], rng.uniform(0, 64, 2000), np.exp(rng.uniform(-12, np.log(64), 2000)),
                        [0.0, 1.0 / 16, np.nextafter(1.0 / 16, 0), np.nextafter(64.0, 0), 1e-300]])
    a = a[a < 64]
    got, _ = eval_table(C, a)
    with mp.workdps(50):
        ref = np.array([float(mp.erfc(x) * mp.exp(mp.mpf(x) ** 2)) for x in a])
    assert np.max(np.abs(got - ref) / ref) < 4e-16


def test_asymptotic_series_beyond_64():
    coef = [1.0, -1.0, 3.0, -15.0, 105.0, -945.0, 10395.0, -135135.0, 2027025.0, -34459425.0]
    for a in [64.0, 64.5, 100.0, 1e3, 1e8]:
        w = 0.5 / (a * a)
        s = 0.0
        for cc in reversed(coef):
            s = s * w + cc
        got = s / a * 0.564189583547756286948
        with mp.workdps(50):
            ref = float(mp.erfc(a) * mp.exp(mp.mpf(a) ** 2))
        assert abs(got - ref) / ref < 4e-16
