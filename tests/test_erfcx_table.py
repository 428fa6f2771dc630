"""The FP64 erfcx table behind the Mills ratio (csrc/erfcx_table.inc), checked on the CPU.

The device code evaluates, for 0 <= a < 16, the degree-9 polynomial of
interval floor(8a) in tau = 16 (a - i/8) - 1 by Horner's rule in double; this
test repeats that evaluation in numpy and compares with erfcx in 50-digit
mpmath, and checks the asymptotic series used beyond 16.
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


def eval_table(C, a):
    fi = np.floor(a * 8.0)
    tau = (a - fi * 0.125) * 16.0 - 1.0
    c = C[fi.astype(int)]
    v = c[:, 9].copy()
    for k in range(8, -1, -1):
        v = v * tau + c[:, k]
    return v


def test_table_matches_erfcx_to_a_few_ulp():
    C = table()
    assert C.shape == (128, 10)
    a = np.concatenate([np.linspace(0, 16, 4001)[:-1], np.random.default_rng(0).uniform(0, 16, 2000)])
    got = eval_table(C, a)
    with mp.workdps(50):
        ref = np.array([float(mp.erfc(x) * mp.exp(mp.mpf(x) ** 2)) for x in a])
    assert np.max(np.abs(got - ref) / ref) < 4e-16


def test_asymptotic_series_beyond_16():
    coef = [1.0, -1.0, 3.0, -15.0, 105.0, -945.0, 10395.0, -135135.0, 2027025.0, -34459425.0]
    for a in [16.0, 16.5, 20.0, 50.0, 1e3, 1e8]:
        w = 0.5 / (a * a)
        s = 0.0
        for cc in reversed(coef):
            s = s * w + cc
        got = s / a * 0.564189583547756286948
        with mp.workdps(50):
            ref = float(mp.erfc(a) * mp.exp(mp.mpf(a) ** 2))
        assert abs(got - ref) / ref < 4e-16
