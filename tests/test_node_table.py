"""The tabulated LBR node (csrc/node_table.inc), checked on the CPU.

The device reads, for w = sqrt|ln(F/K)| < 64, the degree-6 float polynomials of the interval
picked by the bit pattern of w (as a float) and evaluates them in float by Horner's rule. This
test repeats that in numpy float32 and compares with the node computed from the definitions in
40-digit mpmath: e = erfcx(w), s_l = s_c - sqrt(pi/2)(1 - e), s_u = s_c + sqrt(pi/2)(1 + e)
(s_c = sqrt 2 w), b_l = b(-u, s_l), b_max - b_u, and b_s at both nodes (appendix stage 4).
"""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_17065_gb300", "csrc",
                   "node_table.inc")
DEG = 6


def table():
    text = open(INC).read()
    rows = re.findall(r"\{([^{}]+)\}", text.split("=", 1)[1])
    return np.array([[np.float32(v.strip().rstrip("f")) for v in r.split(",")] for r in rows], dtype=np.float32)


def interval_index(w):
    bits = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.int64)
    return np.maximum((bits >> 20) - ((127 - 6) << 3) + 1, 0)


def eval_table(C, w):
    w = np.asarray(w, dtype=np.float32)
    c = C[interval_index(w)]
    tau = (w * c[:, 0] + c[:, 1]).astype(np.float32)
    out = []
    for f in range(6):
        cf = c[:, 2 + f * (DEG + 1): 2 + (f + 1) * (DEG + 1)]
        v = cf[:, DEG].copy()
        for k in range(DEG - 1, -1, -1):
            v = (v * tau + cf[:, k]).astype(np.float32)
        out.append(v.astype(np.float64))
    return out, tau


def node_ref(w):
    """e, s_l / u, b_l / (b_max u), b_s(s_l) / b_max, (b_max - b_u) / b_max, b_s(s_u) / b_max."""
    with mp.workdps(40):
        w = mp.mpf(float(w))
        u = w * w
        c = mp.sqrt(mp.pi / 2)
        e = mp.erfc(w) * mp.exp(u)
        sc = mp.sqrt(2) * w
        sl = sc - c * (1 - e)
        su = sc + c * (1 + e)
        x = -u
        bm = mp.exp(x / 2)
        b = lambda s: mp.exp(x / 2) * mp.ncdf(x / s + s / 2) - mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)  # noqa
        bc = lambda s: mp.exp(x / 2) * mp.ncdf(-x / s - s / 2) + mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)  # noqa
        bs = lambda s: mp.exp(-x * x / (2 * s * s) - s * s / 8) / mp.sqrt(2 * mp.pi)  # noqa
        return [float(v) for v in (e, sl / u, b(sl) / (bm * u), bs(sl) / bm, bc(su) / bm, bs(su) / bm)]


def test_index_and_bounds():
    C = table()
    assert C.shape == (97, 2 + 6 * (DEG + 1))
    lo = np.concatenate([[0.0], [2.0 ** e * (1 + m / 8) for e in range(-6, 6) for m in range(8)]]).astype(np.float32)
    assert np.array_equal(interval_index(lo), np.arange(97))
    assert np.array_equal(interval_index(np.nextafter(lo[1:], np.float32(0))), np.arange(96))
    _, tau = eval_table(C, np.concatenate([lo, np.nextafter(lo[1:], np.float32(0)), [np.float32(63.99)]]))
    assert np.all(tau >= -1.0) and np.all(tau <= 1.0)
    assert np.all(np.frexp(C[:, 0])[0] == 0.5) and np.all(C[:, 1] == np.round(C[:, 1]))


def test_table_matches_the_node_definitions():
    C = table()
    rng = np.random.default_rng(7)
    w = np.concatenate([np.exp(rng.uniform(np.log(1e-3), np.log(63.9), 300)), rng.uniform(0, 64, 100),
                        [1e-3, 1.0 / 64, 1.0, 8.0, 37.6]]).astype(np.float32)
    got, _ = eval_table(C, w)
    ref = np.array([node_ref(x) for x in w])
    for f in range(6):
        rel = np.abs(got[f] - ref[:, f]) / np.abs(ref[:, f])
        assert rel.max() < 4e-7, (f, rel.max())


def test_small_u_limits():
    """As u -> 0: e -> 1, s_l / u -> sqrt(pi/2), and the node's ratios tend to finite limits."""
    C = table()
    got, _ = eval_table(C, np.array([0.0, 1e-6], np.float32))
    assert abs(got[0][0] - 1.0) < 1e-6
    assert abs(got[1][0] - np.sqrt(np.pi / 2)) < 1e-6 * np.sqrt(np.pi / 2)
    ref = node_ref(1e-6)
    for f in range(6):
        assert abs(got[f][1] - ref[f]) <= 4e-7 * abs(ref[f])
