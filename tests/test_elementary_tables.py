"""The table-driven FP64 log and exp of the device code (csrc/elementary_tables.inc,
P. T. P. Tang's method), checked on the CPU: the tables against mpmath, and the method --
the device functions' operations replayed in float64 with exact fused multiply-adds --
against mpmath to within 1 ulp, near 1 for the logarithm included."""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

INC = os.path.join(os.path.dirname(__file__), "..", "paper_2606_17065_gb300", "csrc", "elementary_tables.inc")
MAGIC = 6755399441055744.0


def _tables():
    src = open(INC).read()

    def arr(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return np.array([float(x) for x in body.replace("\n", "").split(",") if x.strip()])

    def const(name):
        return float(re.search(name + r" = ([^;]+);", src).group(1))

    return ({k: arr(k) for k in ("kLogInvC", "kLogCHi", "kLogCLo", "kExp2Hi", "kExp2Lo")},
            {k: const(k) for k in ("kLn2Hi", "kLn2Lo", "kLn2By128Hi", "kLn2By128Lo", "k128ByLn2")})


def fma(a, b, c):
    return np.array([float(mp.mpf(x) * mp.mpf(y) + mp.mpf(z)) for x, y, z in np.broadcast(a, b, c)])


def dlog(v, t, c):
    b = v.view(np.int64)
    e = ((b >> 52) & 0x7ff) - 1023
    m = ((b & 0x000fffffffffffff) | (1023 << 52)).view(np.float64)
    tr = fma(m - 1.0, 1024.0, MAGIC)
    j = tr.view(np.int64) & 0x7ff
    jd = tr - MAGIC
    f = (m - fma(jd, 0.0009765625, 1.0)) * t["kLogInvC"][j]
    q = np.full_like(f, 0.2)
    for k in (-0.25, 1.0 / 3.0, -0.5, 1.0):
        q = fma(q, f, k)
    ed = e.astype(np.float64)
    hi = fma(ed, c["kLn2Hi"], t["kLogCHi"][j])
    lo = fma(ed, c["kLn2Lo"], t["kLogCLo"][j]) + q * f
    return hi + lo


def dexp(v, t, c):
    tr = fma(v, c["k128ByLn2"], MAGIC)
    n = tr.view(np.int64) & 0xffffffff
    n = np.where(n >= 2 ** 31, n - 2 ** 32, n)
    fn = tr - MAGIC
    r = fma(-fn, c["kLn2By128Hi"], v)
    r = fma(-fn, c["kLn2By128Lo"], r)
    p = np.full_like(r, 1.0 / 120.0)
    for k in (1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0):
        p = fma(p, r, k)
    p = p * r
    k = n & 127
    res = fma(t["kExp2Hi"][k], p, t["kExp2Lo"][k]) + t["kExp2Hi"][k]
    return (res.view(np.int64) + ((n >> 7).astype(np.int64) << 52)).view(np.float64)


def test_tables_against_mpmath():
    t, c = _tables()
    mp.mp.dps = 40
    assert len(t["kLogInvC"]) == len(t["kLogCHi"]) == len(t["kLogCLo"]) == 1025
    for j in range(1025):
        cj = 1 + mp.mpf(j) / 1024
        assert t["kLogInvC"][j] == float(1 / cj)
        # hi + lo within the rounding of lo
        assert abs(mp.mpf(t["kLogCHi"][j]) + mp.mpf(t["kLogCLo"][j]) - mp.log(cj)) <= abs(t["kLogCLo"][j]) * 2.0 ** -52 + mp.mpf(2) ** -120
        assert float(t["kLogCHi"][j] * 2 ** 43) == int(t["kLogCHi"][j] * 2 ** 43)  # a multiple of 2^-43
    for k in range(128):
        assert abs(mp.mpf(t["kExp2Hi"][k]) + mp.mpf(t["kExp2Lo"][k]) - mp.mpf(2) ** (mp.mpf(k) / 128)) <= abs(t["kExp2Lo"][k]) * 2.0 ** -52 + mp.mpf(2) ** -120
    assert abs(mp.mpf(c["kLn2Hi"]) + mp.mpf(c["kLn2Lo"]) - mp.log(2)) <= abs(c["kLn2Lo"]) * 2.0 ** -52
    assert abs(mp.mpf(c["kLn2By128Hi"]) + mp.mpf(c["kLn2By128Lo"]) - mp.log(2) / 128) <= abs(c["kLn2By128Lo"]) * 2.0 ** -52
    # the high parts are short enough for exact products with any exponent / reduction count
    assert float(c["kLn2Hi"] * 2 ** 43) == int(c["kLn2Hi"] * 2 ** 43)
    assert float(c["kLn2By128Hi"] * 2 ** 42) == int(c["kLn2By128Hi"] * 2 ** 42)


def test_method_within_one_ulp():
    t, c = _tables()
    mp.mp.dps = 40
    rng = np.random.default_rng(0)
    v = np.concatenate([10.0 ** rng.uniform(-300, 300, 400), 1 + rng.uniform(-1e-3, 1e-3, 200),
                        # each side of every 32nd table node (the reduction's rounding boundaries)
                        (1 + (np.arange(0, 1025, 32) + 0.5) / 1024) * np.array([1.0]).repeat(33),
                        (1 + (np.arange(0, 1025, 32) - 0.5) / 1024)[1:],
                        1 + rng.uniform(-1e-13, 1e-13, 100), rng.uniform(0.5, 2.0, 200),
                        np.array([1.0, 2.0, 0.5, np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0), 2.2250738585072014e-308])])
    got = dlog(v, t, c)
    ref = np.array([float(mp.log(mp.mpf(x))) for x in v])
    nz = ref != 0
    assert np.all(got[~nz] == 0.0)
    assert np.max(np.abs(got[nz] - ref[nz]) / np.spacing(np.abs(ref[nz]))) <= 1.0
    x = np.concatenate([rng.uniform(-707.9, 707.9, 400), rng.uniform(-1, 1, 200), rng.uniform(-1e-9, 1e-9, 100),
                        np.array([0.0, 1.0, -1.0, 707.5, -707.5])])
    got = dexp(x, t, c)
    ref = np.array([float(mp.exp(mp.mpf(a))) for a in x])
    assert np.max(np.abs(got - ref) / np.spacing(ref)) <= 1.0
