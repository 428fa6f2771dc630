"""The solver's stage-1 time value, checked on the CPU against exact rational arithmetic.

In the money (U = a > b, intrinsic a - b) the kernels form the time value P - a + b with three
FP64 additions and no branch: P + (b - a) when a <= 2b, (P - a) + b otherwise, and a fixed
negative value when a > 2b and P < a/2 (then P < a/2 < a - b).  U - P is -(P - a).  This test
repeats those operations in IEEE double (numpy rounds each addition to nearest, as the GPU
does) and checks against fractions.Fraction: the row status (the signs of tv and U - P, and
which of them is zero) is exact on every row, and tv is within half an ulp of the exact value
on every price at or above a/2 (Section 3.1 stage 1: the status decides NaN, 0 or +inf).
"""
from fractions import Fraction

import numpy as np


def device_tv(P, a, b):
    a, b, P = np.float64(a), np.float64(b), np.float64(P)
    d = P - a
    near = a <= 2.0 * b
    tv = (P if near else d) + ((b - a) if near else b)
    itm = a > b
    if not itm:
        tv = P
    elif not near and a > 2.0 * P:
        tv = np.float64(-1.0)
    return tv, -d


def status_of(tv, cv):
    if tv < 0:
        return 1
    if cv < 0:
        return 2
    if tv == 0:
        return 4
    if cv == 0:
        return 5
    return 0


def exact(P, a, b):
    P, a, b = Fraction(float(P)), Fraction(float(a)), Fraction(float(b))
    tv = P - a + b if a > b else P
    return tv, a - P


def _cases(rng, n):
    out = []
    for _ in range(n):
        b = float(np.exp(rng.uniform(-20, 20)))
        a = b * float(np.exp(rng.uniform(-8, 8)))
        lo, hi = max(a - b, 0.0), a
        kind = rng.integers(0, 6)
        if kind == 0:
            P = lo  # at the intrinsic value
        elif kind == 1:
            P = np.nextafter(lo, 0.0)  # one ulp below it
        elif kind == 2:
            P = np.nextafter(lo, np.inf)  # one ulp above it
        elif kind == 3:
            P = rng.uniform(lo, hi)  # inside the interval
        elif kind == 4:
            P = rng.uniform(0.0, lo) if lo > 0 else 0.0  # below it
        else:
            P = hi * float(rng.choice([1.0, 1.0 + 2 ** -52, 1.0 - 2 ** -53, 3.0]))  # at or past the upper bound
        out.append((float(P), a, b))
    # operands that make a - b or P - a cancel, and a, b on either side of a = 2b
    for a, b in ((1.0, 0.5), (1.0, np.nextafter(0.5, 0)), (1.0, np.nextafter(0.5, 1)), (3.0, 1.0), (1.0 + 2 ** -52, 1.0)):
        for P in (a - b, np.nextafter(a - b, 0), np.nextafter(a - b, 2), a / 2, np.nextafter(a / 2, 0), a, 0.0):
            out.append((float(P), float(a), float(b)))
    return out


def test_status_exact_and_value_rounded_once():
    rng = np.random.default_rng(41)
    for P, a, b in _cases(rng, 20000):
        tv, cv = device_tv(P, a, b)
        etv, ecv = exact(P, a, b)
        want = status_of(etv, ecv)
        assert status_of(tv, cv) == want, (P, a, b, tv, cv)
        assert Fraction(float(cv)) == ecv or abs(Fraction(float(cv)) - ecv) <= abs(ecv) * Fraction(1, 2 ** 53)
        if want == 0 and not (a > b and a > 2 * b and P < a / 2):
            # one rounding: within half an ulp of the exact time value
            err = abs(Fraction(float(tv)) - etv)
            assert err <= Fraction(float(np.spacing(abs(float(etv))))) / 2, (P, a, b)


def test_twice_pos_bit_rule():
    """2v from the bit pattern: subnormals double their integer, normals gain an exponent, and
    the top binade goes to +inf; against exact doubling in numpy."""
    def twice_bits(v):
        bits = np.array([v], dtype=np.float64).view(np.int64)[0]
        e = int(bits) >> 52
        r = (int(bits) << 1) if e == 0 else (0x7ff0000000000000 if e >= 2046 else int(bits) + (1 << 52))
        return np.array([r], dtype=np.int64).view(np.float64)[0]
    for v in (0.0, 5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308, 1.0, 3.5, 8.98846567431158e307,
              np.nextafter(8.98846567431158e307, 0), 1.7976931348623157e308):
        with np.errstate(over="ignore"):
            assert twice_bits(v) == np.float64(v) * 2.0, v
