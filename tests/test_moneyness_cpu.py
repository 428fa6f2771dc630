"""The solver's moneyness (x = -|ln(F/K)|, b_max = sqrt(min/max), rsq = 1/sqrt(F K)) from one
reciprocal square root, replayed on the CPU in IEEE double and checked against 50-digit mpmath.

The kernels take rsq = 1/sqrt(F K), b_max = min(F, K) rsq and r = b_max^2 (min/max to a few ulps),
then ln(min/max) = ln r + (min - r max)/min with the residual exact through one fma and
1/min = rsq^2 max (Section 2's normalisation, x = ln(F/K) in the out-of-the-money form).  Each
operation here is one IEEE rounding (numpy), the fma and the reciprocal square root are rounded
once from exact values, and ln r is the correctly rounded logarithm (the device's is within 1 ulp).
A dropped or sign-flipped residual, or b_max from max instead of min, fails the bound.
"""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def rnd(v):
    return float(v)  # mpmath value -> nearest double


def replay(F, K):
    mp.mp.dps = 50
    mn, mx = (K, F) if F > K else (F, K)
    p = F * K
    rsq = rnd(1 / mp.sqrt(mp.mpf(p)))
    bmax = mn * rsq
    r = bmax * bmax
    res = rnd(mp.mpf(mn) - mp.mpf(r) * mp.mpf(mx))  # fma(-r, mx, mn)
    c = res * ((rsq * rsq) * mx)
    x = -abs(rnd(mp.log(mp.mpf(r))) + c)
    return x, bmax, rsq


@pytest.mark.parametrize("seed", [0, 1])
def test_moneyness_against_mpmath(seed):
    mp.mp.dps = 50
    rng = np.random.default_rng(seed)
    F = 10.0 ** rng.uniform(-3, 5, 400)
    k = np.concatenate([rng.uniform(-6, 6, 200), rng.uniform(-1e-6, 1e-6, 100), rng.uniform(-1e-14, 1e-14, 60),
                        np.zeros(20), rng.uniform(-300, 300, 20)])
    K = F * np.exp(k)
    for f, kk in zip(F, K):
        x, bmax, rsq = replay(float(f), float(kk))
        ex = -abs(mp.log(mp.mpf(float(f)) / mp.mpf(float(kk))))
        eb = mp.sqrt(mp.mpf(float(min(f, kk))) / mp.mpf(float(max(f, kk))))
        # x within 2 ulp of its own size plus the first-order remainder c^2/2 (|c| <~ 2^-50)
        assert abs(mp.mpf(x) - ex) <= 2 * np.spacing(abs(float(ex))) + mp.mpf(2) ** -100, (f, kk, x, ex)
        assert x <= 0.0
        assert abs(mp.mpf(bmax) - eb) <= 2.5 * np.spacing(float(eb)), (f, kk)
        assert abs(mp.mpf(rsq) - 1 / mp.sqrt(mp.mpf(float(f)) * mp.mpf(float(kk)))) <= 1.5 * np.spacing(rsq)


def test_at_the_money_is_zero():
    for f in (1e-3, 0.7, 100.0, 3e4):
        x, bmax, _ = replay(f, f)
        assert x == 0.0 or abs(x) <= 2.0 ** -100
        assert abs(bmax - 1.0) <= 2 * np.spacing(1.0)
