"""High-precision reference values (mpmath) used to pin the oracle.

Independent of the oracle: everything here is the textbook definition written
in arbitrary precision -- the normalised Black function as the difference of
normal CDFs (Eq. app_normalized_black), its complement as the sum of two
normal tails, the implied volatility by bisection of that definition
(Eq. iv_inverse_problem), and the adjoint by central finite differences of the
high-precision root (checks Eq. implicit_iv / method_vjp).  Only the CPU pin
tests use it; mpmath is not needed anywhere else.
"""
from __future__ import annotations

import mpmath as mp


def b(x, s):
    """b(x,s) = e^{x/2} Phi(x/s + s/2) - e^{-x/2} Phi(x/s - s/2)."""
    x, s = mp.mpf(x), mp.mpf(s)
    return mp.e ** (x / 2) * mp.ncdf(x / s + s / 2) - mp.e ** (-x / 2) * mp.ncdf(x / s - s / 2)


def b_complement(x, s):
    """e^{x/2} - b(x,s) = e^{x/2} Phi(-x/s - s/2) + e^{-x/2} Phi(x/s - s/2) (no cancellation)."""
    x, s = mp.mpf(x), mp.mpf(s)
    return mp.e ** (x / 2) * mp.ncdf(-x / s - s / 2) + mp.e ** (-x / 2) * mp.ncdf(x / s - s / 2)


def price(F, K, T, sigma, theta):
    """Undiscounted Black-76 price (r = 0), Eq. app_black76, straight from the definition."""
    F, K, T, sigma = map(mp.mpf, (F, K, T, sigma))
    s = sigma * mp.sqrt(T)
    d1 = (mp.log(F / K) + s * s / 2) / s
    d2 = d1 - s
    if theta > 0:
        return F * mp.ncdf(d1) - K * mp.ncdf(d2)
    return K * mp.ncdf(-d2) - F * mp.ncdf(-d1)


def vega(F, K, T, sigma):
    F, K, T, sigma = map(mp.mpf, (F, K, T, sigma))
    s = sigma * mp.sqrt(T)
    d1 = (mp.log(F / K) + s * s / 2) / s
    return F * mp.npdf(d1) * mp.sqrt(T)


def implied_vol(F, K, T, P, theta, iters: int = 200, lo_sigma="1e-12"):
    """Root of price(sigma) = P by bisection in ln(sigma) (the price is increasing in sigma).

    Works on the inputs exactly as given (decimal values of the doubles), so it
    is the exact real root for those doubles, to about (bracket width in ln
    sigma) * 2^-iters relative.  The bracket is [lo_sigma, 1e4]; roots of deep
    lower-tail prices need a floor far below the default.  Returns None outside
    the open no-arbitrage interval.
    """
    F, K, T, P = map(mp.mpf, (F, K, T, P))
    intrinsic = max(F - K, 0) if theta > 0 else max(K - F, 0)
    upper = F if theta > 0 else K
    if not (intrinsic < P < upper):
        return None
    lo, hi = mp.log(mp.mpf(lo_sigma)), mp.log(mp.mpf("1e4"))
    ax = abs(mp.log(F / K))
    for _ in range(iters):
        mid = (lo + hi) / 2
        # |ln(F/K)| / s > 1e4: the time value is below exp(-5e7), far under any positive
        # double difference P - intrinsic (and mpmath's erfc would overflow there)
        if ax > 0 and ax > 1e4 * mp.e ** mid * mp.sqrt(T):
            lo = mid
        elif price(F, K, T, mp.e ** mid, theta) < P:
            lo = mid
        else:
            hi = mid
    return mp.e ** ((lo + hi) / 2)


def iv_gradient_fd(F, K, T, P, theta, rel_h=mp.mpf("1e-15")):
    """Central finite differences of the high-precision root in (P, F, K, T).

    Needs mp.mp.dps high enough that the bisection's accuracy (about
    2^-iters) is far below rel_h^2.
    """
    F, K, T, P = map(mp.mpf, (F, K, T, P))
    base = (F, K, T, P)
    out = []
    for j in (3, 0, 1, 2):  # P, F, K, T
        h = base[j] * rel_h
        up = list(base)
        dn = list(base)
        up[j] += h
        dn[j] -= h
        s_up = implied_vol(*up, theta)
        s_dn = implied_vol(*dn, theta)
        out.append((s_up - s_dn) / (2 * h))
    return out  # d sigma / d(P, F, K, T)


def bs_price(S, K, T, r, q, sigma, theta):
    """Discounted Black-Scholes price, Eq. app_black_scholes in spot coordinates (put by the
    direct put formula, not parity)."""
    S, K, T, r, q, sigma = map(mp.mpf, (S, K, T, r, q, sigma))
    s = sigma * mp.sqrt(T)
    d1 = (mp.log(S / K) + (r - q) * T + s * s / 2) / s
    d2 = d1 - s
    if theta > 0:
        return S * mp.e ** (-q * T) * mp.ncdf(d1) - K * mp.e ** (-r * T) * mp.ncdf(d2)
    return K * mp.e ** (-r * T) * mp.ncdf(-d2) - S * mp.e ** (-q * T) * mp.ncdf(-d1)


def bs_implied_vol(S, K, T, r, q, V, theta, iters: int = 200):
    """Root of bs_price(sigma) = V by bisection in ln(sigma); None outside the price interval."""
    S, K, T, r, q, V = map(mp.mpf, (S, K, T, r, q, V))
    lo_p = bs_price(S, K, T, r, q, mp.mpf("1e-30"), theta)
    hi_p = bs_price(S, K, T, r, q, mp.mpf("1e6"), theta)
    if not (lo_p < V < hi_p):
        return None
    lo, hi = mp.log(mp.mpf("1e-12")), mp.log(mp.mpf("1e4"))
    for _ in range(iters):
        mid = (lo + hi) / 2
        if bs_price(S, K, T, r, q, mp.e ** mid, theta) < V:
            lo = mid
        else:
            hi = mid
    return mp.e ** ((lo + hi) / 2)


def bs_iv_gradient_fd(S, K, T, r, q, V, theta, h=mp.mpf("1e-20")):
    """Central differences of the high-precision root in (V, S, K, T, r, q); steps are
    relative for V, S, K, T and absolute for r, q."""
    base = [mp.mpf(a) for a in (V, S, K, T, r, q)]
    out = []
    for j in range(6):
        step = h * (base[j] if j < 4 else 1)
        up, dn = list(base), list(base)
        up[j] += step
        dn[j] -= step
        s_up = bs_implied_vol(up[1], up[2], up[3], up[4], up[5], up[0], theta)
        s_dn = bs_implied_vol(dn[1], dn[2], dn[3], dn[4], dn[5], dn[0], theta)
        out.append((s_up - s_dn) / (2 * step))
    return out  # d sigma / d(V, S, K, T, r, q)
