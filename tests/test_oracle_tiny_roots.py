"""Pins for the oracle's tiny-root regime: prices far down the lower tail.

The oracle's root bracket descends from s = 1 by squaring its upper end while
the lower end is still 0, so that roots of ~1e-300 (and subnormal ones) are
reached within its iteration cap.  These tests tie that regime to values
fixed outside the oracle:
  * at the money b(0, s) = erf(s / (2 sqrt 2)) (Eq. app_normalized_black at
    k = 0), so sigma = 2 sqrt 2 erfinv(beta) / sqrt(T) exactly, for beta down
    to 1e-300 and subnormal prices;
  * away from the money, the root of the Black-76 price (Eq. app_black76) by
    bisection of the definition in 60-digit arithmetic, on deep lower-tail
    quotes (beta < 1e-30, |ln(F/K)| up to 6, beta down to subnormal);
and plant mistakes in the bracket logic that these pins must catch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_17065_gb300 import workloads

mp = pytest.importorskip("mpmath")
import mp_reference as R  # noqa: E402

EPS = float(np.finfo(np.float64).eps)
TINY = 4.9406564584124654e-324  # one subnormal ulp


def atm_rows():
    """ATM quotes whose time value is tiny: P / F from 1e-30 down to the subnormal range."""
    P = np.array([1e-28, 1e-98, 1e-198, 1e-298, 1e-300, 1e-303, 1e-306, 2.5e-308, 1e-310, 3e-313, 1e-315,
                  7e-318, 1e-320])
    T = np.resize(np.array([1.0, 0.25, 3.0, 1e-2, 1.0 / 365.0]), P.size)
    flag = np.resize(np.array([1, -1], np.int8), P.size)
    F = np.full(P.size, 100.0)
    return F, F.copy(), T, P, flag


def check_atm_tiny(orc):
    """Largest error of the oracle against the ATM closed form, in units of its tolerance."""
    F, K, T, P, flag = atm_rows()
    sig, st = orc.implied_vol(F, K, T, P, flag)
    if not np.all(st == 0):
        return np.inf
    worst = 0.0
    for i in range(P.size):
        with mp.workdps(50):
            beta = mp.mpf(P[i]) / mp.mpf(F[i])
            ref = 2 * mp.sqrt(2) * mp.erfinv(beta) / mp.sqrt(T[i])
        # relative rounding, plus the quantisation of s and of s / sqrt(T) once they are subnormal
        tol = 8 * EPS * float(ref) + 2 * TINY * (1 + 1 / math.sqrt(T[i]))
        worst = max(worst, abs(sig[i] - float(ref)) / tol)
    return worst


def test_iv_atm_closed_form_tiny_prices():
    assert check_atm_tiny(oracle.default()) <= 1.0


def deep_tail_rows(n_stress=4000, seed=23):
    """Lower-tail quotes with beta < 1e-30: stress-distribution rows priced by the oracle's
    (separately pinned) Black price, plus out-of-the-money quotes built at fixed beta from
    1e-250 to subnormal, whose prices need no pricer at all."""
    b = workloads.stress_batch(n_stress, seed=seed, boundary_frac=0.0)
    P, _ = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    itm = np.where(b.flag > 0, np.maximum(b.F - b.K, 0.0), np.maximum(b.K - b.F, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        beta = (P - itm) / np.sqrt(b.F * b.K)
    pick = np.flatnonzero((beta > 0) & (beta < 1e-30) & (itm == 0))[:200]
    F, K, T, flag, P = [b.F[pick]], [b.K[pick]], [b.T[pick]], [b.flag[pick]], [P[pick]]
    xs = np.array([-6.0, -3.0, -1.0, -0.3, -0.05, -1e-3])
    betas = np.array([1e-250, 1e-300, 1e-305, 1e-310, 1e-318])
    for x in xs:
        for bt in betas:
            Fi, Ki = 100.0, 100.0 * math.exp(-x)  # K > F: an out-of-the-money call ...
            for fl, (f, k) in ((1, (Fi, Ki)), (-1, (Ki, Fi))):  # ... and the mirrored put
                F.append([f]); K.append([k]); T.append([0.5]); flag.append([fl])
                P.append([bt * math.sqrt(f * k)])
    cat = lambda a: np.concatenate([np.asarray(v, dtype=np.asarray(a[0]).dtype) for v in a])  # noqa: E731
    return (cat(F).astype(np.float64), cat(K).astype(np.float64), cat(T).astype(np.float64),
            cat(P).astype(np.float64), cat(flag).astype(np.int8))


_DEEP = {}


def deep_tail_reference():
    """The rows and their 60-digit roots, computed once per session."""
    if not _DEEP:
        F, K, T, P, flag = deep_tail_rows()
        refs, kaps = [], []
        for i in range(F.size):
            with mp.workdps(60):
                ref = R.implied_vol(F[i], K[i], T[i], P[i], int(flag[i]), iters=110, lo_sigma="1e-320")
                # conditioning of sigma in the time value: tv / (sigma V), all in 60 digits
                itm = max(mp.mpf(F[i]) - mp.mpf(K[i]), 0) if flag[i] > 0 else max(mp.mpf(K[i]) - mp.mpf(F[i]), 0)
                kap = (mp.mpf(P[i]) - itm) / (ref * R.vega(F[i], K[i], T[i], ref))
            refs.append(ref)
            kaps.append(float(kap))
        _DEEP.update(rows=(F, K, T, P, flag), refs=refs, kaps=np.array(kaps))
    return _DEEP["rows"], _DEEP["refs"], _DEEP["kaps"]


def check_deep_tail(orc):
    (F, K, T, P, flag), refs, kaps = deep_tail_reference()
    sig, st = orc.implied_vol(F, K, T, P, flag)
    if not np.all(st == 0):
        return np.inf
    worst = 0.0
    for i in range(F.size):
        tol = 16 * EPS * (1 + kaps[i])
        worst = max(worst, abs(sig[i] - float(refs[i])) / (tol * float(refs[i])))
    return worst


def test_deep_lower_tail_against_high_precision_bisection():
    (F, K, T, P, flag), _, kaps = deep_tail_reference()
    itm = np.where(flag > 0, np.maximum(F - K, 0.0), np.maximum(K - F, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        beta = (P - itm) / np.sqrt(F * K)
    assert F.size >= 250 and np.all(beta < 1e-30)
    assert np.sum(beta < 1e-300) >= 30 and np.sum(np.abs(np.log(F / K)) > 5) >= 20
    # deep in the lower region sigma is well conditioned in the price (d ln s / d ln beta = s^2/x^2)
    assert np.all(kaps < 1.0)
    assert check_deep_tail(oracle.default()) <= 1.0


BRACKET_MUTATIONS = [
    ("upper end halved instead of squared", "else if (isfinite(hi)) sn = hi < 0.5 ? hi * hi : 0.5 * hi;",
     "else if (isfinite(hi)) sn = 0.5 * hi;"),
    ("absolute Newton stopping test", "if (newton_ok && fabs(sn - s) <= 2.0 * DBL_EPSILON * s) return sn;",
     "if (newton_ok && fabs(sn - s) <= 2.0 * DBL_EPSILON) return sn;"),
    ("absolute bracket-width test", "if (isfinite(hi) && hi - lo <= 4.0 * DBL_EPSILON * hi) return 0.5 * (lo + hi);",
     "if (isfinite(hi) && hi - lo <= 4.0 * DBL_EPSILON) return 0.5 * (lo + hi);"),
]


@pytest.mark.parametrize("name,old,new", BRACKET_MUTATIONS, ids=[m[0] for m in BRACKET_MUTATIONS])
def test_planted_bracket_mistakes_are_caught(tmp_path, name, old, new):
    src = oracle.source_text()
    assert old in src, name
    bad = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libbad.so"))
    assert check_atm_tiny(bad) > 1.0 or check_deep_tail(bad) > 1.0, name
