"""Pins for the CPU oracle: checks against things other than itself.

Each test ties one oracle function to something the paper or mathematics
fixes -- the definition in arbitrary precision, a closed form, a limit, an
invariant or a library routine -- and the last test plants plausible
mistakes in copies of the oracle and checks that these pins catch them.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sps

import oracle
from paper_2606_17065_gb300 import workloads

mp = pytest.importorskip("mpmath")
import mp_reference as R  # noqa: E402

EPS = np.finfo(np.float64).eps


def _points(seed, n):
    rng = np.random.default_rng(seed)
    xs = -(10.0 ** rng.uniform(-10, 1.3, n))
    xs[: n // 10] = 0.0
    ss = 10.0 ** rng.uniform(-4, 1.7, n)
    return xs, ss


def check_b(orc, n=160, seed=3):
    """b and b_max - b against the definition at 60 and 90 digits.

    The tolerance grows with the exponent A + B = x^2/(2 s^2) + s^2/8: a
    relative rounding of x or s moves b by that factor times itself, which is
    the conditioning of b, not an error of the method.
    """
    xs, ss = _points(seed, n)
    worst = 0.0
    for x, s in zip(xs, ss):
        A = 0.5 * (x / s) ** 2 + s * s / 8
        with mp.workdps(60):
            r60, c60 = R.b(x, s), R.b_complement(x, s)
        with mp.workdps(90):
            r90, c90 = R.b(x, s), R.b_complement(x, s)
        # the two precisions must agree far below the tolerance, or the reference is unreliable
        assert abs(r60 - r90) <= mp.mpf("1e-40") * abs(r90) + mp.mpf("1e-400")
        assert abs(c60 - c90) <= mp.mpf("1e-40") * abs(c90) + mp.mpf("1e-400")
        tol = 8 * EPS * (1 + A)
        if r90 > 1e-300:
            err = float(abs(orc.normalised_black(x, s) - r90) / r90)
            worst = max(worst, err / tol)
        if c90 > 1e-300:
            err = float(abs(orc.normalised_black_complement(x, s) - c90) / c90)
            worst = max(worst, err / tol)
        if r90 > 0:
            lb = orc.log_normalised_black(x, s)
            err = float(abs(lb - mp.log(r90)))
            worst = max(worst, err / (8 * EPS * (1 + A)))
    return worst


def test_normalised_black_matches_definition():
    assert check_b(oracle.default()) <= 1.0


def test_normalised_black_atm_is_erf():
    """b(0, s) = 2 Phi(s/2) - 1 = erf(s / (2 sqrt 2)) (Eq. app_normalized_black at k = 0)."""
    for s in [1e-6, 1e-3, 0.05, 0.3, 1.0, 2.5, 7.0]:
        ref = sps.erf(s / (2 * math.sqrt(2)))
        assert abs(oracle.normalised_black(0.0, s) - ref) <= 4 * EPS * ref
        refc = sps.erfc(s / (2 * math.sqrt(2)))
        assert abs(oracle.normalised_black_complement(0.0, s) - refc) <= 8 * EPS * refc


def test_normalised_black_limits():
    """b -> b_max = e^{x/2} as s -> inf and b -> 0 as s -> 0 (Eq. app_b_bounds).

    b(x,s) + (b_max - b)(x,s) = e^{x/2} exercises the identity
    int_0^inf exp(-a^2/u^2 - c^2 u^2) du = sqrt(pi)/(2c) e^{-2ac} behind both
    integrals; at small s the complement alone is e^{x/2}, at large s b alone is.
    """
    for x in [-1e-4, -0.3, -1.0, -4.0]:
        bm = math.exp(0.5 * x)
        s_small = abs(x) / 15.0  # b ~ exp(-112): negligible
        # the scaled integrals carry the conditioning factor 1 + A + B of the exponent
        cond = 1 + 112.5 + s_small ** 2 / 8
        assert abs(oracle.normalised_black_complement(x, s_small) - bm) <= 8 * EPS * cond * bm
        assert oracle.normalised_black(x, s_small) < 1e-40
        s_big = 55.0  # b_max - b ~ exp(-378)
        cond = 1 + 0.5 * (x / s_big) ** 2 + s_big ** 2 / 8
        assert abs(oracle.normalised_black(x, s_big) - bm) <= 8 * EPS * cond * bm
        for s in [0.2, 1.0, 3.0]:
            tot = oracle.normalised_black(x, s) + oracle.normalised_black_complement(x, s)
            cond = 1 + 0.5 * (x / s) ** 2 + s * s / 8
            assert abs(tot - bm) <= 8 * EPS * cond * bm


def test_mills_ratio():
    for z in [-300.0, -40.0, -8.0, -1.5, -0.2, 0.0, 0.4, 3.0, 9.0]:
        with mp.workdps(50):
            ref = mp.ncdf(z) / mp.npdf(z)
        assert abs(oracle.mills(z) - float(ref)) <= 8 * EPS * float(ref)


def test_black_price_and_vega_against_definition():
    b = workloads.body_batch(60, seed=11)
    P, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    for i in range(b.n):
        with mp.workdps(50):
            ref = R.price(b.F[i], b.K[i], b.T[i], b.sigma_star[i], int(b.flag[i]))
            vref = R.vega(b.F[i], b.K[i], b.T[i], b.sigma_star[i])
        sT = b.sigma_star[i] * math.sqrt(b.T[i])
        cond = 1 + 0.5 * (math.log(b.F[i] / b.K[i]) / sT) ** 2 + sT * sT / 8
        assert abs(P[i] - float(ref)) <= 8 * EPS * cond * float(ref) + 1e-300
        assert abs(V[i] - float(vref)) <= 8 * EPS * cond * float(vref) + 1e-300


def test_iv_atm_closed_form():
    """At the money b(0,s) = 2 Phi(s/2) - 1, so sigma = 2 Phi^{-1}((beta + 1)/2)/sqrt(T)."""
    rng = np.random.default_rng(5)
    n = 40
    F = np.full(n, 100.0)
    T = rng.uniform(0.01, 3.0, n)
    P = np.concatenate([10.0 ** rng.uniform(-8, -1, n // 2), rng.uniform(1, 99.999, n - n // 2)])
    flag = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    sig, st = oracle.implied_vol(F, F, T, P, flag)
    assert np.all(st == 0)
    for i in range(n):
        with mp.workdps(40):
            beta = mp.mpf(P[i]) / 100
            ref = 2 * mp.sqrt(2) * mp.erfinv(beta) / mp.sqrt(T[i])
        assert abs(sig[i] - float(ref)) <= 8 * EPS * float(ref), (i, P[i], sig[i], float(ref))


def _kappa_beta(F, K, P, flag, sig, T, V):
    """conditioning of sigma w.r.t. the time value: tv / (sigma V)"""
    itm = np.where(flag > 0, np.maximum(F - K, 0), np.maximum(K - F, 0))
    return (P - itm) / (sig * V)


def test_iv_against_high_precision_bisection():
    """Brute force on tiny inputs: bisection of the definition in 60-digit arithmetic."""
    b = workloads.body_batch(24, seed=21)
    st_b = workloads.stress_batch(24, seed=22, boundary_frac=0.0)
    F = np.concatenate([b.F, st_b.F])
    K = np.concatenate([b.K, st_b.K])
    T = np.concatenate([b.T, st_b.T])
    s0 = np.concatenate([b.sigma_star, st_b.sigma_star])
    flag = np.concatenate([b.flag, st_b.flag])
    P, V = oracle.black_price(F, K, T, s0, flag)
    sig, st = oracle.implied_vol(F, K, T, P, flag)
    checked = 0
    for i in range(len(F)):
        with mp.workdps(60):
            ref = R.implied_vol(F[i], K[i], T[i], P[i], int(flag[i]), iters=120)
        if ref is None:
            # outside the open interval (intrinsic, upper): the exact comparison fixes the status
            with mp.workdps(60):
                itm = max(mp.mpf(F[i]) - mp.mpf(K[i]), 0) if flag[i] > 0 else max(mp.mpf(K[i]) - mp.mpf(F[i]), 0)
                up = mp.mpf(F[i]) if flag[i] > 0 else mp.mpf(K[i])
                Pm = mp.mpf(P[i])
                want = 1 if Pm < itm else 4 if Pm == itm else 5 if Pm == up else 2
            assert st[i] == want
            continue
        assert st[i] == 0
        _, Vi = oracle.black_price(F[i:i + 1], K[i:i + 1], T[i:i + 1], sig[i:i + 1], flag[i:i + 1])
        kap = _kappa_beta(F[i], K[i], P[i], flag[i], sig[i], T[i], Vi[0])
        # a rounding of beta moves sigma by kappa times itself
        tol = 16 * EPS * (1 + kap)
        assert abs(sig[i] - float(ref)) <= tol * float(ref), (i, sig[i], float(ref), kap)
        checked += 1
    assert checked >= 30


def test_put_call_parity_gives_same_sigma():
    """A call and a put at parity-consistent prices share sigma (Appendix, IV as working coordinate)."""
    b = workloads.body_batch(200, seed=31)
    call = np.ones(b.n, np.int8)
    Pc, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, call)
    Pp = Pc - (b.F - b.K)  # parity with r = 0
    ok = Pp > 0
    sc, stc = oracle.implied_vol(b.F, b.K, b.T, Pc, call)
    sp, stp = oracle.implied_vol(b.F, b.K, b.T, Pp, -call)
    good = ok & (stc == 0) & (stp == 0) & (sc > 0)
    assert good.sum() > 150
    # a price error dP moves sigma by dP / (sigma V); Pp carries one rounding of the parity shift
    with np.errstate(divide="ignore", invalid="ignore"):
        tol = 32 * EPS * (1 + (Pc + np.abs(b.F - b.K)) / (sc * V))
        rel = np.abs(sc - sp) / sc
    assert np.all(rel[good] <= tol[good])


def test_round_trip_price():
    """price(sigma(P)) = P to a few ulp of P wherever sigma is finite (Section 4.1, round trip)."""
    for batch in (workloads.body_batch(400, seed=41), workloads.stress_batch(400, seed=42)):
        P, _ = oracle.black_price(batch.F, batch.K, batch.T, batch.sigma_star, batch.flag)
        P = workloads.merge_prices(batch, P)
        sig, st = oracle.implied_vol(batch.F, batch.K, batch.T, P, batch.flag)
        ok = st == 0
        P2, V2 = oracle.black_price(batch.F, batch.K, batch.T, sig, batch.flag)
        # |P2 - P| <~ V * dsigma + rounding: a relative solver error eps in sigma costs eps sigma V
        tol = 32 * EPS * (P + sig * V2)
        assert np.all(np.abs(P2[ok] - P[ok]) <= tol[ok])


def test_status_codes():
    """Invalid rows are NaN (Section 3.1: below intrinsic, super-arbitrage, tau <= 0)."""
    F = np.array([100, 100, 100, 100, 100, 100, 100, -1, 100, 100, 100, 100, np.nan, 100.0])
    K = np.array([90, 110, 90, 110, 90, 110, 100, 100, 100, 100, 100, 100, 100, 100.0])
    T = np.array([1, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, 1, 1, -1.0])
    P = np.array([9.0, 5, 100, 110, 10, 110.5, 5, 5, np.nan, 5, -1e-300, 0.0, 5, 5])
    flag = np.array([1, -1, 1, -1, 1, -1, 1, 1, 1, 0, 1, 1, 1, 1], np.int8)
    sig, st = oracle.implied_vol(F, K, T, P, flag)
    expected = [1, 1, 5, 5, 4, 2, 3, 3, 3, 3, 1, 4, 3, 3]
    assert list(st) == expected
    assert np.all(np.isnan(sig[np.isin(st, [1, 2, 3])]))
    assert np.all(sig[st == 4] == 0) and np.all(np.isinf(sig[st == 5]))


def test_adjoint_against_high_precision_finite_differences():
    """Eq. implicit_iv: gradients of the exact root by central differences in 80 digits."""
    b = workloads.body_batch(10, seed=51)
    P, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    dP, dF, dK, dT = oracle.iv_grad(b.F, b.K, b.T, b.flag, sig)
    for i in range(b.n):
        if st[i] != 0 or P[i] / (sig[i] * V[i]) > 100:
            continue
        with mp.workdps(80):
            ref = R.iv_gradient_fd(b.F[i], b.K[i], b.T[i], P[i], int(b.flag[i]), rel_h=mp.mpf("1e-20"))
        # the oracle evaluates the closed forms at its own sigma: kappa * eps of slack
        kap = P[i] / (sig[i] * V[i])
        for got, want in zip((dP[i], dF[i], dK[i], dT[i]), ref):
            want = float(want)
            assert abs(got - want) <= 1e-12 * (1 + kap) * abs(want) + 1e-300, (i, got, want)


def test_adjoint_invariants():
    """sigma is homogeneous of degree 0 in (F, K, P): F dF + K dK + P dP = 0; dT = -sigma/(2T)."""
    b = workloads.body_batch(300, seed=61)
    P, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    dP, dF, dK, dT = oracle.iv_grad(b.F, b.K, b.T, b.flag, sig)
    ok = (st == 0) & (P < 100 * sig * V)
    terms = np.abs(b.F * dF) + np.abs(b.K * dK) + np.abs(P * dP)
    assert np.all(np.abs(b.F * dF + b.K * dK + P * dP)[ok] <= 64 * EPS * terms[ok])
    assert np.allclose(dT[ok], -sig[ok] / (2 * b.T[ok]), rtol=4 * EPS, atol=0)
    _, Vs = oracle.black_price(b.F, b.K, b.T, sig, b.flag)  # vega at the recovered sigma
    assert np.allclose(dP[ok], 1.0 / Vs[ok], rtol=4 * EPS, atol=0)


def test_gate_modes():
    """Section 3.3: G_tau = {|V| > tau}; NaN / zero / hard-mask / smooth-gate semantics."""
    b = workloads.body_batch(400, seed=71)
    P, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    ok = st == 0
    g = np.random.default_rng(0).normal(size=b.n)
    g[::7] = 0.0
    _, Vs = oracle.black_price(b.F, b.K, b.T, sig, b.flag)
    tau = float(np.median(Vs[ok]))
    exact = np.array(oracle.iv_grad(b.F, b.K, b.T, b.flag, sig, g, tau, 0))
    m1 = np.array(oracle.iv_grad(b.F, b.K, b.T, b.flag, sig, g, tau, 1))
    m2 = np.array(oracle.iv_grad(b.F, b.K, b.T, b.flag, sig, g, tau, 2))
    m3 = np.array(oracle.iv_grad(b.F, b.K, b.T, b.flag, sig, g, tau, 3))
    inG = ok & (np.abs(Vs) > tau)
    off = ok & ~inG
    for m in (m1, m2):
        assert np.array_equal(m[:, inG], exact[:, inG])
    assert np.all(np.isnan(m1[:, off & (g != 0)])) and np.all(m1[:, off & (g == 0)] == 0)
    assert np.all(m2[:, off] == 0)
    w = Vs ** 2 / (Vs ** 2 + tau ** 2)
    assert np.allclose(m3[:, ok], exact[:, ok] * w[ok], rtol=1e-14, atol=0)
    # invalid rows stay NaN under every gate; rows at a bound are outside every G_tau
    for m in (exact, m1, m2, m3):
        assert np.all(np.isnan(m[:, np.isin(st, [1, 2, 3])]))


MUTATIONS = [
    ("s^2/8 sign in the normalised vega", "return -0.5 * h * h - 0.125 * s * s - LN_SQRT_2PI;",
     "return -0.5 * h * h + 0.125 * s * s - LN_SQRT_2PI;"),
    ("d2 = d1 + s", "d2 = d1 - s;", "d2 = d1 + s;"),
    ("call delta sign", "jF = -oracle_mills(d1) / (F * sqT);", "jF = oracle_mills(d1) / (F * sqT);"),
    ("put/call swap in the time value", "two_sum(s1, K, &s2, &e2); }", "two_sum(s1, F, &s2, &e2); }"),
    ("gamma integrand transposed A and B", "double e = (1.0 - v) * (1.0 + v) * (A - B / (v * v));",
     "double e = (1.0 - v) * (1.0 + v) * (B - A / (v * v));"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_are_caught(tmp_path, name, old, new):
    src = oracle.source_text()
    assert old in src, name
    bad = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libbad.so"))
    caught = []
    try:
        caught.append(check_b(bad, n=60, seed=4) > 1.0)
    except AssertionError:
        caught.append(True)
    b = workloads.body_batch(12, seed=81)
    P, V = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    sig_bad, st_bad = bad.implied_vol(b.F, b.K, b.T, P, b.flag)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    caught.append(not np.allclose(sig_bad, b.sigma_star, rtol=1e-10))
    g_bad = np.array(bad.iv_grad(b.F, b.K, b.T, b.flag, sig))
    g_ok = np.array(oracle.iv_grad(b.F, b.K, b.T, b.flag, sig))
    # invariants of the adjoint (homogeneity) catch wrong signs / wrong d2
    hom = np.abs(b.F * g_bad[1] + b.K * g_bad[2] + P * g_bad[0])
    caught.append(bool(np.any(hom > 1e-10 * (np.abs(b.F * g_ok[1]) + np.abs(P * g_ok[0])))))
    assert any(caught), name


def test_black_price_gradient_against_finite_differences():
    """dP/d(sigma, F, K, T) of Eq. app_black76 against 50-digit central differences."""
    b = workloads.body_batch(24, seed=91)
    got = oracle.black_price_grad(b.F, b.K, b.T, b.sigma_star, b.flag)
    for i in range(b.n):
        args = [b.F[i], b.K[i], b.T[i], b.sigma_star[i]]
        with mp.workdps(50):
            base = [mp.mpf(a) for a in args]
            ref = []
            for j in (3, 0, 1, 2):  # sigma, F, K, T
                h = base[j] * mp.mpf("1e-18")
                up, dn = list(base), list(base)
                up[j] += h
                dn[j] -= h
                ref.append((R.price(*up, int(b.flag[i])) - R.price(*dn, int(b.flag[i]))) / (2 * h))
        for g, r in zip((got[0][i], got[1][i], got[2][i], got[3][i]), ref):
            assert abs(g - float(r)) <= 1e-13 * abs(float(r)) + 1e-300, (i, g, float(r))
