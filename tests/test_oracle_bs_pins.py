"""Pins for the oracle's Black-Scholes interface on xi = (S, K, tau, r, q) (Section 2,
Eq. app_forward_price / app_black_scholes; Algorithm 1).

Each test ties the oracle to something other than itself: the spot-coordinate formula in
arbitrary precision, its root by bisection, finite differences of that root, exact
invariances of the problem (scaling of (S, K, V); a common shift of r and q; a rescaling
of time), the reduction to Black-76 at r = q = 0, and planted mistakes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_17065_gb300 import workloads

mp = pytest.importorskip("mpmath")
import mp_reference as R  # noqa: E402

EPS = np.finfo(np.float64).eps


def _cond(S, K, T, r, q, sig):
    """Conditioning of the price in its inputs: 1 + A + B + |d1|/s (A, B the exponents of b_s)."""
    s = sig * math.sqrt(T)
    x = math.log(S / K) + (r - q) * T
    return 1 + 0.5 * (x / s) ** 2 + s * s / 8 + abs(x / s + s / 2) / s


def check_bs_price(orc, b):
    V, vega = orc.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag)
    for i in range(b.n):
        with mp.workdps(50):
            ref = R.bs_price(b.S[i], b.K[i], b.T[i], b.r[i], b.q[i], b.sigma_star[i], int(b.flag[i]))
            s = mp.mpf(b.sigma_star[i]) * mp.sqrt(b.T[i])
            d1 = (mp.log(mp.mpf(b.S[i]) / b.K[i]) + (mp.mpf(b.r[i]) - b.q[i]) * b.T[i] + s * s / 2) / s
            vref = b.S[i] * mp.e ** (-mp.mpf(b.q[i]) * b.T[i]) * mp.npdf(d1) * mp.sqrt(b.T[i])
        c = _cond(b.S[i], b.K[i], b.T[i], b.r[i], b.q[i], b.sigma_star[i])
        # F = S e^{(r-q) tau} and e^{r tau} are rounded once each: a few ulp of S e^{-q tau} in V
        tol = 16 * EPS * (c * float(ref) + b.S[i] * math.exp(-b.q[i] * b.T[i]))
        assert abs(V[i] - float(ref)) <= tol, (i, V[i], float(ref))
        assert abs(vega[i] - float(vref)) <= 16 * EPS * c * float(vref), (i, vega[i], float(vref))


def test_bs_price_and_vega_against_definition():
    check_bs_price(oracle, workloads.bs_batch(48, seed=101))


def test_bs_iv_against_high_precision_bisection():
    b = workloads.bs_batch(20, seed=102)
    V, _ = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag)
    sig, st = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag)
    dV, dS, dK, dT, dr, dq = oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig)
    checked = 0
    for i in range(b.n):
        with mp.workdps(60):
            ref = R.bs_implied_vol(b.S[i], b.K[i], b.T[i], b.r[i], b.q[i], V[i], int(b.flag[i]), iters=120)
        if ref is None:
            continue
        assert st[i] == 0
        # roundings of V, of F = S e^{(r-q)tau} and of B = e^{r tau} V move sigma by their conditioning
        kap = (abs(V[i] * dV[i]) + abs(b.S[i] * dS[i])) / sig[i]
        assert abs(sig[i] - float(ref)) <= 16 * EPS * (1 + kap) * float(ref), (i, sig[i], float(ref), kap)
        checked += 1
    assert checked >= 16


def test_bs_adjoint_against_high_precision_finite_differences():
    """Algorithm 1 backward: d sigma / d(V, S, K, tau, r, q) of the exact root, 80 digits."""
    b = workloads.bs_batch(6, seed=103)
    V, vega = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag)
    sig, st = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag)
    got = oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig)
    done = 0
    for i in range(b.n):
        kap = V[i] / (sig[i] * vega[i])
        if st[i] != 0 or kap > 100:
            continue
        with mp.workdps(80):
            ref = R.bs_iv_gradient_fd(b.S[i], b.K[i], b.T[i], b.r[i], b.q[i], V[i], int(b.flag[i]))
        for j, want in enumerate(ref):
            want = float(want)
            assert abs(got[j][i] - want) <= 1e-12 * (1 + kap) * abs(want) + 1e-300, (i, j, got[j][i], want)
        done += 1
    assert done >= 4


def _bs_rows(n, seed):
    b = workloads.bs_batch(n, seed=seed)
    V, vega = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag)
    sig, st = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag)
    return b, V, vega, sig, st


def invariant_residuals(orc, b, V, sig):
    """Three exact invariances of sigma(V, S, K, tau, r, q), differentiated at the identity:
    (S, K, V) -> lambda (S, K, V):                      S dS + K dK + V dV = 0
    (r, q, V) -> (r + c, q + c, V e^{-c tau}):          dr + dq - tau V dV = 0
    (tau, r, q) -> (lambda tau, r/lambda, q/lambda):    tau dtau - r dr - q dq + sigma/2 = 0
    Returns each residual over the sum of the magnitudes of its terms."""
    dV, dS, dK, dT, dr, dq = orc.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig)
    out = []
    for terms in ((b.S * dS, b.K * dK, V * dV), (dr, dq, -b.T * V * dV),
                  (b.T * dT, -b.r * dr, -b.q * dq, 0.5 * sig)):
        tot = sum(terms)
        mag = sum(np.abs(t) for t in terms)
        out.append(np.abs(tot) / mag)
    return out


def test_bs_adjoint_invariances():
    b, V, vega, sig, st = _bs_rows(400, 104)
    ok = (st == 0) & (V < 100 * sig * vega)
    assert ok.sum() > 300
    for res in invariant_residuals(oracle, b, V, sig):
        assert np.all(res[ok] <= 64 * EPS), res[ok].max()


def test_bs_reduces_to_black_at_zero_rates():
    """r = q = 0: F = S, B = V, and every output is the Black-76 one (Eq. app_black76)."""
    b = workloads.bs_batch(300, seed=105)
    z = np.zeros(b.n)
    V, vega = oracle.bs_price(b.S, b.K, b.T, z, z, b.sigma_star, b.flag)
    P, Vb = oracle.black_price(b.S, b.K, b.T, b.sigma_star, b.flag)
    assert np.array_equal(V, P) and np.array_equal(vega, Vb)
    sig, st = oracle.bs_implied_vol(b.S, b.K, b.T, z, z, V, b.flag)
    sb, stb = oracle.implied_vol(b.S, b.K, b.T, P, b.flag)
    assert np.array_equal(st, stb) and np.array_equal(sig[st == 0], sb[stb == 0])
    ok = (st == 0) & (V < 100 * sig * vega)
    g = oracle.bs_iv_grad(b.S, b.K, b.T, z, z, b.flag, sig)
    gb = oracle.iv_grad(b.S, b.K, b.T, b.flag, sb)
    for got, want in zip(g[:4], gb):
        assert np.allclose(got[ok], want[ok], rtol=1e-13, atol=0)


def test_bs_status_codes_and_gate():
    b, V, vega, sig, st = _bs_rows(400, 106)
    ok = st == 0
    # invalid rates and expiries
    r = b.r.copy()
    q = b.q.copy()
    T = b.T.copy()
    r[:5] = np.nan
    q[5:10] = np.inf
    T[10:15] = 0.0
    s2, st2 = oracle.bs_implied_vol(b.S, b.K, T, r, q, V, b.flag)
    assert np.all(st2[:15] == 3) and np.all(np.isnan(s2[:15]))
    # below the discounted intrinsic value / at it
    disc_itm = np.where(b.flag > 0, np.maximum(b.S * np.exp(-b.q * b.T) - b.K * np.exp(-b.r * b.T), 0),
                        np.maximum(b.K * np.exp(-b.r * b.T) - b.S * np.exp(-b.q * b.T), 0))
    below = disc_itm > 1.0
    s3, st3 = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, 0.5 * disc_itm, b.flag)
    assert np.all(st3[below] == 1)
    # gate on the cash vega V_bs = dV/dsigma at the recovered sigma
    _, vs = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, sig, b.flag)
    tau = float(np.median(vs[ok]))
    g = np.random.default_rng(1).normal(size=b.n)
    g[::5] = 0.0
    ex = np.array(oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig, g, tau, 0))
    m1 = np.array(oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig, g, tau, 1))
    m2 = np.array(oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig, g, tau, 2))
    m3 = np.array(oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, sig, g, tau, 3))
    # the adjoint evaluates V_bs in its own rounding: leave out rows within 1e-12 of tau
    clear = ok & (np.abs(vs / tau - 1) > 1e-12)
    inG = clear & (vs > tau)
    off = clear & ~inG
    assert inG.sum() > 100 and off.sum() > 100
    assert np.array_equal(m1[:, inG], ex[:, inG]) and np.array_equal(m2[:, inG], ex[:, inG])
    assert np.all(np.isnan(m1[:, off & (g != 0)])) and np.all(m1[:, off & (g == 0)] == 0)
    assert np.all(m2[:, off] == 0)
    # w = V^2/(V^2 + tau^2) and w/V in the scaled form that does not underflow
    u = vs / tau
    w = u * u / (1 + u * u)
    wv = (u / tau) / (1 + u * u)
    # V_bs = exp(-d1^2/2 + ...) carries ~d1^2 eps of rounding in either evaluation, w twice that
    d1 = (np.log(b.S / b.K) + (b.r - b.q) * b.T) / (sig * np.sqrt(b.T)) + 0.5 * sig * np.sqrt(b.T)
    rt = 32 * EPS * (8 + d1 * d1)
    want3 = np.concatenate([(g * wv)[None], ex[1:] * w])
    for m, want in ((m3, want3), (ex[:1], (g / vs)[None])):
        assert np.all(np.abs(m[:, ok] - want[:, ok]) <= rt[ok] * np.abs(want[:, ok]))


BS_MUTATIONS = [
    ("carry sign in the forward", "*F = S * exp((r - q) * T);", "*F = S * exp((q - r) * T);"),
    ("discounting by q", "*B = Vm * exp(r * T);", "*B = Vm * exp(q * T);"),
    ("rate sensitivity sign", "j[4] = -theta * sqT * M2;", "j[4] = theta * sqT * M2;"),
    ("r and q swapped in dsigma/dtau", "theta * (q * M1 - r * M2) / sqT;", "theta * (r * M1 - q * M2) / sqT;"),
    ("d1 of the adjoint without carry", "double x = log(S / K) + (r - q) * T;", "double x = log(S / K);"),
]


@pytest.mark.parametrize("name,old,new", BS_MUTATIONS, ids=[m[0] for m in BS_MUTATIONS])
def test_bs_planted_mistakes_are_caught(tmp_path, name, old, new):
    src = oracle.source_text()
    assert old in src, name
    bad = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libbad.so"))
    caught = []
    b = workloads.bs_batch(12, seed=107)
    try:
        check_bs_price(bad, b)
        caught.append(False)
    except AssertionError:
        caught.append(True)
    V, _ = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag)
    sig_bad, _ = bad.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag)
    caught.append(not np.allclose(sig_bad, b.sigma_star, rtol=1e-10))
    sig, _ = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag)
    caught.append(any(bool(np.nanmax(res) > 1e-10) for res in invariant_residuals(bad, b, V, sig)))
    assert any(caught), name
