"""GPU parity of the Black-Scholes interface on xi = (S, K, tau, r, q) (Algorithm 1) against the
oracle, through the C ABI.

Bar: status codes identical on every row whose status is fixed within the rounding of the
input map (rows whose price lies within a few ulp of a bound of the interval -- deep in the
money, the time value below one ulp of the price -- may take any status the oracle gives
within that rounding, with a sigma valid for it); sigma within
1e-13 relative and the six gradients
within 1e-10 relative on the parity domain {status 0, kappa_V <= 100, kappa_S <= 100}, where
kappa_V = V/(sigma V_bs) and kappa_S = |S dsigma/dS|/sigma.  kappa_S joins the domain because
both sides round F = S e^{(r-q) tau} and B = e^{r tau} V once, each with its own exp: one ulp of
F moves sigma by kappa_S ulp.  Off the domain sigma is held to a conditioning-scaled bound.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import _native, workloads  # noqa: E402

from gpu_helpers import EPS, assert_grad_parity, to_dev, to_np  # noqa: E402

pytestmark = pytest.mark.gpu

NAMES = ("dV", "dS", "dK", "dT", "dr", "dq")


def edge_rows(b, V):
    """Rows on and outside the price interval, and bad inputs, planted into a copy of the batch."""
    b = b.subset(np.arange(b.n))
    V = V.copy()
    n = 40
    i = np.arange(n)
    V[i[0:4]] = 0.0                      # OTM at 0 -> at intrinsic (sigma = 0), ITM -> below intrinsic
    V[i[4:8]] = -1.0                     # below intrinsic
    b.r[i[8:10]] = np.nan                # bad rate
    b.q[i[10:12]] = -np.inf              # bad yield
    b.T[i[12:14]] = 0.0                  # expired
    b.S[i[14:16]] = -5.0                 # bad spot
    b.flag[i[16:18]] = 0                 # bad flag
    V[i[18:22]] = 1e6                    # above the upper bound
    b.r[i[22:26]] = 0.0
    b.q[i[22:26]] = 0.0                  # zero carry: F = S exactly
    b.T[i[26:30]] = 1e-8                 # very short expiry
    b.r[i[30:34]] = -0.2                 # strongly negative rate
    V[i[34:40]] = np.nan                 # missing quote
    return b, V


@pytest.fixture(scope="module")
def rows():
    body = workloads.bs_batch(30_000 + 77, seed=201)
    wide = workloads.bs_batch(30_000 + 33, seed=202, wide=True)
    out = []
    for b in (body, wide):
        V, _ = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag, nthreads=0)
        b, V = edge_rows(b, V)
        sig, st = oracle.bs_implied_vol(b.S, b.K, b.T, b.r, b.q, V, b.flag, nthreads=0)
        out.append((b, V, sig, st))
    return out


def domain(b, V, sig, st):
    ok = st == 0
    s1 = np.where(ok, sig, 1.0)
    _, vega = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, s1, b.flag, nthreads=0)
    _, dS, _, _, _, _ = oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, s1, nthreads=0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        kv = V / (s1 * vega)
        ks = np.abs(b.S * dS) / s1
    return ok & (kv <= 100) & (ks <= 100), kv, ks, vega


def gpu_args(b, V):
    return [to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q, V)] + [to_dev(b.flag)]


def status_sets(b, V, st_ref, ulps=4):
    """The statuses the oracle gives when V or S move by up to `ulps` ulp.

    Each side rounds B = e^{r tau} V and F = S e^{(r-q) tau} with its own exp, so a row whose
    price lies within a few ulp of a bound of the interval (deep in the money with a time value
    below one ulp of the price, or at the upper bound) has no unique status.  Returns a boolean
    mask of such rows and, per row, the set of statuses seen (as a bit mask)."""
    seen = (1 << st_ref.astype(np.int64))
    for dV, dS in ((ulps, 0), (-ulps, 0), (0, ulps), (0, -ulps), (ulps, ulps), (ulps, -ulps), (-ulps, ulps),
                   (-ulps, -ulps)):
        V2 = V * (1 + dV * EPS)
        S2 = b.S * (1 + dS * EPS)
        _, st2 = oracle.bs_implied_vol(S2, b.K, b.T, b.r, b.q, V2, b.flag, nthreads=0)
        seen |= (1 << st2.astype(np.int64))
    # between a price above and one below a bound lies the bound itself
    seen |= np.where((seen & 1) & ((seen >> 1) & 1), 1 << 4, 0)
    seen |= np.where((seen & 1) & ((seen >> 2) & 1), 1 << 5, 0)
    return seen != (1 << st_ref.astype(np.int64)), seen


def check_sigma(b, V, sig, st, ref, st_ref, where, tol=1e-13):
    amb, seen = status_sets(b, V, st_ref)
    clear = ~amb
    assert np.array_equal(st[clear], st_ref[clear]), f"{where}: status mismatch on {np.sum(st != st_ref)} rows"
    # ambiguous rows: a status the oracle also gives within the rounding, and a consistent sigma
    assert np.all(((1 << st[amb].astype(np.int64)) & seen[amb]) != 0), f"{where}: ambiguous row out of its set"
    assert np.all(sig[amb & (st == 4)] == 0) and np.all(np.isinf(sig[amb & (st == 5)]))
    assert np.all(np.isnan(sig[amb & np.isin(st, [1, 2, 3])]))
    assert np.all((sig[amb & (st == 0)] > 0) & np.isfinite(sig[amb & (st == 0)]))
    assert np.array_equal(np.isnan(sig[clear]), np.isnan(ref[clear])), f"{where}: NaN pattern differs"
    assert np.all(sig[clear & (st_ref == 4)] == 0) and np.all(np.isinf(sig[clear & (st_ref == 5)]))
    dom, kv, ks, _ = domain(b, V, ref, st_ref)
    dom &= clear
    rel = np.abs(sig - ref) / ref
    assert rel[dom].max() <= tol, f"{where}: max rel sigma error {rel[dom].max():.3e}"
    off = clear & (st_ref == 0) & ~dom
    if off.any():
        bound = 256 * EPS * (1 + kv[off] + ks[off])
        assert np.all(rel[off] <= bound), f"{where}: {np.sum(rel[off] > bound)} rows beyond the bound"
    return dom


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_bs_forward_parity(rows, mode):
    for k, (b, V, ref, st_ref) in enumerate(rows):
        sig, st = pv.bs_iv(*gpu_args(b, V), mode=mode)
        dom = check_sigma(b, V, to_np(sig), to_np(st), ref, st_ref, f"{mode} batch {k}")
        assert dom.sum() > (25_000 if k == 0 else 5_000)


@pytest.mark.parametrize("gate", [0, 1, 2, 3])
def test_bs_forward_backward_parity(rows, gate):
    for k, (b, V, ref, st_ref) in enumerate(rows):
        dom, _, _, vega = domain(b, V, ref, st_ref)
        g = np.random.default_rng(7 + gate).normal(size=b.n)
        g[::9] = 0.0
        tau = float(np.median(vega[dom]))
        out = pv.bs_iv_forward_backward(*gpu_args(b, V), to_dev(g), tau=tau, gate=gate)
        sig, st = to_np(out[0]), to_np(out[1])
        dom = check_sigma(b, V, sig, st, ref, st_ref, f"fwd+bwd gate {gate} batch {k}")
        want = oracle.bs_iv_grad(b.S, b.K, b.T, b.r, b.q, b.flag, ref, g, tau, gate, nthreads=0)
        got = [to_np(t) for t in out[2:]]
        # rows within 1e-12 of the gate threshold may fall either side of it
        clear = np.abs(vega / tau - 1) > 1e-12
        rows_cmp = dom & clear
        for j in range(0, 6, 3):
            assert_grad_parity(got[j:j + 3] + [got[j]], list(want[j:j + 3]) + [want[j]], rows_cmp,
                               where=f"gate {gate} batch {k} {NAMES[j:j + 3]}", vega=vega, gbar=g)
        # invalid rows: NaN in every output and gate
        bad = np.isin(st_ref, [1, 2, 3]) & (st == st_ref)
        for t in got:
            assert np.all(np.isnan(t[bad]))


def test_bs_backward_alone_matches_fused(rows):
    b, V, ref, st_ref = rows[1]
    fused = pv.bs_iv_forward_backward(*gpu_args(b, V), tau=1e-6, gate="nan")
    sig = fused[0]
    alone = pv.bs_iv_backward(*[to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q)], to_dev(b.flag), sig, tau=1e-6,
                              gate="nan")
    # the fused kernel differentiates at the solver's s, the backward alone at sigma sqrt(tau):
    # one rounding apart, which the adjoint's conditioning (kappa_V, kappa_S) amplifies
    dom, _, _, vega = domain(b, V, ref, st_ref)
    dom &= np.abs(vega) >= 1e-280
    for x, y in zip(fused[2:], alone):
        x, y = to_np(x), to_np(y)
        assert np.array_equal(np.isnan(x[dom]), np.isnan(y[dom]))
        m = dom & np.isfinite(y)
        assert np.all(np.abs(x[m] - y[m]) <= 1e-11 * np.abs(y[m]))


def test_bs_zero_carry_equals_black_path():
    """r = q = 0: F = S and B = V exactly, so sigma and the shared gradients are the Black-76 ones."""
    b = workloads.bs_batch(20_000, seed=203, wide=True)
    z = np.zeros(b.n)
    P, _ = oracle.black_price(b.S, b.K, b.T, b.sigma_star, b.flag, nthreads=0)
    bs = pv.bs_iv_forward_backward(*[to_dev(a) for a in (b.S, b.K, b.T, z, z, P)], to_dev(b.flag), tau=1e-6)
    bl = pv.iv_forward_backward(*[to_dev(a) for a in (b.S, b.K, b.T, P)], to_dev(b.flag), tau=1e-6)
    for x, y in zip((bs[0], bs[1], bs[2], bs[3], bs[4], bs[5]), bl):
        assert torch.equal(torch.nan_to_num(x.double(), nan=7.0), torch.nan_to_num(y.double(), nan=7.0))


def test_bs_price_parity():
    b = workloads.bs_batch(20_000, seed=204)
    V, vega = pv.bs_price(*[to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q, b.sigma_star)], to_dev(b.flag))
    Vr, vr = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag, nthreads=0)
    V, vega = to_np(V), to_np(vega)
    s = b.sigma_star * np.sqrt(b.T)
    x = np.log(b.S / b.K) + (b.r - b.q) * b.T
    cond = 1 + 0.5 * (x / s) ** 2 + s * s / 8 + np.abs(x / s + s / 2) / s
    # F and the discount factor are rounded with each side's own exp
    tol = 32 * EPS * (cond * Vr + b.S * np.exp(-b.q * b.T))
    assert np.all(np.abs(V - Vr) <= tol)
    assert np.all(np.abs(vega - vr) <= 32 * EPS * cond * vr)


def test_bs_autograd_matches_backward(rows):
    b, V, ref, st_ref = rows[0]
    dom, _, _, _ = domain(b, V, ref, st_ref)
    idx = np.where(dom)[0][:4096]
    sub = b.subset(idx)
    leaves = [to_dev(a).requires_grad_(True) for a in (V[idx], sub.S, sub.K, sub.T, sub.r, sub.q)]
    sig = pv.bs_implied_volatility_autograd(leaves[0], *leaves[1:], to_dev(sub.flag), 1e-6, "nan")
    w = torch.linspace(0.5, 1.5, sig.numel(), dtype=torch.float64, device=sig.device)
    (sig * w).sum().backward()
    want = oracle.bs_iv_grad(sub.S, sub.K, sub.T, sub.r, sub.q, sub.flag, ref[idx], to_np(w), 1e-6, 1, nthreads=0)
    for leaf, wv, name in zip(leaves, want, NAMES):
        got = to_np(leaf.grad)
        # rows with a cash vega at or below the gate threshold are NaN on both sides (gate "nan")
        assert np.array_equal(np.isnan(got), np.isnan(wv)), name
        assert np.isfinite(wv).mean() > 0.5
        m = np.isfinite(wv)
        rel = np.abs(got[m] - wv[m]) / np.abs(wv[m])
        assert rel.max() <= 1e-10, (name, rel.max())


def test_bs_invariances_at_full_size():
    """At 16M rows (the size of the fused benchmark), properties that hold at any size:
    S dS + K dK + V dV = 0, dr + dq - tau V dV = 0, tau dtau - r dr - q dq + sigma/2 = 0 on every
    well-conditioned row, and price(sigma(V)) = V on a sample."""
    n = workloads.STRESS_N
    b = workloads.bs_batch(n, seed=205)
    d = [to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q, b.sigma_star)]
    fl = to_dev(b.flag)
    V, vega = pv.bs_price(*d, fl)
    sig, st, dV, dS, dK, dT, dr, dq = pv.bs_iv_forward_backward(*d[:5], V, fl, tau=0.0, gate="exact")
    S, K, T, r, q = d[:5]
    # well-conditioned rows whose vega is a normal number (a subnormal vega makes 1/V overflow)
    ok = (st == 0) & (V < 100 * sig * vega) & (vega >= 1e-280)
    assert ok.double().mean().item() > 0.9
    for terms in ((S * dS, K * dK, V * dV), (dr, dq, -T * V * dV), (T * dT, -r * dr, -q * dq, 0.5 * sig)):
        tot = sum(terms)
        mag = sum(t.abs() for t in terms)
        res = (tot.abs() / mag)[ok]
        assert res.max().item() <= 1e-12, res.max().item()
    idx = workloads.sample_indices(n, 4096, seed=9)
    sub = b.subset(idx)
    ref, st_ref = oracle.bs_implied_vol(sub.S, sub.K, sub.T, sub.r, sub.q, to_np(V)[idx], sub.flag, nthreads=0)
    check_sigma(sub, to_np(V)[idx], to_np(sig)[idx], to_np(st)[idx], ref, st_ref, "16M sample")


def test_bs_rejects_learned_mode():
    b = workloads.bs_batch(64, seed=206)
    with pytest.raises(_native.PivotError):
        pv.bs_iv(*gpu_args(b, np.ones(b.n)), mode="learned")
