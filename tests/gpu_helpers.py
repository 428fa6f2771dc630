"""Shared helpers for the GPU parity tests (inputs from workloads, truth from the oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2606_17065_gb300 import workloads

EPS = float(np.finfo(np.float64).eps)
DEV = torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def to_np(t):
    return t.detach().cpu().numpy()


def oracle_inputs(batch, nthreads=0):
    """Prices of a batch from the oracle's Black price (plus the workload's fixed boundary quotes)."""
    P, _ = oracle.black_price(batch.F, batch.K, batch.T, batch.sigma_star, batch.flag, nthreads=nthreads)
    return workloads.merge_prices(batch, P)


def conditioning(F, K, T, P, flag, sig):
    """kappa_P = P/(sigma V) and kappa_beta = tv/(sigma V), V the vega at sigma (oracle)."""
    _, V = oracle.black_price(F, K, T, np.where(np.isfinite(sig), sig, 1.0), flag, nthreads=0)
    itm = np.where(flag > 0, np.maximum(F - K, 0.0), np.maximum(K - F, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        kp = P / (sig * V)
        kb = (P - itm) / (sig * V)
    return kp, kb


def exponent(F, K, T, sig):
    """A + B = x^2/(2 s^2) + s^2/8: the conditioning of b_s in its arguments."""
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        s = sig * np.sqrt(T)
        x = np.log(F / K)
        return 0.5 * (x / s) ** 2 + 0.125 * s * s


def assert_sigma_parity(F, K, T, P, flag, sig, st, ref, st_ref, tol=1e-13, where=""):
    """Status identical on every row; sigma within `tol` relative on the parity domain
    (status 0, kappa_P <= 100); elsewhere within a conditioning-scaled bound."""
    assert np.array_equal(st, st_ref), f"{where}: status mismatch on {np.sum(st != st_ref)} rows"
    ok = st_ref == 0
    assert np.array_equal(np.isnan(sig), np.isnan(ref)), f"{where}: NaN pattern differs"
    assert np.all(sig[st_ref == 4] == 0) and np.all(np.isinf(sig[st_ref == 5]))
    kp, kb = conditioning(F, K, T, P, flag, ref)
    rel = np.abs(sig - ref) / ref
    dom = ok & (kp <= 100)
    if dom.any():
        worst = rel[dom].max()
        assert worst <= tol, f"{where}: max rel sigma error {worst:.3e} on the parity domain"
    off = ok & ~dom
    if off.any():
        bound = 256 * EPS * (1 + kb[off])
        bad = rel[off] > bound
        assert not bad.any(), f"{where}: {bad.sum()} off-domain rows beyond the conditioning bound"
    return dom


def assert_grad_parity(got, want, rows, tol=1e-10, where="", vega=None, gbar=None):
    """Identical non-finite pattern and finite values within `tol` relative on `rows`.

    Where the vega itself is subnormal or zero (|V| < 1e-280) two independent
    evaluations legitimately differ in how the underflow lands (0/0 = NaN
    against 0/1e-315 = 0, subnormal rounding); there only what is unique is
    compared: both sides non-finite or huge, or both zero to 1e-280, or NaN
    against 0 when the upstream cotangent is 0.
    """
    n = rows.shape[0]
    tiny = np.zeros(n, bool) if vega is None else ~(np.abs(vega) >= 1e-280)
    g_up = np.ones(n) if gbar is None else gbar
    strict, loose = rows & ~tiny, rows & tiny
    for name, g, w in zip(("dP", "dF", "dK", "dT"), got, want):
        gs, ws = g[strict], w[strict]
        assert np.array_equal(np.isnan(gs), np.isnan(ws)), f"{where} {name}: NaN pattern differs"
        assert np.array_equal(np.isinf(gs), np.isinf(ws)), f"{where} {name}: inf pattern differs"
        fin = np.isfinite(ws)
        denom = np.maximum(np.abs(ws[fin]), 1e-300)
        rel = np.abs(gs[fin] - ws[fin]) / denom
        if rel.size:
            assert rel.max() <= tol, f"{where} {name}: max rel error {rel.max():.3e}"
        gl, wl, ul = g[loose], w[loose], g_up[loose]
        if gl.size:
            with np.errstate(invalid="ignore", over="ignore"):
                big = lambda a: ~np.isfinite(a) | (np.abs(a) > 1e250)  # noqa: E731
                same = (big(gl) & big(wl)) | (np.abs(gl - wl) <= 1e-280) | (np.isnan(gl) & np.isnan(wl))
                same |= (ul == 0) & ((np.isnan(gl) | (gl == 0)) & (np.isnan(wl) | (wl == 0)))
                same |= np.abs(gl - wl) <= tol * np.abs(wl)
            assert same.all(), f"{where} {name}: {np.sum(~same)} subnormal-vega rows disagree"


def assert_grad_offdomain(F, K, T, P, flag, sig, st, ref, grads_nan, grads_exact, tau=1e-6, tol=1e-10, where=""):
    """The fused path's gradients on solved rows OFF the parity domain (kappa_P > 100), where sigma
    itself is only fixed to the conditioning bound of ``assert_sigma_parity``.

    (a) Against the oracle's adjoint evaluated at the GPU's own sigma (gate mode 1, tau): the
        closed forms of Eq. implicit_iv at one sigma, so `tol` relative as on the domain.
    (b) Against the oracle's adjoint at the oracle's sigma (exact gate): within
        tol + 256 eps (1 + kappa_beta) (2 + 6 (A + B)), the sigma bound times the conditioning of
        the gradient in sigma (|d ln g / d ln s| <= 1 + h^2 + t^2 + (|h| + t)^2 <= 2 + 6 (A + B),
        A + B = h^2/2 + t^2/2 the exponent of b_s), wherever both are finite and the vega is
        normal.
    Returns the number of rows checked."""
    kp, kb = conditioning(F, K, T, P, flag, ref)
    ok = (st == 0) & np.isfinite(sig) & (sig > 0)
    off = ok & ~(kp <= 100)
    if not off.any():
        return 0
    want_at_gpu = oracle.iv_grad(F, K, T, flag, np.where(ok, sig, ref), None, tau, 1, nthreads=0)
    _, Vg = oracle.black_price(F, K, T, np.where(ok, sig, 1.0), flag, nthreads=0)
    assert_grad_parity(grads_nan, want_at_gpu, off, tol=tol, where=f"{where} off-domain at GPU sigma", vega=Vg)
    want_ref = oracle.iv_grad(F, K, T, flag, ref, None, 0.0, 0, nthreads=0)
    _, Vr = oracle.black_price(F, K, T, np.where(np.isfinite(ref), ref, 1.0), flag, nthreads=0)
    AB = exponent(F, K, T, ref)
    with np.errstate(invalid="ignore", over="ignore"):
        bound = tol + 256 * EPS * (1 + kb) * (2 + 6 * AB)
    rows = off & (np.abs(Vr) >= 1e-280) & (np.abs(Vg) >= 1e-280)
    for name, g, w in zip(("dP", "dF", "dK", "dT"), grads_exact, want_ref):
        fin = rows & np.isfinite(g) & np.isfinite(w) & (w != 0)
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            rel = np.abs(g[fin] - w[fin]) / np.abs(w[fin])
        bad = rel > bound[fin]
        assert not bad.any(), (f"{where} {name}: {bad.sum()} off-domain rows beyond the conditioning bound, "
                               f"worst ratio {np.max(rel / bound[fin]):.3e}")
    return int(off.sum())
