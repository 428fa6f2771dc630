"""The differentiable operator in torch (Section 3.2, SPX and NaN-poisoning appendices).

ImpliedVol and BlackPrice wrap the CUDA kernels as autograd nodes; their
gradients are checked against the oracle's analytic adjoint and against
central finite differences of the CUDA forward, the two-vega identity of the
composed loss is checked, and training through the operator is run on the
synthetic SVI surfaces and on the low-vega stress chain.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import training, workloads  # noqa: E402

from gpu_helpers import DEV, assert_grad_parity, conditioning, oracle_inputs, to_dev, to_np  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def body():
    b = workloads.body_batch(4096, seed=21)
    P = oracle_inputs(b)
    ref, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    return b, P, ref, st


def test_implied_vol_autograd_matches_oracle_adjoint(body):
    b, P, ref, st = body
    g = np.random.default_rng(1).normal(size=b.n)
    Pt = to_dev(P).requires_grad_(True)
    Ft, Kt, Tt = (to_dev(a).requires_grad_(True) for a in (b.F, b.K, b.T))
    sig = pv.implied_volatility_autograd(Pt, Ft, Kt, Tt, to_dev(b.flag), 1e-6, "exact")
    (sig * to_dev(g)).sum().backward()
    want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, g, 1e-6, 0, nthreads=0)
    kp, _ = conditioning(b.F, b.K, b.T, P, b.flag, ref)
    dom = (st == 0) & (kp <= 100)
    got = [to_np(t.grad) for t in (Pt, Ft, Kt, Tt)]
    assert_grad_parity(got, want, dom, where="autograd")


def test_implied_vol_autograd_against_finite_differences(body):
    """Central differences of the CUDA forward in P (the paper's FD check, Section 4 appendix)."""
    b, P, ref, st = body
    _, V = oracle.black_price(b.F, b.K, b.T, np.where(np.isfinite(ref), ref, 1.0), b.flag, nthreads=0)
    rows = (st == 0) & (V >= 1.0)  # the paper's well-conditioned band [1, 1e2)
    Pt = to_dev(P).requires_grad_(True)
    sig = pv.implied_volatility_autograd(Pt, to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag), 1e-6, "exact")
    sig.sum().backward()
    ad = to_np(Pt.grad)
    itm = np.where(b.flag > 0, np.maximum(b.F - b.K, 0), np.maximum(b.K - b.F, 0))
    h = 1e-4 * (P - itm)  # steps scale with the time value, so P +- 2h stays inside (intrinsic, upper)
    f = lambda dp: to_np(pv.iv(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(P + dp), to_dev(b.flag))[0])  # noqa
    # fourth-order central difference (Richardson): truncation O(h^4), rounding ~ eps sigma / h
    fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
    rel = np.abs(fd[rows] - ad[rows]) / np.abs(ad[rows])
    assert rows.sum() > 1000
    assert np.median(rel) < 1e-10 and rel.max() < 1e-8


def test_black_price_autograd_matches_oracle():
    b = workloads.body_batch(4096, seed=22)
    g = np.random.default_rng(2).normal(size=b.n)
    st = to_dev(b.sigma_star).requires_grad_(True)
    Ft, Kt, Tt = (to_dev(a).requires_grad_(True) for a in (b.F, b.K, b.T))
    P = pv.black_price_autograd(st, Ft, Kt, Tt, to_dev(b.flag))
    (P * to_dev(g)).sum().backward()
    want = oracle.black_price_grad(b.F, b.K, b.T, b.sigma_star, b.flag, g, nthreads=0)
    got = [to_np(t.grad) for t in (st, Ft, Kt, Tt)]
    s = b.sigma_star * np.sqrt(b.T)
    cond = 1 + 0.5 * (np.log(b.F / b.K) / s) ** 2 + s * s / 8
    for name, gg, ww in zip(("dsigma", "dF", "dK", "dT"), got, want):
        rel = np.abs(gg - ww) / np.maximum(np.abs(ww), 1e-300)
        ok = np.abs(ww) > 1e-280
        assert np.all(rel[ok] <= 64 * 2.2e-16 * cond[ok]), name


def test_two_vega_identity():
    """d/dsigma_hat (sigma_rt - sigma*)^2 = 2 (sigma_rt - sigma*) (1/V) V (SPX appendix, Eq. two_vega)."""
    b = workloads.body_batch(4096, seed=23)
    sig_star = to_dev(b.sigma_star)
    sig_hat = (sig_star * 1.1).detach().requires_grad_(True)
    F, K, T, flag = to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag)
    P_hat = pv.black_price_autograd(sig_hat, F, K, T, flag)
    sig_rt = pv.implied_volatility_autograd(P_hat, F, K, T, flag, 1e-6, "exact")
    ((sig_rt - sig_star) ** 2).sum().backward()
    _, V = pv.black_price(F, K, T, sig_hat.detach(), flag)
    rows = to_np(V) > 1e-2
    want = to_np(2 * (sig_rt - sig_star))
    got = to_np(sig_hat.grad)
    rel = np.abs(got[rows] - want[rows]) / np.abs(want[rows])
    assert rows.sum() > 3000 and rel.max() < 1e-10


def test_nan_poisoning_contract():
    """Without a gate the documented NaN branch (|V| <= 1e-14) poisons Adam at once; with the
    smooth gate every parameter stays finite (the paper's NaN-poisoning diagnostic)."""
    chain = workloads.low_vega_chain(65536, seed=31)
    _, V = oracle.black_price(chain.F, chain.K, chain.T, chain.sigma_star, chain.flag, nthreads=0)
    assert np.mean(np.abs(V) <= 1e-14) > 0.5  # the chain lives in the singular tail
    naive = training.per_quote_round_trip(chain, steps=3, gated=False)
    gated = training.per_quote_round_trip(chain, steps=20, gated=True)
    assert naive["finite_frac"][0] < 0.5
    assert all(f == 1.0 for f in gated["finite_frac"])
    assert all(np.isfinite(gated["loss"]))


def test_svi_iv_loss_training():
    """Adam through the operator on synthetic SVI surfaces: the IV loss falls and no gradient is NaN."""
    batch = workloads.svi_batch(64, seed=5)
    out = training.train_iv_loss(batch, steps=60, lr=1e-3, tau=1e-6, gate="smooth")
    assert out["nan_grad_steps"] == 0
    assert np.all(np.isfinite(out["loss"]))
    assert out["loss"][-1] < 0.1 * out["loss"][0]


def test_svi_iv_loss_full_size():
    """Configuration 5 as specified: 1,024 SVI surfaces, ragged 50-400 quotes over 8 maturities, one
    MLP 2 -> 128 x 4 -> 1 pricer per surface, 100 Adam steps at lr 1e-3 through ImpliedVol."""
    batch = workloads.svi_batch(1024, seed=5)
    assert batch.n_surfaces == 1024 and batch.max_quotes <= 400
    out = training.train_iv_loss(batch, steps=100, lr=1e-3, tau=1e-6, gate="smooth")
    print(f"svi-1024: {out['quotes']} quotes, {1e3 * out['seconds'] / 100:.2f} ms/step, loss {out['loss'][0]:.4g} "
          f"-> {out['loss'][-1]:.4g}, gate kept {out['iv_gate_kept'][-1]:.4f}")
    assert out["nan_grad_steps"] == 0
    assert np.all(np.isfinite(out["loss"]))
    assert out["loss"][-1] <= 0.1 * out["loss"][0]
    assert min(out["iv_gate_kept"]) > 0.9
