"""The learned initial guess (PIVOT_MODE_LEARNED): MLP 2->64->64->64->1, BF16 weights, FP32
accumulation, trained by the library's own kernels on operator-generated pairs.

Checked: the training kernels' gradients against a CPU reference, the trained seed against
LBR's rational seed (what the network gains), and the learned forward / forward+backward
against the oracle at the same bar as the plain FP64 path (the fallback keeps rows outside
the network's training range on the rational path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import training, workloads  # noqa: E402

import mlp_reference as MR  # noqa: E402
from gpu_helpers import assert_grad_parity, assert_sigma_parity, oracle_inputs, to_dev, to_np  # noqa: E402
from test_gpu_parity import edge_rows  # noqa: E402

pytestmark = pytest.mark.gpu


def _features(b, P, sig):
    ax = np.abs(np.log(b.F / b.K))
    itm = np.where(b.flag > 0, np.maximum(b.F - b.K, 0), np.maximum(b.K - b.F, 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        beta = (P - itm) / np.sqrt(b.F * b.K)
        q = 1.0 / np.sqrt(-2.0 * np.log(beta))
        sa = ax * q + np.sqrt(2 * np.pi) * beta
        y = np.log(sig * np.sqrt(b.T) / sa)
    f = np.stack([ax.astype(np.float32), q.astype(np.float32)], 1).astype(np.float64)
    return f, y.astype(np.float32).astype(np.float64), np.isfinite(y) & (sig > 0)


def test_mlp_training_gradient_matches_cpu_reference():
    b = workloads.body_batch(1000, seed=61)
    P = oracle_inputs(b)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    tr = pv.MlpTrainer(seed=3)
    tr.grad(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(P), to_dev(b.flag), to_dev(sig))
    params, grad, loss_sum, rows, step = tr.fields()
    f, y, valid = _features(b, P, sig)
    valid &= st == 0
    ref_loss, ref_grad = MR.loss_and_grad(to_np(params).astype(np.float64), np.where(valid[:, None], f, 0.0),
                                          np.where(valid, y, 0.0), valid)
    assert rows == valid.sum() and step == 0
    assert abs(loss_sum - ref_loss) <= 1e-3 * ref_loss
    g = to_np(grad).astype(np.float64)
    for name, lo, hi in (("w1", 0, 128), ("b1", 128, 192), ("w2", 192, 4288), ("b2", 4288, 4352),
                         ("w3", 4352, 8448), ("b3", 8448, 8512), ("w4", 8512, 8576), ("b4", 8576, 8577)):
        err = np.linalg.norm(g[lo:hi] - ref_grad[lo:hi]) / np.linalg.norm(ref_grad[lo:hi])
        assert err < 1e-2, (name, err)


@pytest.fixture(scope="module")
def trained():
    trainer, hist, secs = training.train_learned_guess(n_rows=4 * 1024 * 1024, steps=4000, batch=16384, lr=3e-3,
                                                       seed=4)
    print("training loss history", hist, f"{secs:.1f} s")
    assert hist[-1][1] < 0.01 * hist[0][1], hist
    return trainer


def test_learned_seed_gains_over_rational_seed(trained):
    """The MLP seed against LBR's rational seed, relative error to the oracle's root."""
    b = workloads.body_batch(20000, seed=62)
    P = oracle_inputs(b)
    ref, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    ok = st == 0
    s_ref = ref * np.sqrt(b.T)
    args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
    s_mlp = to_np(pv.iv_guess(*args, mode="learned", mlp=trained))
    s_rat = to_np(pv.iv_guess(*args, mode="fp64"))
    e_mlp = np.abs(s_mlp[ok] / s_ref[ok] - 1)
    e_rat = np.abs(s_rat[ok] / s_ref[ok] - 1)
    q = [0.5, 0.9, 0.99]
    print("seed rel. error q50/q90/q99: mlp", np.quantile(e_mlp, q), "rational", np.quantile(e_rat, q))
    assert np.quantile(e_mlp, 0.99) < np.quantile(e_rat, 0.99)
    assert np.median(e_mlp) < 1e-2


def test_learned_forward_and_fused_parity(trained):
    for name, b in (("body", workloads.body_batch(4096, seed=63)), ("stress", workloads.stress_batch(20000, seed=64))):
        P = oracle_inputs(b)
        ref, st_ref = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
        args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
        sig, st = pv.iv(*args, mode="learned", mlp=trained)
        assert_sigma_parity(b.F, b.K, b.T, P, b.flag, to_np(sig), to_np(st), ref, st_ref, where=f"learned {name}")
        out = pv.iv_forward_backward(*args, tau=1e-6, gate="nan", mode="learned", mlp=trained)
        sig2, st2, *grads = [to_np(x) for x in out]
        dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig2, st2, ref, st_ref, where=f"learned fused {name}")
        want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, None, 1e-6, 1, nthreads=0)
        assert_grad_parity(grads, want, dom, where=f"learned fused {name}")


def test_learned_edge_cases(trained):
    F, K, T, P, flag = edge_rows()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    sig, st = pv.iv(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag), mode="learned", mlp=trained)
    assert_sigma_parity(F, K, T, P, flag, to_np(sig), to_np(st), ref, st_ref, where="learned edge")
