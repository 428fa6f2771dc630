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
    # Element by element.  The two sides round to BF16 at the same points, but the kernel's SiLU
    # goes through the hardware tanh (relative error below 2^-10.9), so a stored BF16 value (an
    # activation, a SiLU derivative product, a backpropagated dZ) may land one BF16 ulp (2^-8
    # relative) away from the reference's.  A product on the path of an element has at most six
    # such factors (a3 or a2 or a1, silu', dZ3, dZ2, silu', the feature in FP32), so each term
    # moves by at most 6 * 2^-8 of its magnitude; FP32 accumulation over 1,000 rows adds < 1e-4.
    mags = MR.grad_magnitudes(to_np(params).astype(np.float64), np.where(valid[:, None], f, 0.0),
                              np.where(valid, y, 0.0), valid)
    tol = (6 * 2.0 ** -8 + 1e-4) * mags + 1e-30
    ratio = np.abs(g - ref_grad) / tol
    assert ratio.max() <= 1.0, (int(ratio.argmax()), float(ratio.max()))
    # and in aggregate, per layer, the deviation is far below that worst case
    for name, lo, hi in (("w1", 0, 128), ("b1", 128, 192), ("w2", 192, 4288), ("b2", 4288, 4352),
                         ("w3", 4352, 8448), ("b3", 8448, 8512), ("w4", 8512, 8576), ("b4", 8576, 8577)):
        err = np.linalg.norm(g[lo:hi] - ref_grad[lo:hi]) / np.linalg.norm(ref_grad[lo:hi])
        assert err < 1e-2, (name, err)
    print("MLP gradient: max element deviation / bound", float(ratio.max()),
          "median", float(np.median(ratio)))


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


def test_learned_off_domain_gradients_and_counters(trained):
    """The learned form's fused adjoint off the parity domain (as for the plain and mixed forms),
    and its counters: statuses match, every solved row is in an MLP bin or went to the fallback."""
    from gpu_helpers import DEV, assert_grad_offdomain
    b = workloads.stress_batch(65536, seed=65)
    P = oracle_inputs(b)
    ref, st_ref = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
    c = pv.new_counters(DEV)
    sig, st, *g_nan = [to_np(x) for x in pv.iv_forward_backward(*args, tau=1e-6, gate="nan", mode="learned",
                                                                 mlp=trained, counters=c)]
    _, _, *g_exact = [to_np(x) for x in pv.iv_forward_backward(*args, tau=1e-6, gate="exact", mode="learned",
                                                                mlp=trained)]
    assert np.array_equal(st, st_ref)
    assert assert_grad_offdomain(b.F, b.K, b.T, P, b.flag, sig, st, ref, g_nan, g_exact, where="learned") > 1000
    c = to_np(c)
    hist = np.bincount(st, minlength=6)
    assert np.array_equal(c[:6], hist)
    assert c[6:12].sum() <= hist[0] and c[18] >= hist[0] - c[6:12].sum() and c[18] <= hist[0]
    assert np.all(c[12:18] == 0)


def test_learned_edge_cases(trained):
    F, K, T, P, flag = edge_rows()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    sig, st = pv.iv(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag), mode="learned", mlp=trained)
    assert_sigma_parity(F, K, T, P, flag, to_np(sig), to_np(st), ref, st_ref, where="learned edge")
