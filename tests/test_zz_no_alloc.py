"""pivot_mlp_grad_static: the MLP gradient pass with its scratch in a static device array of
the library, for callers that cannot allocate device memory.

Called through the C ABI (ctypes) and checked against pivot_mlp_grad, which accumulates into
the caller's pivot_mlp_trainer, on two calls in a row with different batches: the second call
must not carry the first call's sums.  The file is named so that pytest collects it last; it
also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import _native, training  # noqa: E402

pytestmark = pytest.mark.gpu

NPARAM = 8577
MAX_ROWS = 1 << 26
PIVOT_E_TOO_MANY = 8


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _static_grad(net_ptr, rows, device):
    F, K, T, P, flag, sig = rows
    grad = torch.full((NPARAM,), float("nan"), dtype=torch.float32, device=device)
    loss = torch.full((2,), float("nan"), dtype=torch.float64, device=device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    rc = _native.lib().pivot_mlp_grad_static(ctypes.c_void_p(net_ptr), F.numel(), _p(F), _p(K), _p(T), _p(P),
                                             _p(flag), _p(sig), _p(grad), _p(loss), stream)
    assert rc == 0, _native.error_string(rc)
    torch.cuda.synchronize(device)
    return grad.cpu().numpy().astype(np.float64), loss.cpu().numpy()


def _trainer_grad(seed, rows, device):
    tr = pv.MlpTrainer(device, seed=seed)
    tr.grad(*rows)
    _, grad, loss_sum, n, _ = tr.fields()
    return tr, grad.cpu().numpy().astype(np.float64), np.array([loss_sum, n])


def _close(got, want):
    g, l = got
    wg, wl = want
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(l))
    assert l[1] == wl[1]
    assert abs(l[0] - wl[0]) <= 1e-6 * abs(wl[0])
    err = np.linalg.norm(g - wg) / np.linalg.norm(wg)
    assert err <= 1e-5, err


def test_static_grad_matches_trainer_on_two_calls_in_a_row():
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    a = training.operator_pairs(200_000, seed=21, device=device)
    b = training.operator_pairs(150_000, seed=22, device=device)
    tr_a, ga, la = _trainer_grad(5, a, device)
    tr_b, gb, lb = _trainer_grad(5, b, device)
    assert la[1] > 0 and lb[1] > 0 and la[1] != lb[1]
    got_a = _static_grad(tr_a.weights_ptr(), a, device)
    got_b = _static_grad(tr_b.weights_ptr(), b, device)
    _close(got_a, (ga, la))
    _close(got_b, (gb, lb))
    # a repeat of the first batch gives the first result again
    _close(_static_grad(tr_a.weights_ptr(), a, device), (ga, la))


def test_static_grad_empty_batch_and_row_limit():
    device = torch.device("cuda", 0)
    tr = pv.MlpTrainer(device, seed=1)
    empty = tuple(torch.empty(0, dtype=dt, device=device) for dt in (torch.float64,) * 4 + (torch.int8, torch.float64))
    g, l = _static_grad(tr.weights_ptr(), empty, device)
    assert np.all(g == 0.0) and np.all(l == 0.0)
    # above the stated maximum: refused on the host before any launch
    rc = _native.lib().pivot_mlp_grad_static(ctypes.c_void_p(tr.weights_ptr()), MAX_ROWS + 1, *([None] * 8),
                                             ctypes.c_void_p(0))
    assert rc == PIVOT_E_TOO_MANY
    assert "2^26" in _native.error_string(rc)
