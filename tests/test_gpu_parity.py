"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: status codes identical on every row; sigma within 1e-13 relative and
gradients within 1e-10 relative on the parity domain (status 0 and
kappa_P = P/(sigma V) <= 100); elsewhere sigma within a bound scaled by the
conditioning kappa_beta = (P - intrinsic)/(sigma V) of the time value.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import _native, workloads  # noqa: E402

pytestmark = pytest.mark.gpu

from gpu_helpers import (DEV, EPS, assert_grad_offdomain, assert_grad_parity, assert_sigma_parity,  # noqa: E402
                         conditioning, oracle_inputs, to_dev, to_np)


@pytest.fixture(scope="module")
def body():
    b = workloads.body_batch(workloads.SMALL_N, seed=1)
    P = oracle_inputs(b)
    ref, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    return b, P, ref, st


@pytest.fixture(scope="module")
def stress():
    b = workloads.stress_batch(65536, seed=2)
    P = oracle_inputs(b)
    ref, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    return b, P, ref, st


def gpu_iv(b, P, **kw):
    sig, st = pv.iv(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(P), to_dev(b.flag), **kw)
    torch.cuda.synchronize()
    return to_np(sig), to_np(st)


def test_black_price_parity():
    for b in (workloads.body_batch(20000, seed=3), workloads.stress_batch(20000, seed=4, boundary_frac=0.0)):
        P, V = pv.black_price(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.sigma_star), to_dev(b.flag))
        Pr, Vr = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag, nthreads=0)
        P, V = to_np(P), to_np(V)
        s = b.sigma_star * np.sqrt(b.T)
        cond = 1 + 0.5 * (np.log(b.F / b.K) / s) ** 2 + s * s / 8
        tiny = Pr < 1e-300
        relP = np.abs(P - Pr) / np.maximum(Pr, 1e-300)
        assert np.all(relP[~tiny] <= 32 * EPS * cond[~tiny])
        relV = np.abs(V - Vr) / np.maximum(Vr, 1e-300)
        assert np.all(relV[Vr > 1e-300] <= 32 * EPS * cond[Vr > 1e-300])


def test_forward_parity_body(body):
    b, P, ref, st_ref = body
    sig, st = gpu_iv(b, P)
    dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where="body")
    assert dom.mean() > 0.85


def test_forward_parity_stress(stress):
    b, P, ref, st_ref = stress
    sig, st = gpu_iv(b, P)
    dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where="stress")
    assert dom.sum() > 10000


@pytest.mark.parametrize("steps", [2, 3, 4])
def test_householder_steps(body, steps):
    b, P, ref, st_ref = body
    sig, st = gpu_iv(b, P, householder=steps)
    assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"steps={steps}")


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_backward_parity(body, stress, mode):
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        rng = np.random.default_rng(mode)
        g = rng.normal(size=b.n)
        g[::5] = 0.0
        kp, _ = conditioning(b.F, b.K, b.T, P, b.flag, ref)
        _, Vr = oracle.black_price(b.F, b.K, b.T, np.where(np.isfinite(ref), ref, 1.0), b.flag, nthreads=0)
        tau = float(np.median(Vr[st_ref == 0])) * 0.1
        want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, g, tau, mode, nthreads=0)
        got = pv.iv_backward(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag), to_dev(ref), to_dev(g),
                             tau=tau, gate=mode)
        got = [to_np(x) for x in got]
        # same sigma on both sides: every row is compared
        assert_grad_parity(got, want, np.ones(b.n, bool), where=f"{name} mode={mode}", vega=Vr, gbar=g)


def test_forward_backward_fused_parity(body, stress):
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        tau = 1e-6
        out = pv.iv_forward_backward(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(P), to_dev(b.flag), tau=tau,
                                     gate="nan")
        sig, st, *grads = [to_np(x) for x in out]
        dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"fused {name}")
        want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, None, tau, 1, nthreads=0)
        assert_grad_parity(grads, want, dom, where=f"fused {name}")
        # sigma from the separate forward is the same bits
        sig2, _ = gpu_iv(b, P)
        assert np.array_equal(sig, sig2, equal_nan=True)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("gate", [0, 1, 2, 3])
def test_fused_with_upstream_gradient(body, stress, form, gate):
    """The fused kernels with an upstream gradient gbar (their own adjoint instantiation: the
    products by g kept), every gate, zeros and a NaN among the cotangents: against the oracle's
    VJP with the same cotangents on the parity domain; and with g = 1 on every row, the same bits
    as the call without gbar in the gates where g multiplies the result last."""
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        rng = np.random.default_rng(50 + gate)
        g = rng.normal(size=b.n)
        g[::7] = 0.0
        g[3] = np.nan
        _, Vr = oracle.black_price(b.F, b.K, b.T, np.where(np.isfinite(ref), ref, 1.0), b.flag, nthreads=0)
        tau = float(np.median(Vr[st_ref == 0])) * 0.1
        args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
        sig, st, *grads = [to_np(x) for x in pv.iv_forward_backward(*args, to_dev(g), tau=tau, gate=gate, mode=form)]
        dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"gbar {form} {name}")
        want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, g, tau, gate, nthreads=0)
        assert_grad_parity(grads, want, dom, where=f"gbar {form} {name} gate={gate}", vega=Vr, gbar=g)
        if gate != 3:
            ones = [to_np(x) for x in pv.iv_forward_backward(*args, to_dev(np.ones(b.n)), tau=tau, gate=gate,
                                                              mode=form)]
            none = [to_np(x) for x in pv.iv_forward_backward(*args, tau=tau, gate=gate, mode=form)]
            for x, y in zip(ones, none):
                assert np.array_equal(x, y, equal_nan=True), f"gbar = 1 vs no gbar, {form} {name} gate={gate}"


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_fused_gradients_off_parity_domain(body, stress, mode):
    """The fused kernels' adjoint (the last Householder evaluation's Mills ratios reused) on
    solved rows outside the parity domain: against the oracle at the GPU's sigma, and against
    the oracle at its own sigma under the conditioning-scaled bound."""
    checked = 0
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
        sig, st, *g_nan = [to_np(x) for x in pv.iv_forward_backward(*args, tau=1e-6, gate="nan", mode=mode)]
        _, _, *g_exact = [to_np(x) for x in pv.iv_forward_backward(*args, tau=1e-6, gate="exact", mode=mode)]
        assert np.array_equal(st, st_ref)
        checked += assert_grad_offdomain(b.F, b.K, b.T, P, b.flag, sig, st, ref, g_nan, g_exact,
                                         where=f"{mode} {name}")
    assert checked > 10000, checked


def tiny_root_rows():
    """The oracle pins' tiny-root rows: ATM quotes priced down to subnormal time values, and deep
    lower-tail quotes (beta < 1e-30, |ln(F/K)| up to 6, beta down to subnormal)."""
    import test_oracle_tiny_roots as TR
    F1, K1, T1, P1, f1 = TR.atm_rows()
    F2, K2, T2, P2, f2 = TR.deep_tail_rows()
    cat = np.concatenate
    return cat([F1, F2]), cat([K1, K2]), cat([T1, T2]), cat([P1, P2]), cat([f1, f2]).astype(np.int8)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_tiny_roots(mode):
    F, K, T, P, flag = tiny_root_rows()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    args = [to_dev(a) for a in (F, K, T, P, flag)]
    sig, st, *grads = [to_np(x) for x in pv.iv_forward_backward(*args, tau=1e-300, gate="exact", mode=mode)]
    # subnormal sigma: the bound is one subnormal ulp of s and of s / sqrt(T) on top of the relative one
    sub = ref < 2.3e-308
    assert_sigma_parity(F[~sub], K[~sub], T[~sub], P[~sub], flag[~sub], sig[~sub], st[~sub], ref[~sub],
                        st_ref[~sub], where=f"tiny roots {mode}")
    tiny = 4.9406564584124654e-324
    assert np.array_equal(st[sub], st_ref[sub])
    assert np.all(np.abs(sig[sub] - ref[sub]) <= 8 * EPS * ref[sub] + 2 * tiny * (1 + 1 / np.sqrt(T[sub])))
    want = oracle.iv_grad(F, K, T, flag, ref, None, 0.0, 0)
    _, Vr = oracle.black_price(F, K, T, np.where(np.isfinite(ref), ref, 1.0), flag)
    kp, _ = conditioning(F, K, T, P, flag, ref)
    dom = (st_ref == 0) & (kp <= 100) & ~sub
    assert_grad_parity(grads, want, dom, where=f"tiny roots {mode}", vega=Vr)


def test_counters_match_outputs(stress):
    """pivot_opts.counters: rows by status equal the status array's histogram, bins add up to the
    solved rows, rejected rows of the mixed form are among its float-seeded ones."""
    b, P, ref, st_ref = stress
    args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]
    for mode, nbins in (("fp64", 8), ("mixed", 12)):
        c = pv.new_counters(DEV)
        sig, st = pv.iv(*args, mode=mode, counters=c)
        c2 = pv.new_counters(DEV)
        pv.iv_forward_backward(*args, mode=mode, counters=c2)
        c, c2 = to_np(c), to_np(c2)
        assert np.array_equal(c, c2)
        hist = np.bincount(to_np(st), minlength=6)
        assert np.array_equal(c[:6], hist), (c[:6], hist)
        assert c[6:6 + nbins].sum() == hist[0] and np.all(c[6 + nbins:18] == 0)
        assert np.all(c[19:] == 0)
        if mode == "fp64":
            assert c[18] == 0
        else:
            assert c[18] <= c[6:10].sum() + c[6 + 8:6 + 12].sum()
    # counters add across calls and are left alone when not requested
    c = pv.new_counters(DEV)
    pv.iv(*args, counters=c)
    pv.iv(*args)
    pv.iv(*args, counters=c)
    assert np.array_equal(to_np(c)[:6], 2 * np.bincount(st_ref, minlength=6))


def test_probes():
    """pivot_probe_units runs and reports its work; pivot_probe_stream moves every row exactly."""
    from paper_2606_17065_gb300 import api
    for unit in api.PROBE_UNITS:
        ops = api.probe_units(unit, 4, blocks_per_sm=2)
        assert ops == 152 * 2 * 256 * 4 * 64 or ops > 0
    torch.cuda.synchronize()
    n = 4097
    b = workloads.stress_batch(n, seed=5)
    F, K, T, P = (to_dev(a) for a in (b.F, b.K, b.T, b.sigma_star))
    flag = to_dev(b.flag)
    for width in (1, 2):
        outs = [torch.full((n,), np.nan, dtype=torch.float64, device=DEV), torch.zeros(n, dtype=torch.uint8,
                                                                                       device=DEV)]
        outs += [torch.full((n,), np.nan, dtype=torch.float64, device=DEV) for _ in range(4)]
        api.probe_stream(width, F, K, T, P, flag, outs)
        sig, st, dP, dF, dK, dT = (to_np(o) for o in outs)
        assert np.array_equal(sig, b.sigma_star) and np.array_equal(dT, b.sigma_star)
        assert np.array_equal(dP, b.F) and np.array_equal(dF, b.K) and np.array_equal(dK, b.T)
        assert np.array_equal(st.view(np.int8), b.flag)


def edge_rows():
    F, K, T, P, flag = [], [], [], [], []

    def add(f, k, t, p, fl):
        F.append(f); K.append(k); T.append(t); P.append(p); flag.append(fl)

    add(100.0, 100.0, 1.0, 7.96, 1)          # at the money
    add(100.0, 100.0, 1.0, 7.96, -1)
    add(100.0, 100.0 * (1 + 1e-12), 0.5, 3.0, 1)  # |x| ~ 1e-12
    add(100.0, 100.0, 1.0, 1e-300, 1)        # ATM, tiny price
    add(100.0, 100.0, 1.0, 99.999999, 1)     # ATM, price near the upper bound
    add(100.0, 120.0, 1.0, 0.0, 1)           # OTM call at zero: at intrinsic
    add(100.0, 80.0, 1.0, 20.0, 1)           # ITM call at intrinsic
    add(100.0, 80.0, 1.0, 20.0 + 1e-10, 1)   # just above intrinsic
    add(100.0, 80.0, 1.0, 19.9, 1)           # below intrinsic
    add(100.0, 80.0, 1.0, 100.0, 1)          # at the upper bound F
    add(100.0, 80.0, 1.0, 100.5, 1)          # above the upper bound
    add(100.0, 80.0, 1.0, 80.0, -1)          # put at the upper bound K
    add(100.0, 80.0, 1.0, 79.9999999, -1)    # put just below the upper bound: huge sigma
    add(100.0, 150.0, 1e-8, 1e-200, 1)       # tiny T, deep OTM
    add(100.0, 60.0, 2.0, 1e-310, -1)        # subnormal price
    add(100.0, 100.0 * np.exp(-6), 3.0, 99.7, 1)  # deep ITM, price near F
    add(100.0, 100.0, 0.0, 5.0, 1)           # T = 0
    add(-1.0, 100.0, 1.0, 5.0, 1)            # F < 0
    add(100.0, 100.0, 1.0, np.nan, 1)        # NaN price
    add(100.0, np.inf, 1.0, 5.0, 1)          # inf strike
    add(100.0, 100.0, 1.0, 5.0, 0)           # bad flag
    add(100.0, 100.0, 1.0, 5.0, 3)           # bad flag
    add(1e-100, 1e-100, 1.0, 3e-102, 1)      # tiny scale
    add(1e100, 2e100, 1.0, 1e98, -1)         # large scale
    add(100.0, 100.0 * np.exp(0.3), 1.0, 1e-3, 1)
    add(100.0, 100.0 * np.exp(-0.3), 1.0, 30.0 + 1e-3, 1)
    return (np.array(F), np.array(K), np.array(T), np.array(P), np.array(flag, np.int8))


def test_edge_cases():
    F, K, T, P, flag = edge_rows()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    sig, st = pv.iv(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag))
    sig, st = to_np(sig), to_np(st)
    assert_sigma_parity(F, K, T, P, flag, sig, st, ref, st_ref, where="edge")
    for mode in range(4):
        want = oracle.iv_grad(F, K, T, flag, ref, None, 1e-6, mode)
        got = [to_np(x) for x in pv.iv_backward(to_dev(F), to_dev(K), to_dev(T), to_dev(flag), to_dev(ref),
                                                 tau=1e-6, gate=mode)]
        _, Vr = oracle.black_price(F, K, T, np.where(np.isfinite(ref), ref, 1.0), flag)
        assert_grad_parity(got, want, np.ones(len(F), bool), where=f"edge mode={mode}", vega=Vr)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 255, 257, 4097])
def test_ragged_sizes(n):
    b = workloads.body_batch(n, seed=100 + n)
    P = oracle_inputs(b)
    ref, st_ref = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    sig, st = gpu_iv(b, P)
    assert sig.shape == (n,)
    assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"n={n}")


def test_empty_batch():
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    sig, st = pv.iv(e, e, e, e, torch.empty(0, dtype=torch.int8, device=DEV))
    assert sig.numel() == 0 and st.numel() == 0


def test_capi_argument_errors():
    lib = _native.lib()
    n = 8
    d = torch.ones(n, dtype=torch.float64, device=DEV)
    fl = torch.ones(n, dtype=torch.int8, device=DEV)
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    host = torch.ones(n, dtype=torch.float64)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.pivot_iv_forward(-1, p(d), p(d), p(d), p(d), p(fl), p(out), None, None, s) == 1
    assert lib.pivot_iv_forward(n, None, p(d), p(d), p(d), p(fl), p(out), None, None, s) == 2
    assert lib.pivot_iv_forward(n, p(host), p(d), p(d), p(d), p(fl), p(out), None, None, s) == 5
    mis = ctypes.c_void_p(d.data_ptr() + 4)
    assert lib.pivot_iv_forward(n - 1, mis, p(d), p(d), p(d), p(fl), p(out), None, None, s) == 6
    bad = _native.PivotOpts()
    bad.mode, bad.householder = 0, 9
    assert lib.pivot_iv_forward(n, p(d), p(d), p(d), p(d), p(fl), p(out), None, ctypes.byref(bad), s) == 4
    assert lib.pivot_iv_backward(n, p(d), p(d), p(d), p(fl), p(d), None, -1.0, 1, p(out), None, None, None, s) == 3
    assert lib.pivot_iv_backward(n, p(d), p(d), p(d), p(fl), p(d), None, 0.0, 3, p(out), None, None, None, s) == 3
    assert lib.pivot_iv_backward(n, p(d), p(d), p(d), p(fl), p(d), None, 1e-6, 7, p(out), None, None, None, s) == 3
    assert lib.pivot_iv_forward(0, None, None, None, None, None, None, None, None, s) == 0
    with pytest.raises(_native.PivotError):
        pv.iv(host.to(DEV), d, d, d, fl, mode=5)


def test_host_tensors_round_trip(body):
    """The end-to-end path: host tensors in, host tensors out."""
    b, P, ref, st_ref = body
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    sig, st = pv.iv(t(b.F), t(b.K), t(b.T), t(P), t(b.flag))
    assert not sig.is_cuda
    assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig.numpy(), st.numpy(), ref, st_ref, where="host")


@pytest.mark.parametrize("call", ["iv", "iv_forward_backward", "bs_iv", "bs_iv_forward_backward"])
def test_host_chunked_pipeline_matches_device_path(monkeypatch, call):
    """Host inputs above the chunk size are streamed in chunks (copy-in and kernel streams taking
    turns, one copy-out stream); every output is bit-identical to one call on device-resident
    inputs (ragged last chunk included)."""
    from paper_2606_17065_gb300 import api
    monkeypatch.setattr(api, "HOST_CHUNK", 4096)
    n = 3 * 4096 + 77
    if call.startswith("bs"):
        b = workloads.bs_batch(n, seed=211, wide=True)
        V, _ = oracle.bs_price(b.S, b.K, b.T, b.r, b.q, b.sigma_star, b.flag, nthreads=0)
        arrays = [b.S, b.K, b.T, b.r, b.q, V, b.flag]
    else:
        b = workloads.stress_batch(n, seed=212)
        arrays = [b.F, b.K, b.T, oracle_inputs(b), b.flag]
    fn = getattr(pv, call)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]
    dev = [h.to(DEV) for h in host]
    got = fn(*host)
    want = fn(*dev)
    got = [g for g in got if g is not None]
    want = [w for w in want if w is not None]
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert not g.is_cuda
        assert torch.equal(torch.nan_to_num(g.double(), nan=7.0), torch.nan_to_num(w.cpu().double(), nan=7.0))


@pytest.mark.parametrize("streams", [2, 4, 5])
def test_host_staging_reused_across_calls(monkeypatch, streams):
    """The kept staging buffers and the copy-out stream: two different batches in a row, with
    2 to 5 streams (1 to 4 copy-in/kernel streams), each give the device path's bits; after
    release_host_buffers the next call allocates afresh and still matches."""
    from paper_2606_17065_gb300 import api
    monkeypatch.setattr(api, "HOST_CHUNK", 4096)
    monkeypatch.setattr(api, "HOST_STREAMS", streams)
    monkeypatch.setattr(api, "_streams", {})
    for k, seed in enumerate((214, 215, 216)):
        if k == 2:
            pv.release_host_buffers()
        n = 5 * 4096 + 13 * k
        b = workloads.stress_batch(n, seed=seed)
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (b.F, b.K, b.T, oracle_inputs(b), b.flag)]
        got = pv.iv_forward_backward(*host)
        want = pv.iv_forward_backward(*[h.to(DEV) for h in host])
        for g, w in zip(got, want):
            assert torch.equal(torch.nan_to_num(g.double(), nan=7.0), torch.nan_to_num(w.cpu().double(), nan=7.0))


def test_host_outputs_given_by_the_caller(monkeypatch):
    """iv_forward_backward(..., out=...) writes the caller's host tensors, chunked or not, with the
    same bits as the device path; a wrong dtype or length is refused."""
    from paper_2606_17065_gb300 import api
    monkeypatch.setattr(api, "HOST_CHUNK", 4096)
    for n in (1000, 3 * 4096 + 77):
        b = workloads.stress_batch(n, seed=213)
        arrays = [b.F, b.K, b.T, oracle_inputs(b), b.flag]
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]
        out = [torch.empty(n, dtype=d).pin_memory() for d in (torch.float64, torch.uint8) + (torch.float64,) * 4]
        got = pv.iv_forward_backward(*host, out=out)
        assert all(g is o for g, o in zip(got, out))
        want = pv.iv_forward_backward(*[h.to(DEV) for h in host])
        for g, w in zip(got, want):
            assert torch.equal(torch.nan_to_num(g.double(), nan=7.0), torch.nan_to_num(w.cpu().double(), nan=7.0))
    with pytest.raises(ValueError):
        pv.iv_forward_backward(*host, out=out[:5])
    with pytest.raises(ValueError):
        pv.iv_forward_backward(*[h.to(DEV) for h in host], out=out)


def test_full_size_stress_sampled():
    """16M stress rows in the benchmark's launch configuration; sampled rows checked one by one."""
    b = workloads.stress_batch(workloads.STRESS_N, seed=2)
    F, K, T, flag = to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag)
    P_dev, _ = pv.black_price(F, K, T, to_dev(b.sigma_star), flag, vega=False)
    fixed = torch.from_numpy(b.P_fixed).to(DEV)
    P_dev = torch.where(torch.isnan(fixed), P_dev, fixed)
    idx = workloads.sample_indices(b.n, 20000, seed=9)
    sb = b.subset(idx)
    P_s = oracle_inputs(sb)  # the oracle's own prices on the sampled rows
    P_dev[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(P_s).to(DEV)
    sig, st, dP, dF, dK, dT = pv.iv_forward_backward(F, K, T, P_dev, flag, tau=1e-6, gate="nan")
    torch.cuda.synchronize()
    ref, st_ref = oracle.implied_vol(sb.F, sb.K, sb.T, P_s, sb.flag, nthreads=0)
    sig_s, st_s = to_np(sig[torch.from_numpy(idx).to(DEV)]), to_np(st[torch.from_numpy(idx).to(DEV)])
    dom = assert_sigma_parity(sb.F, sb.K, sb.T, P_s, sb.flag, sig_s, st_s, ref, st_ref, where="16M sample")
    want = oracle.iv_grad(sb.F, sb.K, sb.T, sb.flag, ref, None, 1e-6, 1, nthreads=0)
    got = [to_np(g[torch.from_numpy(idx).to(DEV)]) for g in (dP, dF, dK, dT)]
    assert_grad_parity(got, want, dom, where="16M sample")
    # properties over every row: status in range, sigma finite and > 0 exactly on status 0
    st_all = to_np(st)
    sig_all = to_np(sig)
    assert st_all.max() <= 5
    ok = st_all == 0
    assert np.all(np.isfinite(sig_all[ok]) & (sig_all[ok] > 0))
    assert np.all(np.isnan(sig_all[np.isin(st_all, [1, 2, 3])]))


# ---------------------------------------------------------------------------
# Mixed precision: float node, guess and first Householder step; FP64 final
# step, adjoint, and every row outside the float range.  Same bar as FP64.
# ---------------------------------------------------------------------------
def test_mixed_forward_parity(body, stress):
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        sig, st = gpu_iv(b, P, mode="mixed")
        assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"mixed {name}")


def test_mixed_fused_parity(body, stress):
    for name, (b, P, ref, st_ref) in (("body", body), ("stress", stress)):
        out = pv.iv_forward_backward(to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(P), to_dev(b.flag), tau=1e-6,
                                     gate="nan", mode="mixed")
        sig, st, *grads = [to_np(x) for x in out]
        dom = assert_sigma_parity(b.F, b.K, b.T, P, b.flag, sig, st, ref, st_ref, where=f"mixed fused {name}")
        want = oracle.iv_grad(b.F, b.K, b.T, b.flag, ref, None, 1e-6, 1, nthreads=0)
        assert_grad_parity(grads, want, dom, where=f"mixed fused {name}")


@pytest.mark.parametrize("steps", [2, 3])
def test_mixed_edge_cases_and_steps(steps):
    F, K, T, P, flag = edge_rows()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    sig, st = pv.iv(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag), mode="mixed", householder=steps)
    assert_sigma_parity(F, K, T, P, flag, to_np(sig), to_np(st), ref, st_ref, where=f"mixed edge steps={steps}")


def test_full_size_mixed_sampled():
    """64M rows of the body distribution (the mixed-precision workload), sampled rows checked one by one."""
    b = workloads.body_batch(workloads.LARGE_N, seed=3)
    F, K, T, flag = to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag)
    P_dev, _ = pv.black_price(F, K, T, to_dev(b.sigma_star), flag, vega=False)
    idx = workloads.sample_indices(b.n, 20000, seed=10)
    sb = b.subset(idx)
    P_s = oracle_inputs(sb)
    tidx = torch.from_numpy(idx).to(DEV)
    P_dev[tidx] = torch.from_numpy(P_s).to(DEV)
    sig, st, dP, dF, dK, dT = pv.iv_forward_backward(F, K, T, P_dev, flag, tau=1e-6, gate="nan", mode="mixed")
    torch.cuda.synchronize()
    ref, st_ref = oracle.implied_vol(sb.F, sb.K, sb.T, P_s, sb.flag, nthreads=0)
    dom = assert_sigma_parity(sb.F, sb.K, sb.T, P_s, sb.flag, to_np(sig[tidx]), to_np(st[tidx]), ref, st_ref,
                              where="64M mixed sample")
    want = oracle.iv_grad(sb.F, sb.K, sb.T, sb.flag, ref, None, 1e-6, 1, nthreads=0)
    assert_grad_parity([to_np(g[tidx]) for g in (dP, dF, dK, dT)], want, dom, where="64M mixed sample")
    # every row: the mixed result equals the plain FP64 result to the same bar
    sig64, st64 = pv.iv(F, K, T, P_dev, flag, mode="fp64")
    assert torch.equal(st, st64)
    _, V64 = pv.black_price(F, K, T, torch.where(st64 == 0, sig64, torch.ones_like(sig64)), flag)
    dom_all = (st64 == 0) & (P_dev <= 100 * sig64 * V64)  # the parity domain, every row
    rel = ((sig[dom_all] - sig64[dom_all]).abs() / sig64[dom_all]).max().item()
    assert rel <= 2e-13, rel
    del F, K, T, flag, P_dev, sig, st, dP, dF, dK, dT, sig64, st64
    torch.cuda.empty_cache()


def test_mills_ratio_fp64_table():
    """The library's FP64 Mills ratio (table in w = -z, asymptotic series, reflection for z > 0)
    through Y = Phi/phi, against the oracle's quadrature Mills ratio."""
    # the table's interval ends in w = -z (0, 1/16, then 16 parts per binade up to 128), each with
    # its neighbours, and the switch to the asymptotic series at w = 128
    ends = np.concatenate([[2.0 ** e * (1 + m / 16) for e in range(-4, 7) for m in range(16)], [128.0]])
    z_ends = -np.concatenate([ends, np.nextafter(ends, 0), np.nextafter(ends, np.inf)])
    z = np.concatenate([np.linspace(-37.0, 37.0, 20001), -np.logspace(-12, 3, 400), np.logspace(-12, 1.5, 400),
                        np.linspace(-140.0, -120.0, 2001), z_ends, [0.0, -0.0, np.inf, -np.inf]])
    y = to_np(pv.api.mills_ratio(to_dev(z)))
    ref = np.array([oracle.mills(v) for v in z])
    fin = np.isfinite(ref) & (ref > 0)
    # conditioning of Y in z: |z Y'/Y| ~ z^2 for z > 0 (exp(z^2/2) growth)
    tol = 8 * EPS * (1 + np.where(z > 0, z * z, 0.0))
    rel = np.abs(y[fin] - ref[fin]) / ref[fin]
    assert np.all(rel <= tol[fin]), rel.max()
    assert y[z == -np.inf][0] == 0.0 and np.isinf(y[z == np.inf][0])


def test_extreme_moneyness():
    """|ln(F/K)| from 50 to 1400 (b_max down to e^-700): the reflections through 1/b_s and the
    adjoint's large Mills ratios stay finite where the exact values are."""
    F, K, T, S, flag = [], [], [], [], []
    for ax in (50.0, 300.0, 690.0, 1000.0, 1400.0):
        sc = np.sqrt(2 * ax)
        for sfac in (0.6, 0.9, 1.0, 1.1, 1.5):
            for fl in (1, -1):
                for side in (1, -1):
                    f = np.exp(side * ax / 2)
                    F.append(f); K.append(1.0 / f); T.append(1.0); S.append(sfac * sc); flag.append(fl)
    F, K, T, S = map(np.array, (F, K, T, S))
    flag = np.array(flag, np.int8)
    P, _ = oracle.black_price(F, K, T, S, flag)
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag)
    assert (st_ref == 0).sum() >= 24  # in-the-money rows collapse onto a bound at these scales
    for form in ("fp64", "mixed"):
        sig, st = pv.iv(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag), mode=form)
        sig, st = to_np(sig), to_np(st)
        dom = assert_sigma_parity(F, K, T, P, flag, sig, st, ref, st_ref, where=f"extreme {form}")
        for mode in (0, 1):
            out = pv.iv_forward_backward(to_dev(F), to_dev(K), to_dev(T), to_dev(P), to_dev(flag), tau=1e-300,
                                         gate=mode, mode=form)
            want = oracle.iv_grad(F, K, T, flag, ref, None, 1e-300, mode)
            _, Vr = oracle.black_price(F, K, T, np.where(np.isfinite(ref), ref, 1.0), flag)
            assert_grad_parity([to_np(x) for x in out[2:]], want, dom, where=f"extreme {form} gate={mode}",
                               vega=Vr)
