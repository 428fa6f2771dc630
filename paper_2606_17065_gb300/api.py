"""Torch-facing API over the C ABI (include/pivot.h).

PyTorch provides device memory and the current CUDA stream; every step of the
computation runs in the library's CUDA kernels.  Inputs may be CUDA tensors
(used in place when already float64 / int8 and contiguous) or CPU tensors, in
which case they are copied to the current CUDA device and the results copied
back (the end-to-end path).  There is no CPU implementation.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _native

ROW_OK, ROW_BELOW_INTRINSIC, ROW_ABOVE_UPPER, ROW_BAD_INPUT, ROW_AT_INTRINSIC, ROW_AT_UPPER = range(6)
GATES = {"exact": 0, "nan": 1, "mask": 2, "smooth": 3}
MODES = {"fp64": 0, "mixed": 1, "learned": 2}


def _gate(gate) -> int:
    if isinstance(gate, str):
        if gate not in GATES:
            raise ValueError(f"gate must be one of {sorted(GATES)}")
        return GATES[gate]
    return int(gate)


def _device_of(*ts):
    for t in ts:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            return t.device
    if not torch.cuda.is_available():
        raise RuntimeError("pivot needs a CUDA device (no CPU fallback)")
    return torch.device("cuda", torch.cuda.current_device())


def _on(t, device, dtype):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.device != device:
        t = t.to(device, non_blocking=True)
    if t.dtype != dtype:
        t = t.to(dtype)
    return t.contiguous()


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _host_result(inputs, outs):
    """Copy outputs back to the host when every given input was a host tensor."""
    host = all((not isinstance(t, torch.Tensor)) or not t.is_cuda for t in inputs if t is not None)
    if not host:
        return outs
    res = []
    for o in outs:
        if o is None:
            res.append(None)
            continue
        h = torch.empty(o.shape, dtype=o.dtype, pin_memory=True)
        h.copy_(o, non_blocking=True)
        res.append(h)
    torch.cuda.current_stream(outs[0].device).synchronize()
    return res


# Host inputs of more than this many rows are streamed through the device in
# chunks of this size on three CUDA streams, so that the host-to-device copy of
# one chunk, the kernels of the next and the device-to-host copy of a third
# overlap.
HOST_CHUNK = 1 << 22
HOST_STREAMS = 4  # three for copy-in and kernels, one for every copy-out
# The first and last chunk are split into halving pieces (1/8, 1/8, 1/4, 1/2 and back), so that
# the first kernel starts after a short copy and the last copy back is short.
HOST_RAMP = True
_streams = {}


def _host_chunk(n):
    """Rows per chunk of an n-row host call, or 0 for one unpipelined round trip: HOST_CHUNK on
    large calls; a quarter of the call (at least HOST_CHUNK / 8) down to HOST_CHUNK / 4 rows, so
    that mid-size calls overlap their copies with the kernels too; below that, 0."""
    if n <= HOST_CHUNK // 4:
        return 0
    return min(HOST_CHUNK, max(HOST_CHUNK // 8, -(-n // 4)))


def _chunks(n, C=None):
    """(start, rows) of the chunks of an n-row host call, C rows each (_host_chunk(n), or
    HOST_CHUNK where n is too small to pipeline)."""
    C = C or _host_chunk(n) or HOST_CHUNK
    sizes = [min(C, n - lo) for lo in range(0, n, C)]
    if HOST_RAMP and len(sizes) >= 3 and C >= 64:
        head = [C // 8, C // 8, C // 4, C - C // 8 - C // 8 - C // 4]
        last = sizes[-1]
        tail = [last - last // 2 - last // 4 - last // 8, last // 8, last // 4, last // 2][::-1]
        sizes = head + sizes[1:-1] + [m for m in tail if m > 0]
    out, lo = [], 0
    for m in sizes:
        out.append((lo, m))
        lo += m
    return out


_staging = {}
_staging_lock = threading.Lock()


def _staging_buffers(dev, in_dtypes, out_dtypes, nstreams):
    """Device staging buffers of HOST_CHUNK rows per stream for one signature, kept across
    calls (allocating ~11 tensors per stream on every call delayed the first copy).  The
    caller holds _staging_lock for the whole pipelined call, so two host threads never share
    them; each call ends with every stream synchronised, so the next call may reuse them."""
    key = (dev.index, tuple(in_dtypes), tuple(out_dtypes), nstreams, HOST_CHUNK)
    if key not in _staging:
        _staging[key] = [([None if d is None else torch.empty(HOST_CHUNK, dtype=d, device=dev) for d in in_dtypes],
                          [torch.empty(HOST_CHUNK, dtype=d, device=dev) for d in out_dtypes])
                         for _ in range(nstreams)]
    return _staging[key]


def release_host_buffers():
    """Free the device staging buffers that host-input calls keep between calls (about
    74 B x HOST_CHUNK x (HOST_STREAMS - 1) for the fused call, ~0.9 GB at the defaults)."""
    with _staging_lock:
        _staging.clear()


def _copy_streams(device):
    key = device.index
    if key not in _streams:
        _streams[key] = tuple(torch.cuda.Stream(device) for _ in range(max(2, HOST_STREAMS)))  # >= 1 compute + copy-out
    return _streams[key]


def _is_host(inputs):
    return all((not isinstance(t, torch.Tensor)) or not t.is_cuda for t in inputs if t is not None)


def _host_tensor(t, dtype):
    if t is None:
        return None
    t = torch.as_tensor(t)
    if t.dtype != dtype:
        t = t.to(dtype)
    return t.contiguous()


def _pinned_outputs(n, dtypes):
    """Host outputs of n rows each as views of one pinned allocation (one request to the
    pinned-memory cache rather than one per output), each view 64-byte aligned."""
    offs, total = [], 0
    for d in dtypes:
        offs.append(total)
        total += -(-n * torch.empty((), dtype=d).element_size() // 64) * 64
    buf = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    return [buf[o:o + n * torch.empty((), dtype=d).element_size()].view(d) for o, d in zip(offs, dtypes)]


def _check_out(out, n, dtypes):
    """Caller-provided host outputs: contiguous CPU tensors of n rows and the outputs' dtypes."""
    if len(out) != len(dtypes):
        raise ValueError(f"out must hold {len(dtypes)} tensors")
    for t, d in zip(out, dtypes):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != d or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"out tensors must be contiguous host tensors of {n} rows, dtypes {dtypes}")
    return list(out)


def _rows_call(name, inputs, in_dtypes, out_dtypes, build_args, out=None):
    """Run one row-wise entry point.  `build_args(m, ins, outs)` returns its
    arguments for m rows of device tensors, stream excluded.  Device inputs
    run in place on the current stream; host inputs of more than HOST_CHUNK / 4
    rows are pipelined chunk by chunk (host -> device and kernel on rotating
    streams, device -> host on a stream of its own) into pinned host outputs,
    the caller's (`out`, host inputs only) or new ones."""
    n = next(t for t in inputs if t is not None)
    n = n.numel() if isinstance(n, torch.Tensor) else len(n)
    if out is not None and not _is_host(inputs):
        raise ValueError("out is for host inputs only")
    C = _host_chunk(n) if _is_host(inputs) else 0
    if out is not None and C == 0:
        res = _rows_call(name, inputs, in_dtypes, out_dtypes, build_args)
        for o, r in zip(_check_out(out, n, out_dtypes), res):
            o.copy_(r)
        return list(out)
    if C == 0:
        dev = _device_of(*inputs)
        ins = [_on(t, dev, d) for t, d in zip(inputs, in_dtypes)]
        _check_lengths(n, *ins)
        outs = [torch.empty(n, dtype=d, device=dev) for d in out_dtypes]
        _native.call(name, *build_args(n, ins, outs), _stream(dev))
        return _host_result(inputs, outs)
    dev = _device_of()
    hins = [_host_tensor(t, d) for t, d in zip(inputs, in_dtypes)]
    _check_lengths(n, *hins)
    houts = _check_out(out, n, out_dtypes) if out is not None else _pinned_outputs(n, out_dtypes)
    streams = _copy_streams(dev)
    with _staging_lock:
        bufs = _staging_buffers(dev, [None if h is None else h.dtype for h in hins], out_dtypes, len(streams) - 1)
        main = torch.cuda.current_stream(dev)
        out_stream = streams[-1]          # every device -> host copy, in chunk order
        compute = streams[:-1]            # host -> device copy and kernel of each chunk, in turn
        for st in streams:
            st.wait_stream(main)
        copied = [None] * len(compute)    # per staging set: its last copy-out
        for k, (lo, m) in enumerate(_chunks(n, C)):
            j = k % len(compute)
            st = compute[j]
            dins, douts = bufs[j]
            with torch.cuda.stream(st):
                ins = [None if h is None else d[:m] for d, h in zip(dins, hins)]
                for d, h in zip(ins, hins):
                    if h is not None:
                        d.copy_(h[lo:lo + m], non_blocking=True)
                if copied[j] is not None:
                    st.wait_event(copied[j])  # the set's outputs are free once copied out
                outs = [d[:m] for d in douts]
                _native.call(name, *build_args(m, ins, outs), ctypes.c_void_p(st.cuda_stream))
                done = torch.cuda.Event()
                done.record(st)
            with torch.cuda.stream(out_stream):
                out_stream.wait_event(done)
                for h, d in zip(houts, outs):
                    h[lo:lo + m].copy_(d, non_blocking=True)
                copied[j] = torch.cuda.Event()
                copied[j].record(out_stream)
        for st in streams:
            st.synchronize()
    return houts


def _check_lengths(n, *ts):
    for t in ts:
        if t is not None and t.numel() != n:
            raise ValueError("all arrays must have the same length")


def black_price(F, K, T, sigma, flag, *, vega: bool = True):
    """Undiscounted Black-76 price (r = 0) and vega; returns (P, vega or None)."""
    dev = _device_of(F, K, T, sigma, flag)
    f, k, t, s = (_on(a, dev, torch.float64) for a in (F, K, T, sigma))
    fl = _on(flag, dev, torch.int8)
    n = f.numel()
    _check_lengths(n, k, t, s, fl)
    P = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty(n, dtype=torch.float64, device=dev) if vega else None
    _native.call("pivot_black_price", n, _p(f), _p(k), _p(t), _p(s), _p(fl), _p(P), _p(V), _stream(dev))
    return tuple(_host_result((F, K, T, sigma, flag), [P, V]))


def black_price_backward(F, K, T, sigma, flag, gbar=None):
    """VJP of the Black-76 price (r = 0) in (sigma, F, K, T); returns (dsigma, dF, dK, dT)."""
    dev = _device_of(F, K, T, sigma, flag, gbar)
    f, k, t, s = (_on(a, dev, torch.float64) for a in (F, K, T, sigma))
    fl = _on(flag, dev, torch.int8)
    g = _on(gbar, dev, torch.float64)
    n = f.numel()
    _check_lengths(n, k, t, s, fl, g)
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
    _native.call("pivot_black_price_backward", n, _p(f), _p(k), _p(t), _p(s), _p(fl), _p(g),
                 *[_p(o) for o in outs], _stream(dev))
    return tuple(_host_result((F, K, T, sigma, flag, gbar), outs))


def mills_ratio(z):
    """Y(z) = Phi(z)/phi(z) evaluated by the library's FP64 kernel."""
    dev = _device_of(z)
    zz = _on(z, dev, torch.float64)
    y = torch.empty_like(zz)
    _native.call("pivot_mills_ratio", zz.numel(), _p(zz), _p(y), _stream(dev))
    return _host_result((z,), [y])[0]


def elementary(fn: str, x):
    """The library's FP64 log (fn="log"), exp (fn="exp"), the guesses' -Phi^{-1} (fn="neg_ncdfinv",
    x in (0, 1/2]), the solver's fast reciprocal (fn="rcp") or the guesses' cube root (fn="cbrt"),
    evaluated by its kernel."""
    dev = _device_of(x)
    xx = _on(x, dev, torch.float64)
    y = torch.empty_like(xx)
    _native.call("pivot_elementary", {"log": 0, "exp": 1, "neg_ncdfinv": 2, "rcp": 3, "cbrt": 4}[fn], xx.numel(), _p(xx), _p(y), _stream(dev))
    return _host_result((x,), [y])[0]


def _opts(mode, householder, mlp=None, fallback: float = 0.0, counters=None):
    o = _native.PivotOpts()
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.householder = int(householder)
    o.mlp = None if mlp is None else mlp.weights_ptr()
    o.fallback = float(fallback)
    if counters is not None:
        if not (counters.is_cuda and counters.dtype in (torch.int64, torch.uint64) and counters.is_contiguous()
                and counters.numel() >= _native.COUNTERS_LEN):
            raise ValueError(f"counters must be a contiguous CUDA int64 tensor of {_native.COUNTERS_LEN} entries")
        o.counters = counters.data_ptr()
    return o


def new_counters(device=None):
    """A zeroed device tensor for the per-launch counters of ``iv`` / ``iv_forward_backward``
    (layout in include/pivot.h: rows by status, solved rows by bin, rejected accelerated rows)."""
    dev = device or _device_of()
    return torch.zeros(_native.COUNTERS_LEN, dtype=torch.int64, device=dev)


class MlpTrainer:
    """Device state of the learned initial guess (pivot_mlp_trainer in include/pivot.h).

    ``init``, ``grad`` and ``adam`` run the library's own kernels; ``weights_ptr``
    is what PIVOT_MODE_LEARNED reads.
    """

    def __init__(self, device=None, seed: int = 0):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        off = ctypes.c_int64(0)
        nbytes = _native.lib().pivot_mlp_trainer_bytes(ctypes.byref(off))
        self.net_offset = int(off.value)
        self.buf = torch.zeros(int(nbytes), dtype=torch.uint8, device=self.device)
        self.init(seed)

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())

    def weights_ptr(self):
        return self.buf.data_ptr() + self.net_offset

    def init(self, seed: int = 0):
        _native.call("pivot_mlp_init", self.ptr(), ctypes.c_uint64(seed), _stream(self.device))

    def grad(self, F, K, T, P, flag, sigma):
        """Accumulate the gradient of sum (MLP - ln(s/s_a))^2 over the rows (the operator's own pairs)."""
        f, k, t, p, s = (_on(a, self.device, torch.float64) for a in (F, K, T, P, sigma))
        fl = _on(flag, self.device, torch.int8)
        _native.call("pivot_mlp_grad", self.ptr(), f.numel(), _p(f), _p(k), _p(t), _p(p), _p(fl), _p(s),
                     _stream(self.device))

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _native.call("pivot_mlp_adam", self.ptr(), float(lr), float(beta1), float(beta2), float(eps),
                     _stream(self.device))

    def fields(self):
        """(param, grad, loss_sum, rows, step) read back from the device (a synchronising copy)."""
        n = 8577
        f32 = self.buf[: 4 * 4 * n].view(torch.float32)
        tail = self.buf[4 * 4 * n: 4 * 4 * n + 24]
        d = tail[:16].view(torch.float64).cpu()
        step = int(tail[16:24].view(torch.int64).cpu()[0])
        return f32[:n].clone(), f32[n:2 * n].clone(), float(d[0]), float(d[1]), step


def iv_guess(F, K, T, P, flag, *, mode="fp64", mlp=None):
    """The initial guess s^(0) alone: LBR's rational seed (fp64) or the MLP seed (learned)."""
    dev = _device_of(F, K, T, P, flag)
    f, k, t, p = (_on(a, dev, torch.float64) for a in (F, K, T, P))
    fl = _on(flag, dev, torch.int8)
    n = f.numel()
    out = torch.empty(n, dtype=torch.float64, device=dev)
    o = _opts(mode, 0, mlp)
    _native.call("pivot_iv_guess", n, _p(f), _p(k), _p(t), _p(p), _p(fl), ctypes.byref(o), _p(out), _stream(dev))
    return _host_result((F, K, T, P, flag), [out])[0]


def iv(F, K, T, P, flag, *, mode="fp64", householder: int = 0, status: bool = True, mlp=None,
       fallback: float = 0.0, counters=None):
    """Implied volatility (Algorithm 1 forward); returns (sigma, status or None).  ``counters``
    (from ``new_counters``) accumulates the launch's row counts."""
    o = _opts(mode, householder, mlp, fallback, counters)
    f64 = torch.float64
    outs = _rows_call("pivot_iv_forward", (F, K, T, P, flag), (f64, f64, f64, f64, torch.int8),
                      (f64, torch.uint8) if status else (f64,),
                      lambda m, i, u: (m, *[_p(t) for t in i], _p(u[0]), _p(u[1]) if status else None,
                                       ctypes.byref(o)))
    return (outs[0], outs[1] if status else None)


def iv_backward(F, K, T, flag, sigma, gbar=None, *, tau: float = 1e-6, gate="nan"):
    """Gated IFT vector-Jacobian product (Eq. method_vjp, Section 3.3); returns (dP, dF, dK, dT)."""
    dev = _device_of(F, K, T, flag, sigma, gbar)
    f, k, t, s = (_on(a, dev, torch.float64) for a in (F, K, T, sigma))
    fl = _on(flag, dev, torch.int8)
    g = _on(gbar, dev, torch.float64)
    n = f.numel()
    _check_lengths(n, k, t, s, fl, g)
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
    _native.call("pivot_iv_backward", n, _p(f), _p(k), _p(t), _p(fl), _p(s), _p(g), float(tau), _gate(gate),
                 *[_p(o) for o in outs], _stream(dev))
    return tuple(_host_result((F, K, T, flag, sigma, gbar), outs))


def iv_forward_backward(F, K, T, P, flag, gbar=None, *, tau: float = 1e-6, gate="nan", mode="fp64",
                        householder: int = 0, mlp=None, fallback: float = 0.0, counters=None, out=None):
    """Forward and gated adjoint in one pass; returns (sigma, status, dP, dF, dK, dT).  With host
    inputs, ``out`` may give the six host outputs (pinned memory for overlapped copies)."""
    o = _opts(mode, householder, mlp, fallback, counters)
    f64 = torch.float64
    gm = _gate(gate)
    outs = _rows_call("pivot_iv_forward_backward", (F, K, T, P, flag, gbar),
                      (f64, f64, f64, f64, torch.int8, f64), (f64, torch.uint8, f64, f64, f64, f64),
                      lambda m, i, u: (m, *[_p(t) for t in i], float(tau), gm, *[_p(t) for t in u],
                                       ctypes.byref(o)), out=out)
    return tuple(outs)


class ImpliedVol(torch.autograd.Function):
    """sigma = JaeckelIV(P; F, K, T, flag) as an autograd node (Algorithm 1, Section 3.2).

    Forward runs the CUDA LBR solver with gradients suppressed and saves only
    (F, K, T, flag, sigma); backward returns the gated IFT VJP for P, F, K, T.
    """

    @staticmethod
    def forward(ctx, P, F, K, T, flag, tau=1e-6, gate="nan"):
        sig, _ = iv(F.detach(), K.detach(), T.detach(), P.detach(), flag, status=False)
        ctx.save_for_backward(F.detach(), K.detach(), T.detach(), flag, sig)
        ctx.tau, ctx.gate = float(tau), gate
        return sig

    @staticmethod
    def backward(ctx, gsig):
        F, K, T, flag, sig = ctx.saved_tensors
        dP, dF, dK, dT = iv_backward(F, K, T, flag, sig, gsig.contiguous(), tau=ctx.tau, gate=ctx.gate)
        need = ctx.needs_input_grad
        return (dP if need[0] else None, dF if need[1] else None, dK if need[2] else None,
                dT if need[3] else None, None, None, None)


def implied_volatility_autograd(P, F, K, T, flag, tau: float = 1e-6, gate="nan"):
    """Differentiable implied volatility (the paper's operator), see ``ImpliedVol``."""
    return ImpliedVol.apply(P, F, K, T, flag, tau, gate)


class BlackPrice(torch.autograd.Function):
    """P = Black-76 price (r = 0) of (sigma; F, K, T, flag) as an autograd node.

    The smooth price node of Section 3.2: its backward inserts the vega that
    cancels the 1/vega of ``ImpliedVol`` in a composed loss (the two-vega
    identity of the SPX appendix).
    """

    @staticmethod
    def forward(ctx, sigma, F, K, T, flag):
        P, _ = black_price(F.detach(), K.detach(), T.detach(), sigma.detach(), flag, vega=False)
        ctx.save_for_backward(F.detach(), K.detach(), T.detach(), sigma.detach(), flag)
        return P

    @staticmethod
    def backward(ctx, gP):
        F, K, T, sigma, flag = ctx.saved_tensors
        ds, dF, dK, dT = black_price_backward(F, K, T, sigma, flag, gP.contiguous())
        need = ctx.needs_input_grad
        return (ds if need[0] else None, dF if need[1] else None, dK if need[2] else None,
                dT if need[3] else None, None)


def black_price_autograd(sigma, F, K, T, flag):
    """Differentiable Black-76 price, see ``BlackPrice``."""
    return BlackPrice.apply(sigma, F, K, T, flag)


# ---------------------------------------------------------------------------------------------
# Black-Scholes interface on xi = (S, K, tau, r, q) with the discounted price V (Section 2,
# Eq. app_black_scholes; Algorithm 1).  T is the paper's tau (years); the gate threshold keeps
# the name ``tau`` as in the Black-76 calls.
# ---------------------------------------------------------------------------------------------
def bs_price(S, K, T, r, q, sigma, flag, *, vega: bool = True):
    """Discounted Black-Scholes price and cash vega dV/dsigma; returns (V, vega or None)."""
    dev = _device_of(S, K, T, r, q, sigma, flag)
    s_, k, t, rr, qq, sg = (_on(a, dev, torch.float64) for a in (S, K, T, r, q, sigma))
    fl = _on(flag, dev, torch.int8)
    n = s_.numel()
    _check_lengths(n, k, t, rr, qq, sg, fl)
    V = torch.empty(n, dtype=torch.float64, device=dev)
    vg = torch.empty(n, dtype=torch.float64, device=dev) if vega else None
    _native.call("pivot_bs_price", n, _p(s_), _p(k), _p(t), _p(rr), _p(qq), _p(sg), _p(fl), _p(V), _p(vg),
                 _stream(dev))
    return tuple(_host_result((S, K, T, r, q, sigma, flag), [V, vg]))


def bs_iv(S, K, T, r, q, V, flag, *, mode="fp64", householder: int = 0, status: bool = True, counters=None):
    """Implied volatility from the discounted price; returns (sigma, status or None)."""
    o = _opts(mode, householder, counters=counters)
    f64 = torch.float64
    outs = _rows_call("pivot_bs_iv_forward", (S, K, T, r, q, V, flag), (f64,) * 6 + (torch.int8,),
                      (f64, torch.uint8) if status else (f64,),
                      lambda m, i, u: (m, *[_p(t) for t in i], _p(u[0]), _p(u[1]) if status else None,
                                       ctypes.byref(o)))
    return (outs[0], outs[1] if status else None)


def bs_iv_backward(S, K, T, r, q, flag, sigma, gbar=None, *, tau: float = 1e-6, gate="nan"):
    """Gated VJP in xi; returns (dV, dS, dK, dT, dr, dq)."""
    dev = _device_of(S, K, T, r, q, flag, sigma, gbar)
    s_, k, t, rr, qq, sg = (_on(a, dev, torch.float64) for a in (S, K, T, r, q, sigma))
    fl = _on(flag, dev, torch.int8)
    g = _on(gbar, dev, torch.float64)
    n = s_.numel()
    _check_lengths(n, k, t, rr, qq, sg, fl, g)
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(6)]
    _native.call("pivot_bs_iv_backward", n, _p(s_), _p(k), _p(t), _p(rr), _p(qq), _p(fl), _p(sg), _p(g),
                 float(tau), _gate(gate), *[_p(o) for o in outs], _stream(dev))
    return tuple(_host_result((S, K, T, r, q, flag, sigma, gbar), outs))


def bs_iv_forward_backward(S, K, T, r, q, V, flag, gbar=None, *, tau: float = 1e-6, gate="nan", mode="fp64",
                           householder: int = 0, counters=None):
    """Forward and gated adjoint in xi in one pass; returns (sigma, status, dV, dS, dK, dT, dr, dq)."""
    o = _opts(mode, householder, counters=counters)
    f64 = torch.float64
    gm = _gate(gate)
    outs = _rows_call("pivot_bs_iv_forward_backward", (S, K, T, r, q, V, flag, gbar),
                      (f64,) * 6 + (torch.int8, f64), (f64, torch.uint8) + (f64,) * 6,
                      lambda m, i, u: (m, *[_p(t) for t in i], float(tau), gm, *[_p(t) for t in u],
                                       ctypes.byref(o)))
    return tuple(outs)


class ImpliedVolBS(torch.autograd.Function):
    """sigma = JaeckelIV(V; S, K, tau, r, q, flag) as an autograd node (Algorithm 1 on xi).

    Saves (S, K, tau, r, q, flag, sigma) only; backward is the gated IFT VJP for V, S, K,
    tau, r and q."""

    @staticmethod
    def forward(ctx, V, S, K, T, r, q, flag, tau=1e-6, gate="nan"):
        sig, _ = bs_iv(S.detach(), K.detach(), T.detach(), r.detach(), q.detach(), V.detach(), flag, status=False)
        ctx.save_for_backward(S.detach(), K.detach(), T.detach(), r.detach(), q.detach(), flag, sig)
        ctx.tau, ctx.gate = float(tau), gate
        return sig

    @staticmethod
    def backward(ctx, gsig):
        S, K, T, r, q, flag, sig = ctx.saved_tensors
        grads = bs_iv_backward(S, K, T, r, q, flag, sig, gsig.contiguous(), tau=ctx.tau, gate=ctx.gate)
        need = ctx.needs_input_grad
        return tuple(g if need[j] else None for j, g in enumerate(grads)) + (None, None, None)


def bs_implied_volatility_autograd(V, S, K, T, r, q, flag, tau: float = 1e-6, gate="nan"):
    """Differentiable implied volatility on xi = (S, K, tau, r, q), see ``ImpliedVolBS``."""
    return ImpliedVolBS.apply(V, S, K, T, r, q, flag, tau, gate)


# ---------------------------------------------------------------------------------------------
# Throughput probes (include/pivot.h, pivot_probe_*): measured unit rates for the rooflines.
# ---------------------------------------------------------------------------------------------
PROBE_UNITS = {"fp64_fma": 0, "fp32_fma": 1, "mufu_ex2": 2, "mufu_tanh": 3}


def probe_units(unit: str, iters: int, blocks_per_sm: int = 8, device=None):
    """Launch one unit probe on the current stream; returns the lane operations it performs."""
    dev = device or _device_of()
    sink = torch.zeros(1 << 16, dtype=torch.float64, device=dev)
    ops = ctypes.c_double(0.0)
    _native.call("pivot_probe_units", PROBE_UNITS[unit], int(blocks_per_sm), int(iters), _p(sink),
                 ctypes.byref(ops), _stream(dev))
    return float(ops.value)


def probe_stream(width: int, F, K, T, P, flag, outs, blocks_per_sm: int = 8):
    """The 74-byte-per-row stream of the fused forward+backward (no arithmetic); `outs` =
    (sigma, status, dP, dF, dK, dT) device tensors."""
    dev = F.device
    sig, st, dP, dF, dK, dT = outs
    _native.call("pivot_probe_stream", int(width), F.numel(), _p(F), _p(K), _p(T), _p(P), _p(flag), _p(sig),
                 _p(st), _p(dP), _p(dF), _p(dK), _p(dT), int(blocks_per_sm), _stream(dev))
