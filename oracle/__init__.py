"""Plain FP64 CPU oracle for the PIVOT hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  It wraps ``pivot_oracle.c`` (plain C, compiled with
gcc here or on the GPU host) through ctypes and shares nothing with the CUDA
path.  See ``pivot_oracle.c`` for what each function computes and the paper
passages it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pivot_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_BELOW_INTRINSIC, STATUS_ABOVE_UPPER, STATUS_BAD_INPUT = 0, 1, 2, 3
STATUS_AT_INTRINSIC, STATUS_AT_UPPER = 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    vp = ctypes.c_void_p
    for name in ("oracle_normalised_black", "oracle_normalised_black_complement",
                 "oracle_log_normalised_black"):
        getattr(lib, name).argtypes = [d, d]
        getattr(lib, name).restype = d
    lib.oracle_mills.argtypes = [d]
    lib.oracle_mills.restype = d
    lib.oracle_black_price.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.oracle_iv.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.oracle_iv_grad.argtypes = [i64, vp, vp, vp, vp, vp, vp, d, i32, vp, vp, vp, vp, i32]
    lib.oracle_black_price_grad.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.oracle_bs_price.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.oracle_bs_iv.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.oracle_bs_iv_grad.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, d, i32, vp, vp, vp, vp, vp, vp, i32]
    for name in ("oracle_black_price", "oracle_iv", "oracle_iv_grad", "oracle_black_price_grad",
                 "oracle_bs_price", "oracle_bs_iv", "oracle_bs_iv_grad", "oracle_max_threads"):
        getattr(lib, name).restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def compile_variant(src_text: str, out_path: str):
    """Compile a modified copy of the oracle source (used by tests that plant a
    mistake in the oracle and check that a pin catches it) and return an
    ``Oracle`` bound to it."""
    cpath = out_path + ".c"
    with open(cpath, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-I", _HERE, "-o", out_path,
                    cpath, "-lm"], check=True)
    return Oracle(_bind(ctypes.CDLL(out_path)))


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """The oracle functions bound to one compiled library."""

    def __init__(self, lib):
        self.lib = lib

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def normalised_black(self, x: float, s: float) -> float:
        """b(x, s) for x <= 0 (Eq. app_normalized_black, out-of-the-money form)."""
        return self.lib.oracle_normalised_black(float(x), float(s))

    def normalised_black_complement(self, x: float, s: float) -> float:
        """b_max(x) - b(x, s) = e^{x/2} - b(x, s) for x <= 0 (Eq. app_b_bounds)."""
        return self.lib.oracle_normalised_black_complement(float(x), float(s))

    def log_normalised_black(self, x: float, s: float) -> float:
        return self.lib.oracle_log_normalised_black(float(x), float(s))

    def mills(self, z: float) -> float:
        """Phi(z)/phi(z)."""
        return self.lib.oracle_mills(float(z))

    def black_price(self, F, K, T, sigma, flag, nthreads: int = 1):
        """Undiscounted Black-76 price (r = 0) and vega, Eq. app_black76 / app_vega_closed_form."""
        F, K, T, sigma = map(_f64, (F, K, T, sigma))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        n = F.shape[0]
        P = np.empty(n)
        V = np.empty(n)
        rc = self.lib.oracle_black_price(n, _ptr(F), _ptr(K), _ptr(T), _ptr(sigma), _ptr(flag), _ptr(P), _ptr(V),
                                        nthreads)
        if rc:
            raise ValueError(f"oracle_black_price returned {rc}")
        return P, V

    def implied_vol(self, F, K, T, P, flag, nthreads: int = 1):
        """sigma and status per row, Eq. iv_inverse_problem (see pivot_oracle.h for codes)."""
        F, K, T, P = map(_f64, (F, K, T, P))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        n = F.shape[0]
        sig = np.empty(n)
        st = np.empty(n, dtype=np.uint8)
        rc = self.lib.oracle_iv(n, _ptr(F), _ptr(K), _ptr(T), _ptr(P), _ptr(flag), _ptr(sig), _ptr(st), nthreads)
        if rc:
            raise ValueError(f"oracle_iv returned {rc}")
        return sig, st

    def black_price_grad(self, F, K, T, sigma, flag, gbar=None, nthreads: int = 1):
        """(dsigma, dF, dK, dT): VJP of the Black-76 price, Eq. app_black76 differentiated."""
        F, K, T, sigma = map(_f64, (F, K, T, sigma))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        g = None if gbar is None else _f64(gbar)
        n = F.shape[0]
        out = [np.empty(n) for _ in range(4)]
        rc = self.lib.oracle_black_price_grad(n, _ptr(F), _ptr(K), _ptr(T), _ptr(sigma), _ptr(flag), _ptr(g),
                                              *[_ptr(o) for o in out], nthreads)
        if rc:
            raise ValueError(f"oracle_black_price_grad returned {rc}")
        return tuple(out)

    def iv_grad(self, F, K, T, flag, sigma, gbar=None, tau: float = 0.0, gate_mode: int = 0, nthreads: int = 1):
        """(dP, dF, dK, dT): gated IFT vector-Jacobian product, Eq. method_vjp and Section 3.3."""
        F, K, T, sigma = map(_f64, (F, K, T, sigma))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        g = None if gbar is None else _f64(gbar)
        n = F.shape[0]
        out = [np.empty(n) for _ in range(4)]
        rc = self.lib.oracle_iv_grad(n, _ptr(F), _ptr(K), _ptr(T), _ptr(flag), _ptr(sigma), _ptr(g), float(tau),
                                    int(gate_mode), *[_ptr(o) for o in out], nthreads)
        if rc:
            raise ValueError(f"oracle_iv_grad returned {rc}")
        return tuple(out)

    # -- Black-Scholes interface on xi = (S, K, tau, r, q) -------------------------------------
    def bs_price(self, S, K, T, r, q, sigma, flag, nthreads: int = 1):
        """Discounted Black-Scholes price and cash vega, Eq. app_black_scholes."""
        S, K, T, r, q, sigma = map(_f64, (S, K, T, r, q, sigma))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        n = S.shape[0]
        V = np.empty(n)
        vega = np.empty(n)
        rc = self.lib.oracle_bs_price(n, _ptr(S), _ptr(K), _ptr(T), _ptr(r), _ptr(q), _ptr(sigma), _ptr(flag),
                                      _ptr(V), _ptr(vega), nthreads)
        if rc:
            raise ValueError(f"oracle_bs_price returned {rc}")
        return V, vega

    def bs_implied_vol(self, S, K, T, r, q, V, flag, nthreads: int = 1):
        """sigma and status per row from the discounted price (Algorithm 1 forward normalisation)."""
        S, K, T, r, q, V = map(_f64, (S, K, T, r, q, V))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        n = S.shape[0]
        sig = np.empty(n)
        st = np.empty(n, dtype=np.uint8)
        rc = self.lib.oracle_bs_iv(n, _ptr(S), _ptr(K), _ptr(T), _ptr(r), _ptr(q), _ptr(V), _ptr(flag), _ptr(sig),
                                   _ptr(st), nthreads)
        if rc:
            raise ValueError(f"oracle_bs_iv returned {rc}")
        return sig, st

    def bs_iv_grad(self, S, K, T, r, q, flag, sigma, gbar=None, tau: float = 0.0, gate_mode: int = 0,
                   nthreads: int = 1):
        """(dV, dS, dK, dT, dr, dq): Algorithm 1 backward on xi with the gate of Section 3.3."""
        S, K, T, r, q, sigma = map(_f64, (S, K, T, r, q, sigma))
        flag = np.ascontiguousarray(flag, dtype=np.int8)
        g = None if gbar is None else _f64(gbar)
        n = S.shape[0]
        out = [np.empty(n) for _ in range(6)]
        rc = self.lib.oracle_bs_iv_grad(n, _ptr(S), _ptr(K), _ptr(T), _ptr(r), _ptr(q), _ptr(flag), _ptr(sigma),
                                        _ptr(g), float(tau), int(gate_mode), *[_ptr(o) for o in out], nthreads)
        if rc:
            raise ValueError(f"oracle_bs_iv_grad returned {rc}")
        return tuple(out)


def bs_price(*a, **k):
    return default().bs_price(*a, **k)


def bs_implied_vol(*a, **k):
    return default().bs_implied_vol(*a, **k)


def bs_iv_grad(*a, **k):
    return default().bs_iv_grad(*a, **k)


def black_price_grad(*a, **k):
    return default().black_price_grad(*a, **k)


def default() -> Oracle:
    """The oracle built from ``pivot_oracle.c``."""
    return Oracle(_load())


def max_threads() -> int:
    return default().max_threads()


def normalised_black(x, s):
    return default().normalised_black(x, s)


def normalised_black_complement(x, s):
    return default().normalised_black_complement(x, s)


def log_normalised_black(x, s):
    return default().log_normalised_black(x, s)


def mills(z):
    return default().mills(z)


def black_price(*a, **k):
    return default().black_price(*a, **k)


def implied_vol(*a, **k):
    return default().implied_vol(*a, **k)


def iv_grad(*a, **k):
    return default().iv_grad(*a, **k)
