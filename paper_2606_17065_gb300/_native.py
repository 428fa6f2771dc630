"""ctypes binding of include/pivot.h (argument marshalling only).

The CUDA library must be built (``paper_2606_17065_gb300.build.build()``);
there is no CPU fallback: every call fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from .build import INCLUDE, LIB_PATH

_lock = threading.Lock()
_lib = None

c_i64, c_i32, c_dbl, c_vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p


class PivotOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("householder", ctypes.c_int32), ("mlp", ctypes.c_void_p),
                ("fallback", ctypes.c_double), ("counters", ctypes.c_void_p)]


COUNTERS_LEN = 24
ABI_VERSION = 200  # the pivot_opts layout above


_SIGNATURES = {
    "pivot_black_price": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_black_price_backward": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_iv_forward": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_iv_backward": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_dbl, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_iv_forward_backward": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_dbl, c_i32, c_vp, c_vp, c_vp, c_vp,
                                  c_vp, c_vp, c_vp, c_vp],
    "pivot_bs_price": [c_i64] + [c_vp] * 10,
    "pivot_bs_iv_forward": [c_i64] + [c_vp] * 11,
    "pivot_bs_iv_backward": [c_i64] + [c_vp] * 8 + [c_dbl, ctypes.c_int32] + [c_vp] * 7,
    "pivot_bs_iv_forward_backward": [c_i64] + [c_vp] * 8 + [c_dbl, ctypes.c_int32] + [c_vp] * 10,
    "pivot_mills_ratio": [c_i64, c_vp, c_vp, c_vp],
    "pivot_elementary": [c_i32, c_i64, c_vp, c_vp, c_vp],
    "pivot_mlp_trainer_bytes": [c_vp],
    "pivot_iv_guess": [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_mlp_init": [c_vp, ctypes.c_uint64, c_vp],
    "pivot_mlp_grad": [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_mlp_adam": [c_vp, c_dbl, c_dbl, c_dbl, c_dbl, c_vp],
    "pivot_mlp_grad_static": [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
    "pivot_probe_units": [c_i32, c_i32, c_i64, c_vp, c_vp, c_vp],
    "pivot_probe_stream": [c_i32, c_i64] + [c_vp] * 11 + [c_i32, c_vp],
    "pivot_error_string": [ctypes.c_int],
    "pivot_version": [],
}


class PivotError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} failed with code {code}: {error_string(code)}")


def declared_symbols() -> list[str]:
    """Every function declared in include/*.h."""
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            text = open(os.path.join(INCLUDE, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+(pivot_\w+)\s*\(", text, flags=re.M)
    return names


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"the CUDA extension {LIB_PATH} is not built; run "
                "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        handle.pivot_error_string.restype = ctypes.c_char_p
        handle.pivot_mlp_trainer_bytes.restype = ctypes.c_int64
        if handle.pivot_version() < ABI_VERSION:
            raise RuntimeError(f"{LIB_PATH} is ABI {handle.pivot_version()}, this binding needs {ABI_VERSION}: rebuild it")
        _lib = handle
        return _lib


def error_string(code: int) -> str:
    return lib().pivot_error_string(int(code)).decode()


def call(name: str, *args) -> None:
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise PivotError(name, rc)
