"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/*.h declares, and rejects bad arguments before touching the device."""
import ctypes

from paper_2606_17065_gb300 import _native


def test_library_exports_every_declared_symbol():
    lib = _native.lib()
    names = _native.declared_symbols()
    assert {"pivot_black_price", "pivot_iv_forward", "pivot_iv_backward", "pivot_iv_forward_backward"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_error_strings():
    lib = _native.lib()
    assert lib.pivot_version() >= _native.ABI_VERSION
    for code in range(0, 7):
        assert _native.error_string(code)


def test_argument_errors_before_any_device_access():
    lib = _native.lib()
    fake = ctypes.c_void_p(0x1000)
    # n < 0 is rejected first
    assert lib.pivot_black_price(-1, fake, fake, fake, fake, fake, fake, None, None) == 1
    assert lib.pivot_iv_forward(-5, fake, fake, fake, fake, fake, fake, None, None, None) == 1
    # gate checks precede pointer checks
    assert lib.pivot_iv_backward(4, fake, fake, fake, fake, fake, None, -1.0, 1, None, None, None, None, None) == 3
    assert lib.pivot_iv_backward(4, fake, fake, fake, fake, fake, None, float("nan"), 1, None, None, None, None,
                                 None) == 3
    assert lib.pivot_iv_backward(4, fake, fake, fake, fake, fake, None, 0.0, 3, None, None, None, None, None) == 3
    assert lib.pivot_iv_backward(4, fake, fake, fake, fake, fake, None, 1e-6, 4, None, None, None, None, None) == 3
    # bad options
    o = _native.PivotOpts()
    o.mode, o.householder = 0, -1
    assert lib.pivot_iv_forward(4, fake, fake, fake, fake, fake, fake, None, ctypes.byref(o), None) == 4
    o.mode, o.householder = 7, 0
    assert lib.pivot_iv_forward(4, fake, fake, fake, fake, fake, fake, None, ctypes.byref(o), None) == 4
    # n == 0 launches nothing and succeeds, even with NULL pointers
    assert lib.pivot_iv_forward(0, None, None, None, None, None, None, None, None, None) == 0
    assert lib.pivot_iv_forward_backward(0, None, None, None, None, None, None, 0.0, 0, None, None, None, None,
                                         None, None, None, None) == 0


def test_elementary_function_codes():
    """pivot_elementary takes fn 0 (log), 1 (exp), 2 (the guesses' -Phi^-1), 3 (the fast
    reciprocal), 4 (the guesses' cube root); any other code is
    PIVOT_E_OPTS, and an empty batch succeeds without touching the device."""
    lib = _native.lib()
    fake = ctypes.c_void_p(0x1000)
    for fn in (-1, 5, 99):
        assert lib.pivot_elementary(fn, 4, fake, fake, None) == 4
    for fn in (0, 1, 2, 3, 4):
        assert lib.pivot_elementary(fn, 0, None, None, None) == 0
        assert lib.pivot_elementary(fn, -1, fake, fake, None) == 1


def test_probe_argument_errors():
    """pivot_probe_units / pivot_probe_stream reject bad units, widths, sizes and a NULL
    lane_ops before any device access; an empty stream succeeds."""
    lib = _native.lib()
    fake = ctypes.c_void_p(0x1000)
    ops = ctypes.c_double(0.0)
    for unit, bps, iters in ((-1, 8, 1), (4, 8, 1), (0, 0, 1), (0, 33, 1), (0, 8, 0)):
        assert lib.pivot_probe_units(unit, bps, iters, fake, ctypes.byref(ops), None) == 4
    assert lib.pivot_probe_units(0, 8, 1, fake, None, None) == 2
    args = [fake] * 11
    assert lib.pivot_probe_stream(1, -1, *args, 8, None) == 1
    assert lib.pivot_probe_stream(3, 4, *args, 8, None) == 4
    assert lib.pivot_probe_stream(1, 4, *args, 0, None) == 4
    assert lib.pivot_probe_stream(2, 0, *([None] * 11), 8, None) == 0


def test_opts_layout_and_counters_validation():
    """pivot_opts carries the counters pointer last; the binding refuses a counters tensor that
    is not a CUDA int64 array of PIVOT_COUNTERS_LEN entries."""
    import pytest
    import torch

    from paper_2606_17065_gb300 import api
    assert ctypes.sizeof(_native.PivotOpts) == 32
    assert _native.PivotOpts.counters.offset == 24
    with pytest.raises(ValueError):
        api._opts("fp64", 0, counters=torch.zeros(24, dtype=torch.int64))  # host memory
    text = open(_native.INCLUDE + "/pivot.h").read()
    assert f"#define PIVOT_COUNTERS_LEN {_native.COUNTERS_LEN}" in text
