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
    assert lib.pivot_version() >= 100
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
    """pivot_elementary takes fn 0 (log), 1 (exp), 2 (the guesses' -Phi^-1); any other code is
    PIVOT_E_OPTS, and an empty batch succeeds without touching the device."""
    lib = _native.lib()
    fake = ctypes.c_void_p(0x1000)
    for fn in (-1, 3, 99):
        assert lib.pivot_elementary(fn, 4, fake, fake, None) == 4
    for fn in (0, 1, 2):
        assert lib.pivot_elementary(fn, 0, None, None, None) == 0
        assert lib.pivot_elementary(fn, -1, fake, fake, None) == 1
