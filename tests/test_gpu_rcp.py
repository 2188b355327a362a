"""The elimination pivots' reciprocal (csrc/device.cuh pivot_rcp: an approximate reciprocal
refined by two Newton-Raphson steps) against the correctly rounded 1/x on the GPU, over
inputs spread across the normal range: within two units in the last place."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_pivot_reciprocal_is_within_two_ulp(lib):
    from paper_2301_04758_gb300 import _lib
    l = _lib.load()
    e64, e32 = ctypes.c_double(), ctypes.c_double()
    assert l.vef_rcp_selftest(1 << 22, ctypes.byref(e64), ctypes.byref(e32)) == _lib.VEF_OK
    print(f"pivot_rcp: max relative difference {e64.value:.3e} (FP64), {e32.value:.3e} (FP32)")
    assert e64.value <= 4 * 2.0 ** -53   # two ulp at the top of a binade
    assert e32.value == 0.0   # FP32 uses the correctly rounded reciprocal itself
    assert l.vef_rcp_selftest(0, ctypes.byref(e64), ctypes.byref(e32)) == _lib.VEF_ERR_INVALID_ARG
