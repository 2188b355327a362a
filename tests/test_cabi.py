"""The C-ABI library builds, loads and exports every entry point include/vef.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vef.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vef_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_04758_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("vef_mesh_create", "vef_sweep", "vef_moments", "vef_adjoint_sweep",
                 "vef_source_iterate"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    import ctypes
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2301_04758_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_status_strings_and_no_device_failure(libpath):
    from paper_2301_04758_gb300 import _lib
    lib = _lib.load()
    assert lib.vef_status_string(_lib.VEF_ERR_TIMEOUT) == b"VEF_ERR_TIMEOUT"
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    h = ctypes.c_void_p()
    st = lib.vef_mesh_create(4, 4, 1, 1, 0.0, None, ctypes.byref(h))
    assert st == _lib.VEF_ERR_CUDA          # fails loudly, no CPU fallback
    assert not h.value
