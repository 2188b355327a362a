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


def test_mesh_create_checks_its_ranges_before_the_device(libpath):
    """Out-of-range sizes are refused by the host before any CUDA call, so the status is
    VEF_ERR_INVALID_ARG with or without a GPU: at most 2^22 elements (the packed task code
    holds 22 bits of element index), orders 1..4, a finite distortion, an output pointer."""
    import ctypes
    import math
    from paper_2301_04758_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    for args in [(2049, 2048, 3, 2, 0.05), (1 << 22, 2, 1, 1, 0.0), (0, 8, 1, 1, 0.0), (8, -1, 1, 1, 0.0),
                 (8, 8, 0, 2, 0.0), (8, 8, 5, 2, 0.0), (8, 8, 3, 0, 0.0), (8, 8, 3, 5, 0.0),
                 (8, 8, 3, 2, math.nan), (8, 8, 3, 2, math.inf)]:
        assert lib.vef_mesh_create(*args, None, ctypes.byref(h)) == _lib.VEF_ERR_INVALID_ARG, args
        assert not h.value
        assert lib.vef_last_error() != b""
    assert lib.vef_mesh_create(8, 8, 3, 2, 0.05, None, None) == _lib.VEF_ERR_INVALID_ARG


def test_wait_selftest_checks_arguments_before_the_device(libpath):
    from paper_2301_04758_gb300 import _lib
    lib = _lib.load()
    for kind, polls in [(2, 10), (-1, 10), (0, 0), (1, (1 << 24) + 1)]:
        assert lib.vef_wait_selftest(kind, 0, polls, None) == _lib.VEF_ERR_INVALID_ARG, (kind, polls)
    import torch
    if not torch.cuda.is_available():
        assert lib.vef_wait_selftest(0, 0, 16, None) == _lib.VEF_ERR_CUDA


def test_python_api_fails_loudly_without_library_or_gpu(libpath, tmp_path):
    """No CPU fallback anywhere on the product path: a missing library is an error that
    says how to build it, and without a GPU the wrappers raise the library's status."""
    from paper_2301_04758_gb300 import _lib
    with pytest.raises(RuntimeError, match="build"):
        _lib.load(str(tmp_path / "libvef.so"))
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2301_04758_gb300.api import Mesh
    with pytest.raises(_lib.VefError) as e:
        Mesh(4, 4, 1, 1, 0.0)
    assert e.value.status == _lib.VEF_ERR_CUDA


def test_header_is_plain_c(tmp_path):
    """include/vef.h is a C interface: it compiles as strict C99 (no CUDA or C++ types in
    the signatures) and as C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    src = tmp_path / "use_vef.c"
    src.write_text('#include <string.h>\n#include "vef.h"\n'
                   'int main(void) { vef_opts o; memset(&o, 0, sizeof o); return (int)VEF_OK + o.flags; }\n')
    for lang in (["-x", "c", "-std=c99", "-pedantic"], ["-x", "c++", "-std=c++17"]):
        r = subprocess.run([gcc, *lang, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_option_marshalling():
    """The Python keywords map onto vef_opts as include/vef.h defines it."""
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import _opts
    o = _opts()
    assert (o.precision, o.tol, o.max_passes, o.tile_override, o.flags) == (_lib.VEF_FP64, 0.0, 0, 0, 0)
    o = _opts("mixed", 1e-12, 5, 408, "iterative", "cluster", "separate")
    assert (o.precision, o.tol, o.max_passes, o.tile_override) == (_lib.VEF_MIXED, 1e-12, 5, 408)
    assert o.flags == _lib.VEF_GROUPS_ITERATIVE | _lib.VEF_SWEEP_CLUSTER | _lib.VEF_APPLY_SEPARATE == 7
    for bad in (dict(precision="fp16"), dict(groups="lagged"), dict(kernel="warp"), dict(apply="later")):
        with pytest.raises(KeyError):
            _opts(**bad)
    hdr = open(os.path.join(ROOT, "include", "vef.h")).read()
    for name in ("VEF_GROUPS_ITERATIVE", "VEF_SWEEP_CLUSTER", "VEF_APPLY_SEPARATE", "VEF_FP64", "VEF_MIXED"):
        m = re.search(name + r"\s*=\s*(\d+)", hdr)
        assert m and int(m.group(1)) == getattr(_lib, name), name


def test_status_codes_agree_with_the_library(libpath):
    from paper_2301_04758_gb300 import _lib
    lib = _lib.load()
    names = ["VEF_OK", "VEF_ERR_INVALID_ARG", "VEF_ERR_CUDA", "VEF_ERR_OOM", "VEF_ERR_TIMEOUT",
             "VEF_ERR_NOT_CONVERGED", "VEF_ERR_NONPOSITIVE_DENOM", "VEF_ERR_NOT_IMPLEMENTED", "VEF_ERR_BOUNDS"]
    for name in names:
        assert lib.vef_status_string(getattr(_lib, name)).decode() == name
    hdr = open(os.path.join(ROOT, "include", "vef.h")).read()
    for name in names[1:] + ["VEF_STATUS_TIMEOUT", "VEF_STATUS_NOT_CONVERGED", "VEF_STATUS_NONPOSITIVE",
                             "VEF_STATUS_SINGULAR", "VEF_STATUS_BOUNDS"]:
        m = re.search(name + r"\s*=\s*(\d+)", hdr)
        assert m and int(m.group(1)) == getattr(_lib, name), name
    assert lib.vef_build_checked() == 0   # the normal build
