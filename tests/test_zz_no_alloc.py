"""vef_eddington_noalloc: the allocation-free Eddington-tensor entry point.

It serves callers that cannot allocate device memory (an application that owns the
whole GPU through its own pool, or a loop that must not trigger the synchronisation of
cudaMalloc / cudaFree).  Its scratch is one fixed device array shared by every call, so
this test calls it twice in a row, with different angular fluxes, and checks each
result against vef_moments (the allocating entry point) through the C ABI.  The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from _gpu import dev, host, rel
from vef_inputs import level_symmetric

pytestmark = pytest.mark.gpu


def _noalloc(lib, psi, om, w, E, p):
    import torch
    nq = p + 2
    out = torch.empty(3, E, nq * nq, dtype=torch.float64, device="cuda")
    omh = np.ascontiguousarray(om, dtype=np.float64)
    wh = np.ascontiguousarray(w, dtype=np.float64)
    st = lib.vef_eddington_noalloc(ctypes.c_void_p(psi.data_ptr()), omh.ctypes.data_as(ctypes.c_void_p),
                                   wh.ctypes.data_as(ctypes.c_void_p), len(wh), E, p,
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_noalloc_matches_vef_moments_on_two_calls(lib):
    import torch
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    p, nx, ny = 2, 7, 5
    om, w = level_symmetric(8)
    mesh = Mesh(nx, ny, 3, p, 0.05)
    rng = np.random.default_rng(17)
    for call in range(2):
        psi = dev(rng.uniform(0.2, 3.0 + call, (len(w), mesh.E, mesh.n)))
        ref = mesh.moments(psi, om, w, outputs=("E",))["E"]
        st, got = _noalloc(lib, psi, om, w, mesh.E, p)
        assert st == _lib.VEF_OK, lib.vef_last_error()
        torch.cuda.synchronize()
        assert rel(host(got), host(ref)) < 1e-13, call


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    from paper_2301_04758_gb300 import _lib
    om, w = level_symmetric(4)
    psi = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    omh = np.ascontiguousarray(om)
    wh = np.ascontiguousarray(w)
    st = lib.vef_eddington_noalloc(ctypes.c_void_p(psi.data_ptr()), omh.ctypes.data_as(ctypes.c_void_p),
                                   wh.ctypes.data_as(ctypes.c_void_p), len(wh), 300 * 300, 2,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert st == _lib.VEF_ERR_INVALID_ARG
    assert b"524288" in lib.vef_last_error()
