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


def test_noalloc_at_its_limits_allocates_nothing(lib):
    """The largest direction set (D = 256, passed by value) at p = 4 with the largest mesh
    the scratch holds (E (p+1)^2 = 524275 <= 524288 nodal values) matches vef_moments, one
    element more is rejected, and a call leaves the device's free memory unchanged."""
    import torch
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    p, nx, ny, D = 4, 67, 313, 256            # E = 20971 = floor(524288 / 25)
    E = nx * ny
    assert E * 25 <= 524288 < (E + 1) * 25
    rng = np.random.default_rng(256)
    z, ph = rng.uniform(0.05, 0.95, D), rng.uniform(0.0, 2 * np.pi, D)
    om = np.stack([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph)], axis=1)
    w = np.full(D, 4 * np.pi / D)
    mesh = Mesh(nx, ny, 1, p, 0.0)
    psi = torch.rand(D, E, 25, dtype=torch.float64, device="cuda") + 0.1
    ref = mesh.moments(psi, om, w, outputs=("E",))["E"]
    st, got = _noalloc(lib, psi, om, w, E, p)          # warm: the scratch address is looked up
    assert st == _lib.VEF_OK, lib.vef_last_error()
    torch.cuda.synchronize()
    assert rel(host(got), host(ref)) < 1e-13
    free0, _ = torch.cuda.mem_get_info()
    st, got = _noalloc(lib, psi, om, w, E, p)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == _lib.VEF_OK and free1 == free0
    assert rel(host(got), host(ref)) < 1e-13
    omh, wh = np.ascontiguousarray(om), np.ascontiguousarray(w)
    st = lib.vef_eddington_noalloc(ctypes.c_void_p(psi.data_ptr()), omh.ctypes.data_as(ctypes.c_void_p),
                                   wh.ctypes.data_as(ctypes.c_void_p), D, E + 1, p,
                                   ctypes.c_void_p(got.data_ptr()), None)
    assert st == _lib.VEF_ERR_INVALID_ARG
    w257 = np.full(D + 1, 4 * np.pi / (D + 1))
    om257 = np.ascontiguousarray(np.concatenate([om, om[:1]]))
    st = lib.vef_eddington_noalloc(ctypes.c_void_p(psi.data_ptr()), om257.ctypes.data_as(ctypes.c_void_p),
                                   w257.ctypes.data_as(ctypes.c_void_p), D + 1, 10, p,
                                   ctypes.c_void_p(got.data_ptr()), None)
    assert st == _lib.VEF_ERR_INVALID_ARG


def test_noalloc_writes_nan_where_phi_vanishes(lib):
    """psi zero on one element: the scalar flux vanishes there, so exactly that element's
    Eddington-tensor entries are NaN (the call still returns VEF_OK, as documented); every
    other entry matches vef_moments."""
    import torch
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    p, nx, ny = 3, 6, 4
    om, w = level_symmetric(6)
    mesh = Mesh(nx, ny, 3, p, 0.05)
    rng = np.random.default_rng(5)
    psi_h = rng.uniform(0.2, 2.0, (len(w), mesh.E, mesh.n))
    bad = 13
    psi_h[:, bad, :] = 0.0
    psi = dev(psi_h)
    st, got = _noalloc(lib, psi, om, w, mesh.E, p)
    assert st == _lib.VEF_OK
    torch.cuda.synchronize()
    g = host(got)
    assert np.isnan(g[:, bad, :]).all()
    keep = np.ones(mesh.E, bool)
    keep[bad] = False
    assert np.isfinite(g[:, keep, :]).all()
    ref = mesh.moments(psi, om, w, outputs=("E",))["E"]
    torch.cuda.synchronize()
    r = host(ref)
    assert rel(g[:, keep, :], r[:, keep, :]) < 1e-13
