"""The bounds-checked build (libvef_checked.so, compiled with VEF_CHECKED) on the GPU.

compute-sanitizer is closed on this machine; the checked build stands in for it: every index
the sweep, adjoint, group and factorisation kernels take from the schedule (record and
member indices, element indices, shared-memory trace-slot ids) is tested before its access,
and one outside its array would set VEF_STATUS_BOUNDS and be skipped.  These tests run the
library's main paths through the checked build on small curved meshes with coupled element
groups, at every order, and require that no call reports VEF_ERR_BOUNDS and that the
results equal the normal build's (the checks change no arithmetic), which in turn match the
oracle in the other parity tests.
"""
import numpy as np
import pytest

from _gpu import dev, host, rel, random_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    from paper_2301_04758_gb300 import _lib, build
    normal = _lib.load()
    checked = _lib.load(build.build(checked=True))
    assert normal.vef_build_checked() == 0 and checked.vef_build_checked() == 1
    return normal, checked


def _run(p, seed):
    """Sweep (FP64 and mixed), closures, adjoint gradients and the HRT solve through the
    library _lib.load() currently returns."""
    from paper_2301_04758_gb300.api import Mesh
    prob = random_problem(9, 8, 3, 0.1, p, 6, seed=seed)
    mesh = Mesh(9, 8, 3, p, 0.1)
    st, ss = dev(prob["sigma_t"]), dev(prob["sigma_s"])
    kw = dict(phi_in=dev(prob["phi_in"]), source=dev(prob["source"]), inflow=dev(prob["inflow"]))
    out = {}
    psi, info = mesh.sweep(st, ss, prob["omega"], prob["weights"], info=True, **kw)
    out["psi"] = host(psi)
    out["groups"] = info["coupled_groups"]
    out["psi_mixed"] = host(mesh.sweep(st, ss, prob["omega"], prob["weights"], precision="mixed", **kw))
    mom = mesh.moments(psi, prob["omega"], prob["weights"], inflow=kw["inflow"],
                       outputs=("phi", "P", "Eb", "Jin"))
    out.update({k: host(v) for k, v in mom.items()})
    g = mesh.region_weights((0.3, 0.3), (0.7, 0.7))
    dst, dss, _ = mesh.adjoint(st, ss, prob["omega"], prob["weights"], psi, g, phi_in=kw["phi_in"])
    out["dst"], out["dss"] = host(dst), host(dss)
    q0 = dev(4.0 * np.pi * prob["source"])
    phi, J, _, hinfo = mesh.hrt_solve(st, ss, mom["phi"], mom["P"], mom["Eb"], mom["Jin"], q0, tol=1e-13)
    out["hrt_phi"], out["hrt_J"] = host(phi), host(J)
    mesh.sync()
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_checked_build_runs_clean_and_matches_the_normal_build(libs, monkeypatch, p):
    from paper_2301_04758_gb300 import _lib
    normal, checked = libs
    monkeypatch.setattr(_lib, "_lib", normal)
    ref = _run(p, 700 + p)
    monkeypatch.setattr(_lib, "_lib", checked)
    got = _run(p, 700 + p)   # any VEF_ERR_BOUNDS raises here
    assert ref["groups"] > 0, "the mesh should exercise the coupled-group paths"
    for k, v in ref.items():
        if k == "groups":
            assert got[k] == v
        else:
            assert rel(got[k], v) < 1e-13, (k, rel(got[k], v))


def test_bounds_status_maps_to_its_error():
    """The host side of the check: a recorded VEF_STATUS_BOUNDS (set here through the status
    hook, as a checked kernel would set it) makes the next synchronising call return
    VEF_ERR_BOUNDS and is then cleared."""
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    lib = _lib.load()
    mesh = Mesh(4, 4, 1, 1, 0.0)
    assert lib.vef_mesh_inject_status(mesh.handle, _lib.VEF_STATUS_BOUNDS, None) == _lib.VEF_OK
    with pytest.raises(_lib.VefError, match="VEF_ERR_BOUNDS") as err:
        mesh.sync()
    assert err.value.status == _lib.VEF_ERR_BOUNDS
    mesh.sync()   # cleared by the failing call
    assert lib.vef_mesh_inject_status(mesh.handle, 32, None) == _lib.VEF_ERR_INVALID_ARG
