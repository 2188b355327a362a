"""Failure detection on the GPU without a fault: a bounded wait that nothing completes
reports VEF_ERR_TIMEOUT through the status word, within its poll budget, and the CUDA
context stays usable (a sweep right after matches the oracle).  A timeout recorded on the
host side (the injection hook, standing in for a wait that ran out) makes the sweeps'
staging waits stop at once, so a call made while it is pending returns quickly."""
import time

import pytest

from _gpu import dev, host, rel, random_problem
from oracle.transport import Discretization, sweep as o_sweep

pytestmark = pytest.mark.gpu


# an mbarrier try-wait on an incomplete phase may suspend the thread for a system-dependent
# time per poll, so that form gets fewer polls (the printed time per poll measures it)
@pytest.mark.parametrize("kind,polls", [(0, 1 << 16), (1, 1 << 10)], ids=["global_flag", "mbarrier"])
def test_bounded_wait_times_out_and_the_context_survives(lib, kind, polls):
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    assert lib.vef_wait_selftest(kind, 1, polls, None) == _lib.VEF_OK
    t = time.perf_counter()
    st = lib.vef_wait_selftest(kind, 0, polls, None)
    elapsed = time.perf_counter() - t
    print(f"kind {kind}: {polls} polls ran out in {elapsed * 1e3:.2f} ms "
          f"({elapsed / polls * 1e9:.0f} ns per poll, launch included)")
    assert st == _lib.VEF_ERR_TIMEOUT
    assert b"timeout" in lib.vef_last_error()
    assert elapsed < 20.0
    prob = random_problem(4, 3, 3, 0.05, 2, 4, seed=77)
    mesh = Mesh(4, 3, 3, 2, 0.05)
    psi, info = mesh.sweep(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"], prob["weights"],
                           phi_in=dev(prob["phi_in"]), source=dev(prob["source"]),
                           inflow=dev(prob["inflow"]), info=True)
    disc = Discretization(4, 3, 3, 0.05, 2)
    ref = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"], inflow=prob["inflow"])
    assert info["timed_out"] == 0
    assert rel(host(psi), ref) < 1e-12


@pytest.mark.parametrize("kind", ["sweep", "adjoint", "cluster"])
def test_pending_timeout_stops_the_staging_waits(lib, kind):
    """With a timeout already in the status word the forward sweep (single-CTA and cluster
    forms) and the adjoint sweep return within a short bound and report VEF_ERR_TIMEOUT; the
    word is then clear and the same call reproduces the oracle."""
    import ctypes
    import torch
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    from oracle.adjoint import adjoint as o_adjoint, region_weights
    N, p = 40, 2
    prob = random_problem(N, N, 3, 0.08, p, 8, seed=91, with_inflow=False)
    mesh = Mesh(N, N, 3, p, 0.08)
    st, ss = dev(prob["sigma_t"]), dev(prob["sigma_s"])
    phi, q = dev(prob["phi_in"]), dev(prob["source"])
    om, w = prob["omega"], prob["weights"]
    k = "cluster" if kind == "cluster" else "cta"
    psi = mesh.sweep(st, ss, om, w, phi_in=phi, source=q, kernel=k)     # schedules built, warm
    g = mesh.region_weights((0.6, 0.6), (0.8, 0.8))
    if kind == "adjoint":
        mesh.adjoint(st, ss, om, w, psi, g, phi_in=phi)
    torch.cuda.synchronize()
    mesh.sync()

    def call(info):
        if kind == "adjoint":
            return mesh.adjoint(st, ss, om, w, psi, g, phi_in=phi, info=info)
        return mesh.sweep(st, ss, om, w, phi_in=phi, source=q, kernel=k, info=info)

    assert lib.vef_mesh_inject_status(mesh.handle, _lib.VEF_STATUS_TIMEOUT, None) == _lib.VEF_OK
    t = time.perf_counter()
    with pytest.raises(RuntimeError, match="VEF_ERR_TIMEOUT|timeout"):
        call(True)
    elapsed = time.perf_counter() - t
    print(f"{kind}: call with a pending timeout returned in {elapsed * 1e3:.1f} ms")
    assert elapsed < 5.0
    out = call(True)            # the word was cleared by the failing call
    disc = Discretization(N, N, 3, 0.08, p)
    ref = o_sweep(disc, om, w, prob["sigma_t"], prob["sigma_s"], phi_in=prob["phi_in"], source=prob["source"])
    if kind == "adjoint":
        gh = host(g)
        _, dst, dss = o_adjoint(disc, om, w, prob["sigma_t"], prob["sigma_s"], ref, gh, phi_in=prob["phi_in"])
        assert out[-1]["timed_out"] == 0
        assert rel(host(out[0]), dst) < 1e-12 and rel(host(out[1]), dss) < 1e-12
    else:
        assert out[1]["timed_out"] == 0
        assert rel(host(out[0]), ref) < 1e-12
    assert lib.vef_mesh_inject_status(mesh.handle, 0, None) == _lib.VEF_ERR_INVALID_ARG
    assert lib.vef_mesh_inject_status(None, 1, None) == _lib.VEF_ERR_INVALID_ARG
