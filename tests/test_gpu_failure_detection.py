"""Failure detection on the GPU without a fault: a bounded wait that nothing completes
reports VEF_ERR_TIMEOUT through the status word, within its poll budget, and the CUDA
context stays usable (a sweep right after matches the oracle)."""
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
