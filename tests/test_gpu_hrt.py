"""GPU parity of the hybridized RT VEF solve (vef_hrt_solve) against the CPU oracle.

The oracle (oracle/hrt.py, pinned in tests/test_oracle_hrt.py) eliminates the same element
blocks and solves the multiplier system directly; the library eliminates them on the GPU and
solves the multiplier system by BiCGStab (two-level Schwarz preconditioner: element patches
plus a coarse bilinear space) to a relative residual of 1e-14, so phi, J and lambda agree to
about the conditioning of H times that.
"""
import numpy as np
import pytest

from _gpu import dev, host, rel, random_problem
from oracle.hrt import HRT
from oracle.transport import Discretization

pytestmark = pytest.mark.gpu


def _vef_inputs(disc, seed):
    g = disc.mesh
    rng = np.random.default_rng(seed)
    phi = rng.uniform(1.0, 2.0, (g.E, disc.n))
    P = np.stack([rng.uniform(0.25, 0.45, (g.E, disc.n)) * phi, rng.uniform(-0.05, 0.05, (g.E, disc.n)) * phi,
                  rng.uniform(0.25, 0.45, (g.E, disc.n)) * phi])
    Eb = rng.uniform(0.45, 0.55, (g.nbf, disc.nq))
    Jin = -rng.uniform(0.0, 0.3, (g.nbf, disc.nq))
    Q0 = rng.uniform(0.5, 1.5, (g.E, disc.n))
    Q1 = rng.uniform(-0.2, 0.2, (2, g.E, disc.n))
    st = rng.uniform(0.5, 5.0, g.E)
    ss = rng.uniform(0.3, 0.95, g.E) * st
    return phi, P, Eb, Jin, Q0, Q1, st, ss


def _oracle(disc, phi, P, Eb, Jin, Q0, Q1, st, ss):
    hrt = HRT(disc)
    Eq, Ef = hrt.eddington_data(phi, P)
    Q0q = np.einsum("qj,ej->eq", disc.B, Q0)
    Q1q = None if Q1 is None else np.einsum("qj,cej->eqc", disc.B, Q1)
    return hrt.solve(st, ss, Eq, Ef, Eb, Jin, Q0q, Q1q)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hrt_solve_matches_the_oracle(lib, p):
    from paper_2301_04758_gb300.api import Mesh
    nx, ny = 6, 5
    disc = Discretization(nx, ny, 3, 0.08, p)
    phi, P, Eb, Jin, Q0, Q1, st, ss = _vef_inputs(disc, 300 + p)
    ref = _oracle(disc, phi, P, Eb, Jin, Q0, Q1, st, ss)
    mesh = Mesh(nx, ny, 3, p, 0.08)
    gphi, gJ, glam, info = mesh.hrt_solve(dev(st), dev(ss), dev(phi), dev(P), dev(Eb), dev(Jin), dev(Q0),
                                          dev(Q1), tol=1e-14)
    assert info["rel_residual"] <= 1e-14 and info["multipliers"] == ref["lam"].size, info
    assert rel(host(glam), ref["lam"]) < 1e-10, info
    assert rel(host(gphi), ref["phi"]) < 1e-10, info
    assert rel(host(gJ), ref["J"]) < 1e-10, info


@pytest.mark.parametrize("nx,ny,p", [(25, 23, 1), (25, 23, 2), (14, 13, 3), (12, 12, 4)])
def test_hrt_solve_on_meshes_with_ragged_coarse_cells(lib, nx, ny, p):
    """The preconditioner's coarse grid has at most 11 cells per direction, each a block of
    whole elements, the last ones smaller (25 x 23: cells of 3 x 3 elements, the last column
    one element wide and the last row two high).  The Krylov answer does not depend on the
    preconditioner, so this checks that the coarse space with ragged cells converges to the
    oracle's direct solution within the iteration limit."""
    from paper_2301_04758_gb300.api import Mesh
    disc = Discretization(nx, ny, 3, 0.08, p)
    phi, P, Eb, Jin, Q0, Q1, st, ss = _vef_inputs(disc, 900 + p)
    ref = _oracle(disc, phi, P, Eb, Jin, Q0, Q1, st, ss)
    mesh = Mesh(nx, ny, 3, p, 0.08)
    gphi, gJ, glam, info = mesh.hrt_solve(dev(st), dev(ss), dev(phi), dev(P), dev(Eb), dev(Jin), dev(Q0),
                                          dev(Q1), tol=1e-13)
    assert info["rel_residual"] <= 1e-13 and info["multipliers"] == ref["lam"].size, info
    assert rel(host(glam), ref["lam"]) < 1e-9, info
    assert rel(host(gphi), ref["phi"]) < 1e-9, info
    assert rel(host(gJ), ref["J"]) < 1e-9, info


def test_one_vef_step_after_a_transport_sweep(lib):
    """A transport sweep, its closures (phi, P, E_b, J_in) and the HRT VEF solve, all on the
    GPU, against the same chain in the oracle: one outer iteration of the VEF method on a
    sine-curved mesh with a scattering source and inflow."""
    from paper_2301_04758_gb300.api import Mesh
    from oracle.transport import sweep as o_sweep
    from oracle.moments import angular_moments, boundary_closures
    nx, p = 7, 2
    prob = random_problem(nx, nx, 3, 0.05, p, 6, seed=510)
    disc = Discretization(nx, nx, 3, 0.05, p)
    psi_ref = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                      phi_in=prob["phi_in"], source=prob["source"], inflow=prob["inflow"])
    phi_r, _, P_r = angular_moments(psi_ref, prob["omega"], prob["weights"])
    Eb_r, Jin_r, _ = boundary_closures(disc, psi_ref, prob["omega"], prob["weights"], prob["inflow"])
    Q0 = 4 * np.pi * prob["source"]
    ref = _oracle(disc, phi_r, P_r, Eb_r, Jin_r, Q0, None, prob["sigma_t"], prob["sigma_s"])
    mesh = Mesh(nx, nx, 3, p, 0.05)
    st, ss = dev(prob["sigma_t"]), dev(prob["sigma_s"])
    psi = mesh.sweep(st, ss, prob["omega"], prob["weights"], phi_in=dev(prob["phi_in"]),
                     source=dev(prob["source"]), inflow=dev(prob["inflow"]))
    mom = mesh.moments(psi, prob["omega"], prob["weights"], inflow=dev(prob["inflow"]),
                       outputs=("phi", "P", "Eb", "Jin"))
    gphi, gJ, _, info = mesh.hrt_solve(st, ss, mom["phi"], mom["P"], mom["Eb"], mom["Jin"], dev(Q0), tol=1e-14)
    assert rel(host(gphi), ref["phi"]) < 1e-10, info
    assert rel(host(gJ), ref["J"]) < 1e-10, info
