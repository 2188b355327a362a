"""The VEF fixed-point iteration on the GPU (vef_vef_iterate: sweep, closures, hybridized RT
VEF solve per iteration) against the paper's Table tdl and the oracle's iteration."""
import os

import numpy as np
import pytest

from _gpu import dev, host, rel
from oracle.iteration import vef_iterate
from oracle.transport import Discretization
from vef_inputs import level_symmetric

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tdl_hrt_orthogonal.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [(float(a), int(b)) for a, b in rows]


def _tdl(eps, E, n):
    return np.full(E, 1.0 / eps), np.full(E, 1.0 / eps - eps), np.full((E, n), eps)


@pytest.mark.parametrize("eps,iterations", _golden())
def test_table_tdl_iteration_counts_and_oracle_parity(lib, eps, iterations):
    """Orthogonal 8x8 mesh, S4, p = 2, phi^0 = 0, tolerance 1e-6: the GPU iteration takes the
    paper's HRT iteration counts and its scalar flux matches the oracle's."""
    from paper_2301_04758_gb300.api import Mesh
    om, w = level_symmetric(4)
    mesh = Mesh(8, 8, 1, 2, 0.0)
    st, ss, q = _tdl(eps, mesh.E, mesh.n)
    phi, J, psi, dphi, info = mesh.vef_iterate(dev(st), dev(ss), om, w, source=dev(q), tol=1e-6)
    assert info["converged"] == 1 and info["iterations"] == iterations, (info, host(dphi))
    disc = Discretization(8, 8, 1, 0.0, 2)
    ref, Jref, its, _ = vef_iterate(disc, om, w, st, ss, q, K=40, tol=1e-6)
    assert its == iterations
    assert rel(host(phi), ref) < 1e-9
    assert rel(host(J), Jref) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_curved_mesh_with_inflow_against_the_oracle(lib, precision):
    """Sine-curved Q3 mesh, eps = 1e-1, an isotropic inflow of 0.5 on the whole boundary
    (the angular flux stays positive, as the VEF data need): same iteration count and
    scalar flux as the oracle, with FP64 sweeps and with mixed-precision sweeps."""
    from paper_2301_04758_gb300.api import Mesh
    nx, p, eps = 8, 2, 1e-1
    om, w = level_symmetric(4)
    mesh = Mesh(nx, nx, 3, p, 0.05)
    st, ss, q = _tdl(eps, mesh.E, mesh.n)
    inflow = np.full((len(w), mesh.nbf, mesh.nq), 0.5)
    disc = Discretization(nx, nx, 3, 0.05, p)
    ref, _, its, hist = vef_iterate(disc, om, w, st, ss, q, inflow=inflow, K=40, tol=1e-8)
    phi, _, _, dphi, info = mesh.vef_iterate(dev(st), dev(ss), om, w, source=dev(q), inflow=dev(inflow), tol=1e-8,
                                             precision=precision)
    assert info["iterations"] == its, (info, hist, host(dphi))
    assert rel(host(phi), ref) < (1e-9 if precision == "fp64" else 1e-8)
