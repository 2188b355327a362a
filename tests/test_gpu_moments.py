"""GPU parity of the moment / closure pass (paper Eq. vef_disc) against the oracle."""
import numpy as np
import pytest

from _gpu import dev, host, rel, random_problem
from oracle.transport import Discretization
from oracle.moments import closures
from vef_inputs import level_symmetric

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,sn", [(1, 4), (2, 8), (3, 12), (4, 16)])
def test_moments_match_oracle(lib, p, sn):
    from paper_2301_04758_gb300.api import Mesh
    nx, ny = 6, 5
    om, w = level_symmetric(sn)
    rng = np.random.default_rng(p)
    E, n, nq = nx * ny, (p + 1) ** 2, p + 2
    psi = rng.uniform(0.1, 2.0, (len(w), E, n))
    inflow = rng.uniform(0.0, 1.0, (len(w), 2 * nx + 2 * ny, nq))
    mesh = Mesh(nx, ny, 3, p, 0.05)
    out = mesh.moments(dev(psi), om, w, inflow=dev(inflow))
    mesh.sync()
    disc = Discretization(nx, ny, 3, 0.05, p)
    rc = closures(disc, psi, om, w, inflow)
    for k_gpu, k_ref in (("phi", "phi"), ("J", "J"), ("P", "P"), ("E", "E"), ("Eb", "Eb"),
                         ("Jin", "Jin")):
        assert rel(host(out[k_gpu]), rc[k_ref]) < 1e-13, k_gpu


def test_isotropic_gives_one_third_and_eb_table(lib):
    from paper_2301_04758_gb300.api import Mesh
    om, w = level_symmetric(8)
    mesh = Mesh(4, 4, 3, 2, 0.07)
    psi = np.ones((len(w), mesh.E, mesh.n)) * 3.0
    out = mesh.moments(dev(psi), om, w)
    E = host(out["E"])
    assert np.abs(E[0] - 1 / 3).max() < 1e-14 and np.abs(E[1]).max() < 1e-14
    assert np.abs(host(out["Eb"]) - 0.5085137).max() < 6e-8


def test_nonpositive_denominator_reported(lib):
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    om, w = level_symmetric(4)
    mesh = Mesh(2, 2, 1, 1, 0.0)
    psi = np.ones((len(w), mesh.E, mesh.n))
    psi[:, 0] = 0.0
    out = mesh.moments(dev(psi), om, w)
    with pytest.raises(_lib.VefError) as ei:
        mesh.sync()
    assert ei.value.status == _lib.VEF_ERR_NONPOSITIVE_DENOM
    E = host(out["E"])
    assert np.isnan(E[:, 0]).all() and np.isfinite(E[:, 1:]).all()
    mesh.sync()   # status was cleared by the previous check
