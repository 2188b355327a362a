"""Pins for the oracle's moment / closure pass (paper Eq. vef_disc)."""
import os

import numpy as np
import pytest

from oracle.transport import Discretization
from oracle.moments import closures, angular_moments
from oracle import mms
from vef_inputs import level_symmetric
from _problems import nodal_xy

FOUR_PI = 4.0 * np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _psi_from(disc, om, fn):
    xn, yn = nodal_xy(disc)
    return np.stack([fn(xn, yn, om[d]) for d in range(len(om))])


@pytest.mark.parametrize("N", [4, 8, 12])
def test_isotropic_and_linear_flux_give_one_third(N):
    """Isotropic psi and linearly anisotropic psi = (a + Omega.b)/(4 pi) both give
    E = I/3 (the paper notes this for the diffusion-like MMS case)."""
    om, w = level_symmetric(N)
    disc = Discretization(4, 3, 3, 0.05, 2)
    for fn in (lambda x, y, O: 1.0 + x * y + 0 * O[0],
               lambda x, y, O: (2.0 + x + O[0] * (0.3 + y) - 0.5 * O[1] * x) / FOUR_PI):
        r = closures(disc, _psi_from(disc, om, fn), om, w)
        np.testing.assert_allclose(r["E"][0], 1 / 3, rtol=1e-13)
        np.testing.assert_allclose(r["E"][2], 1 / 3, rtol=1e-13)
        np.testing.assert_allclose(r["E"][1], 0.0, atol=1e-14)
        assert not r["nonpositive"]


def test_mms_moments_at_nodes_match_closed_forms():
    """phi, J, P of the manufactured psi: S4 integrates the degree-4 angular
    integrands exactly, so the nodal moments equal the closed forms (with the
    2 Theta_12/15 reading of the off-diagonal of P)."""
    om, w = level_symmetric(4)
    disc = Discretization(3, 3, 3, 0.05, 2)
    psi = _psi_from(disc, om, mms.psi)
    phi, J, P = angular_moments(psi, om, w)
    xn, yn = nodal_xy(disc)
    np.testing.assert_allclose(phi, mms.phi(xn, yn), rtol=1e-13)
    np.testing.assert_allclose(J, mms.current(xn, yn), atol=1e-14)
    np.testing.assert_allclose(P, mms.second_moment(xn, yn), rtol=1e-13, atol=1e-14)


def test_mms_eddington_tensor_converges():
    om, w = level_symmetric(4)
    errs = []
    for nx in (4, 8, 16):
        disc = Discretization(nx, nx, 3, 0.05, 2)
        r = closures(disc, _psi_from(disc, om, mms.psi), om, w)
        x, y = disc.mesh.xq[..., 0], disc.mesh.xq[..., 1]
        exact = mms.second_moment(x, y) / mms.phi(x, y)
        errs.append(np.abs(r["E"] - exact).max())
    rate = np.log2(errs[1] / errs[2])
    assert rate > 2.5, errs


def _golden_eb():
    out = {}
    for line in open(os.path.join(GOLDEN, "eb_isotropic_lqn.txt")):
        if line.strip() and not line.startswith("#"):
            N, v = line.split()
            out[int(N)] = float(v)
    return out


@pytest.mark.parametrize("N", [4, 8, 12, 16])
def test_boundary_factor_and_inflow_current(N):
    om, w = level_symmetric(N)
    disc = Discretization(3, 4, 3, 0.07, 2)
    g = disc.mesh
    psi = _psi_from(disc, om, lambda x, y, O: 2.0 + x - y + 0 * O[0])
    c = 0.8
    inflow = np.full((len(w), g.nbf, disc.nq), c)
    r = closures(disc, psi, om, w, inflow)
    np.testing.assert_allclose(r["Eb"], _golden_eb()[N], atol=6e-8)
    # half-range sums by axis: bottom/top faces use |eta|, left/right |mu|
    half_mu = np.sum(w * np.abs(om[:, 0])) / 2
    half_eta = np.sum(w * np.abs(om[:, 1])) / 2
    for bf, (e, f) in enumerate(g.boundary_faces()):
        expect = -c * (half_eta if f in (0, 2) else half_mu)
        np.testing.assert_allclose(r["Jin"][bf], expect, rtol=1e-13)


def test_nonpositive_denominator_flagged():
    om, w = level_symmetric(4)
    disc = Discretization(2, 2, 1, 0.0, 1)
    psi = np.ones((len(w), disc.mesh.E, disc.n))
    psi[:, 0, :] = 0.0
    r = closures(disc, psi, om, w)
    assert r["nonpositive"]
    assert np.isnan(r["E"][:, 0]).all() and np.isfinite(r["E"][:, 1:]).all()
