"""The oracle's VEF fixed-point iteration (transport sweep, closures, hybridized RT VEF solve)
against the paper's own numbers and the diffusion limit.

* Table tdl (tests/golden/tdl_hrt_orthogonal.txt): the iteration counts of the HRT method
  on the orthogonal 8x8 thick-diffusion-limit problem are reproduced exactly from phi^0 = 0
  with the paper's stopping rule (max norm of successive differences <= 1e-6);
* the converged VEF scalar flux tends to the closed-form diffusion limit
  -(1/3) Lap(phi) + phi = 4 pi, phi = 0 on the boundary, as eps -> 0.
"""
import os

import numpy as np
import pytest

from oracle.iteration import vef_iterate
from oracle.transport import Discretization
from vef_inputs import level_symmetric
from _problems import nodal_xy
from test_oracle_diffusion_limit import _diffusion_series

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tdl_hrt_orthogonal.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [(float(a), int(b)) for a, b in rows]


def _tdl(eps, disc):
    E, n = disc.mesh.E, disc.n
    return np.full(E, 1.0 / eps), np.full(E, 1.0 / eps - eps), np.full((E, n), eps)


@pytest.mark.parametrize("eps,iterations", _golden())
def test_fixed_point_counts_match_table_tdl(eps, iterations):
    om, w = level_symmetric(4)
    disc = Discretization(8, 8, 1, 0.0, 2)
    st, ss, q = _tdl(eps, disc)
    _, _, its, hist = vef_iterate(disc, om, w, st, ss, q, K=40, tol=1e-6)
    assert its == iterations, hist
    assert hist[-1] <= 1e-6 < hist[-2]


def test_converged_vef_flux_approaches_the_diffusion_limit():
    om, w = level_symmetric(4)
    disc = Discretization(8, 8, 1, 0.0, 2)
    xn, yn = nodal_xy(disc)
    limit = _diffusion_series(xn, yn)
    gaps = []
    for eps in (1e-2, 1e-3):
        st, ss, q = _tdl(eps, disc)
        phi, _, _, _ = vef_iterate(disc, om, w, st, ss, q, K=40, tol=1e-10)
        gaps.append(np.linalg.norm(phi - limit) / np.linalg.norm(limit))
    assert gaps[1] < gaps[0] and gaps[1] < 2e-2, gaps
