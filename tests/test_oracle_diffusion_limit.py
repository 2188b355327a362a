"""Thick diffusion limit of the oracle's transport discretisation (Sec. "Thick Diffusion
Limit": sigma_t = 1/eps, sigma_a = eps, sigma_s = 1/eps - eps, q = eps, S4, p = 2,
8 x 8 mesh on the unit square).

As eps -> 0 the scattering-coupled transport solution tends to the solution of the
diffusion equation  -(1/3) Lap(phi) + phi = 4 pi  (the 1/3 is sum_d w_d mu_d^2 / 4 pi, the
4 pi is the isotropic source q = eps integrated over angle, both divided by eps) with phi = 0
on the boundary (the vacuum boundary layer is O(eps) thick).  That problem has a
closed-form sine series.  The gap between the two shrinks like eps, and the Eddington
tensor tends to I/3 away from the boundary.  A dropped scattering term, a wrong sign of
the streaming term, a mis-normalised angular weight or source, or a wrong geometric
factor on the curved mesh each breaks the limit.

The coupled system over all directions is solved at once (sparse direct), the same brute
force the source-iteration pin uses.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.transport import Discretization
from oracle.moments import closures
from vef_inputs import level_symmetric
from _problems import nodal_xy

FOUR_PI = 4.0 * np.pi


def _coupled_psi(disc, om, w, st, ss, q):
    E, n, D = disc.mesh.E, disc.n, len(w)
    Ms = sp.block_diag([sp.csr_matrix(ss[e] / FOUR_PI * disc.M[e]) for e in range(E)], format="csr")
    blocks = [[None] * D for _ in range(D)]
    rhs = []
    for d in range(D):
        L, c = disc.operator(om[d], st)
        rhs.append(disc.rhs(c, d, ss, None, q, None).ravel())
        for dd in range(D):
            blk = -w[dd] * Ms
            if dd == d:
                blk = blk + L
            blocks[d][dd] = blk
    return spla.spsolve(sp.bmat(blocks).tocsc(), np.concatenate(rhs)).reshape(D, E, n)


def _diffusion_series(x, y, modes=100):
    """-(1/3) Lap(phi) + phi = 4 pi on [0,1]^2, phi = 0 on the boundary.  The constant 1
    has the double sine coefficients 16 / (pi^2 j k) for odd j, k (zero otherwise), and
    each mode sin(j pi x) sin(k pi y) is divided by its eigenvalue 1 + (j^2 + k^2) pi^2 / 3."""
    phi = np.zeros_like(x)
    for j in range(1, 2 * modes, 2):
        sx = np.sin(j * np.pi * x)
        for k in range(1, 2 * modes, 2):
            c = 16.0 * FOUR_PI / (np.pi ** 2 * j * k) / (1.0 + (j * j + k * k) * np.pi ** 2 / 3.0)
            phi += c * sx * np.sin(k * np.pi * y)
    return phi


def test_series_solves_the_diffusion_problem():
    """The closed form itself: a five-point finite-difference residual of the series is
    small in the interior, and it vanishes on the boundary."""
    h = 1.0 / 64
    xs = np.arange(1, 64) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    phi = _diffusion_series(X, Y)
    pad = np.pad(phi, 1)
    lap = (pad[2:, 1:-1] + pad[:-2, 1:-1] + pad[1:-1, 2:] + pad[1:-1, :-2] - 4 * phi) / h ** 2
    res = -lap / 3.0 + phi - FOUR_PI
    assert np.abs(res[8:-8, 8:-8]).max() < 1e-2 * FOUR_PI
    assert np.abs(_diffusion_series(np.zeros(5), np.linspace(0, 1, 5))).max() == 0.0


@pytest.mark.parametrize("m,alpha", [(1, 0.0), (3, 0.05)], ids=["orthogonal", "sine_q3"])
def test_thick_diffusion_limit(m, alpha):
    om, w = level_symmetric(4)
    disc = Discretization(8, 8, m, alpha, 2)
    E, n = disc.mesh.E, disc.n
    xn, yn = nodal_xy(disc)
    limit = _diffusion_series(xn, yn)
    ie, je = np.arange(E) % 8, np.arange(E) // 8
    inner = (ie > 0) & (ie < 7) & (je > 0) & (je < 7)
    gaps, e_dev = [], []
    for eps in (1e-2, 1e-3):
        st = np.full(E, 1.0 / eps)
        ss = np.full(E, 1.0 / eps - eps)
        q = np.full((E, n), eps)
        r = closures(disc, _coupled_psi(disc, om, w, st, ss, q), om, w)
        gaps.append(np.linalg.norm(r["phi"] - limit) / np.linalg.norm(limit))
        Ei = r["E"][:, inner]
        e_dev.append(max(np.abs(Ei[0] - 1 / 3).max(), np.abs(Ei[2] - 1 / 3).max(), np.abs(Ei[1]).max()))
    # O(eps) approach of the diffusion solution (measured 4.4e-2 and 4.4e-3 on both meshes)
    assert gaps[0] < 6e-2 and gaps[1] < 6e-3, gaps
    assert gaps[0] / gaps[1] > 8.0, gaps
    # E -> I/3 in the interior, faster than eps (measured 4e-4 / 7e-4 and 4e-6 / 8e-6)
    assert e_dev[1] < 2e-5 and e_dev[0] / e_dev[1] > 30.0, e_dev
