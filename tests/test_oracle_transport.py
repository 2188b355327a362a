"""Pins for the oracle's upwind DG transport solve (closed forms, invariants, orders).

Each test is chosen so that a plausible slip in the weak form (a dropped or
transposed streaming term, a wrong face normal sign or neighbour index, a missing
sigma term) breaks it:
  * constant solution: exact for any mesh order, cross sections and p;
  * linear solution psi = a + b.x: exact when the mesh map is in Q_p and the
    quadrature integrates the transformed integrands exactly;
  * per-element particle balance (test function v = 1);
  * pure absorber exp(-sigma_t s): O(h^(p+1)) L2 convergence;
  * the paper's manufactured solution on sine-curved Q3 meshes: O(h^(p+1));
  * a brute-force dense solve of the same global system.
"""
import numpy as np
import pytest

from oracle.transport import Discretization, sweep
from vef_inputs import level_symmetric
from _problems import nodal_xy, boundary_values, l2_error_psi, mms_problem, fit_order
from oracle import mms

FOUR_PI = 4.0 * np.pi


@pytest.mark.parametrize("nx,m,p,alpha", [(4, 3, 1, 0.05), (4, 3, 2, 0.08), (3, 2, 3, 0.05), (5, 1, 2, 0.0)])
def test_constant_solution_exact(nx, m, p, alpha):
    om, w = level_symmetric(4)
    disc = Discretization(nx, nx + 1, m, alpha, p)
    E, n = disc.mesh.E, disc.n
    rng = np.random.default_rng(7)
    st = rng.uniform(0.1, 20.0, E)
    ss = rng.uniform(0.0, 1.0, E) * st
    c = 1.7
    phi_in = np.full((E, n), FOUR_PI * c)
    q = np.repeat(((st - ss) * c)[:, None], n, axis=1)
    inflow = np.full((len(w), disc.mesh.nbf, disc.nq), c)
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=q, inflow=inflow)
    np.testing.assert_allclose(psi, c, rtol=1e-12)


@pytest.mark.parametrize("nx,m,p,alpha", [(4, 1, 1, 0.0), (4, 1, 3, 0.0), (4, 2, 2, 0.05), (3, 3, 3, 0.05)])
def test_linear_solution_exact(nx, m, p, alpha):
    om, w = level_symmetric(6)
    disc = Discretization(nx, nx, m, alpha, p)
    E, n = disc.mesh.E, disc.n
    a, b = 2.0, np.array([0.7, -0.4])
    st = np.linspace(0.5, 4.0, E)
    ss = 0.3 * st
    xn, yn = nodal_xy(disc)
    lin = a + b[0] * xn + b[1] * yn
    phi_in = FOUR_PI * lin
    src = np.stack([om[d] @ b + st[:, None] * lin - ss[:, None] * phi_in / FOUR_PI
                    for d in range(len(w))])
    inflow = boundary_values(disc, om, lambda x, y, O: a + b[0] * x + b[1] * y)
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=src, inflow=inflow)
    np.testing.assert_allclose(psi, np.broadcast_to(lin, psi.shape), rtol=1e-11, atol=1e-12)


def test_particle_balance_per_element():
    om, w = level_symmetric(4)
    disc = Discretization(4, 4, 3, 0.06, 2)
    g = disc.mesh
    E, n = g.E, disc.n
    rng = np.random.default_rng(3)
    st = rng.uniform(0.5, 5.0, E)
    ss = 0.5 * st
    phi_in = rng.uniform(0.5, 2.0, (E, n))
    q = rng.uniform(0.0, 1.0, (E, n))
    inflow = rng.uniform(0.0, 1.0, (len(w), g.nbf, disc.nq))
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=q, inflow=inflow)
    for d in range(len(w)):
        c = np.einsum("k,efkx,x->efk", g.wf, g.nds, om[d])
        for e in range(E):
            outflow = 0.0
            for f in range(4):
                own = disc.Bf[f] @ psi[d, e]
                nb = g.nb[e, f]
                if nb >= 0:
                    up = disc.Bf[g.nbface[e, f]] @ psi[d, nb]
                else:
                    up = inflow[d, g.nbface[e, f]]
                outflow += np.sum(c[e, f] * np.where(c[e, f] >= 0, own, up))
            absorb = st[e] * np.sum(g.wq * g.J[e] * (disc.B @ psi[d, e]))
            srcint = np.sum(g.wq * g.J[e] * (disc.B @ (ss[e] * phi_in[e] / FOUR_PI + q[e])))
            assert abs(outflow + absorb - srcint) <= 1e-12 * abs(srcint)


def _absorber(x, y, O, sig=2.0):
    x0 = 0.0 if O[0] > 0 else 1.0
    return np.exp(-sig * (x - x0) / O[0])


@pytest.mark.parametrize("p", [1, 2])
def test_pure_absorber_convergence(p):
    om, w = level_symmetric(4)
    errs, hs = [], []
    for nx in (4, 8, 16):
        disc = Discretization(nx, nx, 3, 0.05, p)
        E = disc.mesh.E
        inflow = boundary_values(disc, om, _absorber)
        psi = sweep(disc, om, w, np.full(E, 2.0), np.zeros(E), inflow=inflow)
        errs.append(l2_error_psi(disc, psi, om, w, _absorber))
        hs.append(1.0 / nx)
    assert fit_order(hs, errs) > p + 1 - 0.25
    assert errs[-1] < 1e-2


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mms_convergence_sine_mesh(p):
    om, w = level_symmetric(4)
    errs, hs = [], []
    for nx in (4, 8, 16):
        disc, st, ss, src, inflow = mms_problem(nx, 3, 0.05, p, om)
        psi = sweep(disc, om, w, st, ss, source=src, inflow=inflow)
        errs.append(l2_error_psi(disc, psi, om, w, mms.psi))
        hs.append(1.0 / nx)
    assert fit_order(hs, errs) > p + 1 - 0.3


def test_sparse_solve_matches_dense():
    om, w = level_symmetric(4)
    disc = Discretization(3, 3, 3, 0.08, 2)
    E = disc.mesh.E
    rng = np.random.default_rng(11)
    st = rng.uniform(0.2, 3.0, E)
    ss = 0.9 * st
    phi_in = rng.uniform(0.0, 1.0, (E, disc.n))
    inflow = rng.uniform(0.0, 1.0, (len(w), disc.mesh.nbf, disc.nq))
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=np.ones((E, disc.n)), inflow=inflow)
    for d in range(len(w)):
        L, c = disc.operator(om[d], st)
        b = disc.rhs(c, d, ss, phi_in, np.ones((E, disc.n)), inflow)
        dense = np.linalg.solve(L.toarray(), b.ravel())
        np.testing.assert_allclose(psi[d].ravel(), dense, rtol=1e-12, atol=1e-14)
