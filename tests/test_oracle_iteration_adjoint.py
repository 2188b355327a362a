"""Pins for source iteration and the adjoint gradients."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.transport import Discretization, sweep
from oracle.iteration import source_iterate
from oracle.adjoint import adjoint, region_weights
from vef_inputs import level_symmetric, seeded_media

FOUR_PI = 4.0 * np.pi


def _coupled_direct(disc, om, w, st, ss, q, inflow):
    """Brute force: the scattering-coupled system over all directions at once,
    psi_d - L_d^{-1}(M sigma_s/(4 pi) sum_d' w_d' psi_d') = L_d^{-1} b_d, solved as one
    sparse system in (psi_1..psi_D)."""
    E, n, D = disc.mesh.E, disc.n, len(w)
    blocks = [[None] * D for _ in range(D)]
    rhs = []
    Ms = sp.block_diag([sp.csr_matrix(ss[e] / FOUR_PI * disc.M[e]) for e in range(E)], format="csr")
    for d in range(D):
        L, c = disc.operator(om[d], st)
        rhs.append(disc.rhs(c, d, ss, None, q, inflow).ravel())
        for dd in range(D):
            blk = -w[dd] * Ms
            if dd == d:
                blk = blk + L
            blocks[d][dd] = blk
    A = sp.bmat(blocks).tocsc()
    psi = spla.spsolve(A, np.concatenate(rhs)).reshape(D, E, n)
    return np.einsum("d,den->en", w, psi)


def test_source_iteration_converges_to_coupled_solution():
    om, w = level_symmetric(4)
    disc = Discretization(3, 3, 3, 0.05, 1)
    E = disc.mesh.E
    st, ss = seeded_media(E, 5, log10_range=(-0.5, 0.5), c_range=(0.3, 0.6))
    q = np.ones((E, disc.n))
    inflow = np.zeros((len(w), disc.mesh.nbf, disc.nq))
    phi_star = _coupled_direct(disc, om, w, st, ss, q, inflow)
    phi, _, dinf = source_iterate(disc, om, w, st, ss, source=q, inflow=inflow, K=40)
    np.testing.assert_allclose(phi, phi_star, rtol=1e-11)
    assert dinf[0] > dinf[5] > dinf[20]
    # contraction no faster than ... and no slower than the largest scattering ratio
    ratio = dinf[20] / dinf[19]
    assert 0.0 < ratio <= (ss / st).max() + 1e-9


def test_constant_fixed_point_of_source_iteration():
    om, w = level_symmetric(4)
    disc = Discretization(3, 3, 3, 0.05, 2)
    E, n = disc.mesh.E, disc.n
    st = np.full(E, 2.0)
    ss = np.full(E, 1.0)
    c = 0.5
    q = np.full((E, n), (2.0 - 1.0) * c)
    inflow = np.full((len(w), disc.mesh.nbf, disc.nq), c)
    phi, _, dinf = source_iterate(disc, om, w, st, ss, source=q, inflow=inflow, K=3,
                                  phi0=np.full((E, n), FOUR_PI * c))
    np.testing.assert_allclose(phi, FOUR_PI * c, rtol=1e-12)
    assert dinf.max() < 1e-11


def _R(disc, om, w, st, ss, phi_in, q, inflow, g):
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=q, inflow=inflow)
    return float(np.sum(g * np.einsum("d,den->en", w, psi))), psi


def test_adjoint_gradients_match_central_differences():
    om, w = level_symmetric(4)
    disc = Discretization(4, 4, 3, 0.05, 2)
    E, n = disc.mesh.E, disc.n
    st, ss = seeded_media(E, 5)
    rng = np.random.default_rng(2)
    phi_in = rng.uniform(0.5, 1.5, (E, n))
    q = np.ones((E, n))
    inflow = rng.uniform(0.0, 0.2, (len(w), disc.mesh.nbf, disc.nq))
    g = region_weights(disc, (0.3, 0.3), (0.8, 0.8))
    R0, psi = _R(disc, om, w, st, ss, phi_in, q, inflow, g)
    lam, dst, dss = adjoint(disc, om, w, st, ss, psi, g, phi_in=phi_in)
    # R = sum_d lambda_d^T b_d
    Rb = 0.0
    for d in range(len(w)):
        L, c = disc.operator(om[d], st)
        Rb += np.sum(lam[d] * disc.rhs(c, d, ss, phi_in, q, inflow))
    np.testing.assert_allclose(Rb, R0, rtol=1e-12)
    for e in (0, 5, 10, 15):
        for arr, grad in ((st, dst), (ss, dss)):
            h = 1e-6 * arr[e]
            arr[e] += h
            Rp, _ = _R(disc, om, w, st, ss, phi_in, q, inflow, g)
            arr[e] -= 2 * h
            Rm, _ = _R(disc, om, w, st, ss, phi_in, q, inflow, g)
            arr[e] += h
            fd = (Rp - Rm) / (2 * h)
            assert abs(fd - grad[e]) <= 1e-6 * max(abs(fd), 1e-3 * abs(grad).max()), (e, fd, grad[e])


def test_adjoint_pure_absorber_closed_form():
    """sigma_s = 0, boundary data exp(-sigma0 (x - x0)/mu) held fixed: the exact
    flux is psi = exp(-sigma0 (x - x0)/mu) and d psi/d sigma = -s psi, with s the path
    length from the inflow boundary along the (mu, eta) ray.  The adjoint's total
    dR/dsigma_t for R = int phi over [0,1]^2 approaches -sum_d w_d int s psi dx."""
    om, w = level_symmetric(4)
    sig = 1.5
    disc = Discretization(8, 8, 1, 0.0, 3)
    E = disc.mesh.E

    def ex(x, y, O):
        x0 = 0.0 if O[0] > 0 else 1.0
        return np.exp(-sig * (x - x0) / O[0])

    from _problems import boundary_values
    inflow = boundary_values(disc, om, ex)
    g = region_weights(disc, (0.0, 0.0), (1.0, 1.0))
    psi = sweep(disc, om, w, np.full(E, sig), np.zeros(E), inflow=inflow)
    _, dst, _ = adjoint(disc, om, w, np.full(E, sig), np.zeros(E), psi, g)
    h = 1.0 / 1500
    xs = (np.arange(1500) + 0.5) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    expect = 0.0
    for d in range(len(w)):
        mu, eta = om[d]
        dx = X if mu > 0 else 1 - X
        dy = Y if eta > 0 else 1 - Y
        s = np.minimum(dx / abs(mu), dy / abs(eta))
        expect -= w[d] * np.sum(s * ex(X, Y, om[d])) * h * h
    np.testing.assert_allclose(dst.sum(), expect, rtol=2e-3)


def test_region_weights_integrate_exactly_on_an_aligned_region():
    """On a straight 10 x 10 mesh the region [0.6, 0.8]^2 is a union of whole elements, so
    sum g * phi is the exact integral of any phi in Q_p over it: phi = x^2 y (p = 2)
    gives (0.8^3 - 0.6^3)/3 * (0.8^2 - 0.6^2)/2, and phi = 1 the area 0.04."""
    from _problems import nodal_xy
    disc = Discretization(10, 10, 1, 0.0, 2)
    g = region_weights(disc, (0.6, 0.6), (0.8, 0.8))
    xn, yn = nodal_xy(disc)
    exact = (0.8 ** 3 - 0.6 ** 3) / 3 * (0.8 ** 2 - 0.6 ** 2) / 2
    np.testing.assert_allclose(np.sum(g * xn ** 2 * yn), exact, rtol=1e-13)
    np.testing.assert_allclose(np.sum(g), 0.04, rtol=1e-13)
    # only the four elements inside carry weight
    assert np.count_nonzero(np.abs(g).sum(axis=1) > 0) == 4
