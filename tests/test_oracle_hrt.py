"""Pins for the oracle's hybridized RT VEF discretisation (oracle/hrt.py).

  * Piola-mapped fields: the gradient formula (map's first and second derivatives)
    against finite differences of the mapped field, and its trace against the Piola
    identity div v = div_hat v_hat / J (paper Eqs. piola_grad, piola_div), on curved
    elements; the Lagrange second derivatives and the map's Hessian they use;
  * a manufactured solution with a spatially varying, non-diagonal Eddington tensor on
    sine-curved Q3 meshes: phi and J converge at O(h^(p+1)) (a dropped or mis-signed
    term of A, G, D, Ma, the boundary form or the hybridization breaks the order);
  * the element-local elimination (H lambda = C1 (W g + X f), back substitution) equals the
    brute-force solve of the global saddle-point system;
  * the element block inverse equals the paper's Schur-complement formulas for W, X, Y, Z;
  * in the thick diffusion limit E = I/3 the method is the RT discretisation of diffusion:
    G = -D^T / 3 and C2 = C1^T / 3 element by element, and H is symmetric positive definite.
"""
import numpy as np
import pytest

from oracle.basis import gll_points, lagrange_deriv2
from oracle.hrt import HRT, rt_basis
from oracle.mesh import control_points, map_hessian, map_jacobian
from oracle.transport import Discretization

sy = pytest.importorskip("sympy")


def test_lagrange_second_derivatives_and_map_hessian():
    nodes = gll_points(4)
    x = np.linspace(0.0, 1.0, 9)
    for k in range(5):   # exact for the polynomials the nodes interpolate
        V = nodes ** k
        want = k * (k - 1) * x ** max(k - 2, 0) if k >= 2 else 0.0 * x
        np.testing.assert_allclose(lagrange_deriv2(nodes, x) @ V, want, atol=1e-11)
    ctrl = control_points(3, 3, 3, 0.08)
    px, py = np.array([0.3, 0.71, 0.05]), np.array([0.2, 0.9, 0.5])
    H = map_hessian(ctrl, 3, px, py)
    h = 1e-6
    for l, (dx, dy) in enumerate(((h, 0.0), (0.0, h))):
        _, Fp = map_jacobian(ctrl, 3, px + dx, py + dy)
        _, Fm = map_jacobian(ctrl, 3, px - dx, py - dy)
        np.testing.assert_allclose((Fp - Fm) / (2 * h), H[..., :, :, l], atol=1e-8)


@pytest.mark.parametrize("p", [1, 3])
def test_piola_gradient_against_finite_differences(p):
    disc = Discretization(3, 3, 3, 0.08, p)
    hrt = HRT(disc)
    g = disc.mesh
    e = 4
    # Piola identity: the trace of grad v is the reference divergence over J
    np.testing.assert_allclose(np.einsum("knii->kn", hrt.gq[e]), hrt.div / g.J[e][:, None], atol=1e-11)
    px, py = g.ref_vol
    eps = 1e-6

    def mapped(qx, qy):
        V = rt_basis(p, qx, qy)[0]
        _, F = map_jacobian(g.ctrl, g.m, qx, qy)
        J = F[..., 0, 0] * F[..., 1, 1] - F[..., 0, 1] * F[..., 1, 0]
        return np.einsum("kij,knj->kni", F[e], V) / J[e][:, None, None], F[e]
    dxi = (mapped(px + eps, py)[0] - mapped(px - eps, py)[0]) / (2 * eps)
    deta = (mapped(px, py + eps)[0] - mapped(px, py - eps)[0]) / (2 * eps)
    Finv = np.linalg.inv(mapped(px, py)[1])
    fd = np.einsum("knil,klm->knim", np.stack([dxi, deta], -1), Finv)
    assert np.abs(fd - hrt.gq[e]).max() < 1e-7 * np.abs(hrt.gq[e]).max()


# ------------------------------------------------------------------- manufactured solution
X, Y = sy.symbols("x y")
PHI = 1 + sy.sin(sy.pi * X) * sy.sin(sy.pi * Y) + X * Y / 2
E11 = sy.Rational(1, 3) + sy.Rational(1, 10) * sy.sin(sy.pi * X) * sy.cos(sy.pi * Y)
E22 = sy.Rational(2, 3) - E11
E12 = sy.Rational(1, 20) * X * Y
ST, SA = 2.0, 0.3
_EPHI = [[E11 * PHI, E12 * PHI], [E12 * PHI, E22 * PHI]]
JX = -(sy.diff(_EPHI[0][0], X) + sy.diff(_EPHI[0][1], Y)) / ST      # first moment, Q1 = 0
JY = -(sy.diff(_EPHI[1][0], X) + sy.diff(_EPHI[1][1], Y)) / ST
Q0 = sy.diff(JX, X) + sy.diff(JY, Y) + SA * PHI                     # zeroth moment
_F = {k: sy.lambdify((X, Y), v, "numpy") for k, v in
      dict(phi=PHI, E11=E11, E12=E12, E22=E22, Jx=JX, Jy=JY, Q0=Q0).items()}


def _f(k, x, y):
    return np.broadcast_to(_F[k](x, y), np.shape(x)).astype(float)


def _tensor(x, y):
    a, b, c = _f("E11", x, y), _f("E12", x, y), _f("E22", x, y)
    return np.stack([np.stack([a, b], -1), np.stack([b, c], -1)], -2)


def mms_data(disc, Eb_value=0.5):
    """VEF data of the manufactured solution: E at the volume and face points, E_b and the
    J_in that makes the Miften-Larsen condition J.n = E_b phi + 2 J_in exact, Q0."""
    g = disc.mesh
    Eq = _tensor(g.xq[..., 0], g.xq[..., 1])
    Ef = _tensor(g.xf[..., 0], g.xf[..., 1])
    Eb = np.full((g.nbf, disc.nq), Eb_value)
    Jin = np.zeros((g.nbf, disc.nq))
    for bf, (e, f) in enumerate(g.boundary_faces()):
        xb, yb = g.xf[e, f, :, 0], g.xf[e, f, :, 1]
        un = g.nds[e, f] / np.linalg.norm(g.nds[e, f], axis=1)[:, None]
        Jn = _f("Jx", xb, yb) * un[:, 0] + _f("Jy", xb, yb) * un[:, 1]
        Jin[bf] = (Jn - Eb_value * _f("phi", xb, yb)) / 2.0
    return Eq, Ef, Eb, Jin, _f("Q0", g.xq[..., 0], g.xq[..., 1])


def _errors(disc, hrt, sol):
    g = disc.mesh
    x, y = g.xq[..., 0], g.xq[..., 1]
    w = g.wq * g.J
    phiq = np.einsum("qj,ej->eq", disc.B, sol["phi"])
    Jq = hrt.current_at_points(sol["J"])
    ephi = np.sqrt(np.sum(w * (phiq - _f("phi", x, y)) ** 2))
    eJ = np.sqrt(np.sum(w * ((Jq[..., 0] - _f("Jx", x, y)) ** 2 + (Jq[..., 1] - _f("Jy", x, y)) ** 2)))
    return ephi, eJ


@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_solution_converges_at_order_p_plus_one(p):
    hs, ephi, eJ = [], [], []
    for nx in (4, 8, 16):
        disc = Discretization(nx, nx, 3, 0.05, p)
        hrt = HRT(disc)
        Eq, Ef, Eb, Jin, Q0q = mms_data(disc)
        E = disc.mesh.E
        sol = hrt.solve(np.full(E, ST), np.full(E, ST - SA), Eq, Ef, Eb, Jin, Q0q)
        a, b = _errors(disc, hrt, sol)
        hs.append(1.0 / nx)
        ephi.append(a)
        eJ.append(b)
    order = lambda e: np.polyfit(np.log(hs), np.log(e), 1)[0]
    assert order(ephi) > p + 1 - 0.15, ephi
    assert order(eJ) > p + 1 - 0.15, eJ


def _random_vef_data(disc, seed):
    """Non-constant VEF data from a positive random angular flux's moments."""
    g = disc.mesh
    rng = np.random.default_rng(seed)
    phi = rng.uniform(1.0, 2.0, (g.E, disc.n))
    P = np.stack([rng.uniform(0.25, 0.45, (g.E, disc.n)) * phi, rng.uniform(-0.05, 0.05, (g.E, disc.n)) * phi,
                  rng.uniform(0.25, 0.45, (g.E, disc.n)) * phi])
    return phi, P, rng


@pytest.mark.parametrize("p", [1, 2])
def test_elimination_equals_the_global_saddle_point_solve(p):
    disc = Discretization(4, 5, 3, 0.08, p)
    hrt = HRT(disc)
    g = disc.mesh
    phi, P, rng = _random_vef_data(disc, 9 + p)
    Eq, Ef = hrt.eddington_data(phi, P)
    Eb = rng.uniform(0.45, 0.55, (g.nbf, disc.nq))
    Jin = -rng.uniform(0.0, 0.3, (g.nbf, disc.nq))
    Q0q = rng.uniform(0.5, 1.5, (g.E, disc.nq ** 2))
    Q1q = rng.uniform(-0.2, 0.2, (g.E, disc.nq ** 2, 2))
    st = rng.uniform(0.5, 5.0, g.E)
    ss = rng.uniform(0.3, 0.95, g.E) * st
    a = hrt.solve(st, ss, Eq, Ef, Eb, Jin, Q0q, Q1q)
    b = hrt.solve_full(st, ss, Eq, Ef, Eb, Jin, Q0q, Q1q)
    for k in ("phi", "J", "lam"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-11 * np.abs(b[k]).max())


def test_block_inverse_equals_the_schur_complement_formulas():
    disc = Discretization(3, 3, 3, 0.08, 2)
    hrt = HRT(disc)
    g = disc.mesh
    phi, P, rng = _random_vef_data(disc, 4)
    Eq, Ef = hrt.eddington_data(phi, P)
    Eb = np.full((g.nbf, disc.nq), 0.5)
    Jin = np.zeros((g.nbf, disc.nq))
    st = np.full(g.E, 3.0)
    ss = np.full(g.E, 2.5)
    nJ = hrt.nJ
    for e in (0, 4):
        L, C1, C2, gv, fv = hrt.element(e, st, st - ss, Eq, Ef, Eb, Jin, np.ones((g.E, disc.nq ** 2)))
        A, G, D, Ma = L[:nJ, :nJ], L[:nJ, nJ:], L[nJ:, :nJ], L[nJ:, nJ:]
        Ai = np.linalg.inv(A)
        Si = np.linalg.inv(Ma - D @ Ai @ G)
        W = Ai @ (np.eye(nJ) + G @ Si @ D @ Ai)
        Li = np.linalg.inv(L)
        np.testing.assert_allclose(Li[:nJ, :nJ], W, atol=1e-9 * np.abs(W).max())
        np.testing.assert_allclose(Li[:nJ, nJ:], -Ai @ G @ Si, atol=1e-9 * np.abs(W).max())
        np.testing.assert_allclose(Li[nJ:, :nJ], -Si @ D @ Ai, atol=1e-9 * np.abs(Si).max())
        np.testing.assert_allclose(Li[nJ:, nJ:], Si, atol=1e-9 * np.abs(Si).max())


def test_thick_diffusion_limit_is_the_rt_diffusion_discretisation():
    disc = Discretization(4, 4, 3, 0.08, 2)
    hrt = HRT(disc)
    g = disc.mesh
    third = np.eye(2) / 3.0
    Eq = np.broadcast_to(third, (g.E, disc.nq ** 2, 2, 2)).copy()
    Ef = np.broadcast_to(third, (g.E, 4, disc.nq, 2, 2)).copy()
    Eb = np.full((g.nbf, disc.nq), 0.5)
    Jin = np.zeros((g.nbf, disc.nq))
    st = np.full(g.E, 2.0)
    ss = np.full(g.E, 1.5)
    nJ = hrt.nJ
    for e in range(g.E):
        L, C1, C2, _, _ = hrt.element(e, st, st - ss, Eq, Ef, Eb, Jin, np.ones((g.E, disc.nq ** 2)))
        G, D = L[:nJ, nJ:], L[nJ:, :nJ]
        np.testing.assert_allclose(G, -D.T / 3.0, atol=1e-12 * np.abs(D).max())
        np.testing.assert_allclose(C2, C1.T / 3.0, atol=1e-12 * np.abs(C1).max())
    H = hrt.solve(st, ss, Eq, Ef, Eb, Jin, np.ones((g.E, disc.nq ** 2)))["H"].toarray()
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() > 0.0
