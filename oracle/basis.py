"""1D quadrature rules and Lagrange bases on [0, 1] (test infrastructure only).

* Gauss-Lobatto (GLL) points: the mesh control-point nodes (paper Sec. "Description
  of the Mesh": the m+1 Gauss-Lobatto points of [0,1]) and, here, the nodes of the
  DG basis of Y_p (closed points are allowed for DG, paper Sec. "Discontinuous
  Galerkin").
* Gauss-Legendre (GL) rule with n points: volume and face quadrature.
* Lagrange interpolating polynomials and their derivatives, by the product formula.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_points(m):
    """The m+1 Gauss-Lobatto points on [0,1]: 0, 1 and the roots of P_m' mapped."""
    if m < 1:
        raise ValueError("order must be >= 1")
    if m == 1:
        t = np.array([-1.0, 1.0])
    else:
        inner = npleg.Legendre.basis(m).deriv().roots()
        t = np.concatenate(([-1.0], np.sort(inner.real), [1.0]))
    x = 0.5 * (t + 1.0)
    x[0], x[-1] = 0.0, 1.0
    return x


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0,1]: (points, weights), weights sum to 1."""
    t, w = npleg.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange(nodes, x):
    """Values V[k, a] = l_a(x_k) of the Lagrange polynomials through `nodes`."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    V = np.ones((len(x), len(nodes)))
    for a in range(len(nodes)):
        for c in range(len(nodes)):
            if c != a:
                V[:, a] *= (x - nodes[c]) / (nodes[a] - nodes[c])
    return V


def lagrange_deriv(nodes, x):
    """Derivatives D[k, a] = l_a'(x_k): sum over the dropped factor of the product."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    q = len(nodes)
    D = np.zeros((len(x), q))
    for a in range(q):
        for k in range(q):
            if k == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[k]))
            for c in range(q):
                if c != a and c != k:
                    term *= (x - nodes[c]) / (nodes[a] - nodes[c])
            D[:, a] += term
    return D


def lagrange_deriv2(nodes, x):
    """Second derivatives S[k, a] = l_a''(x_k): sum over ordered pairs of dropped factors."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    q = len(nodes)
    S = np.zeros((len(x), q))
    for a in range(q):
        for k in range(q):
            if k == a:
                continue
            for l in range(q):
                if l == a or l == k:
                    continue
                term = np.full(len(x), 1.0 / ((nodes[a] - nodes[k]) * (nodes[a] - nodes[l])))
                for c in range(q):
                    if c != a and c != k and c != l:
                        term *= (x - nodes[c]) / (nodes[a] - nodes[c])
                S[:, a] += term
    return S


def tensor_values(nodes, px, py):
    """2D tensor basis l_{a}(x) l_{b}(y) at points (px[k], py[k]); dof a + (p+1) b.
    Returns (V, dV/dxi, dV/deta), each [npts][(p+1)^2]."""
    vx, vy = lagrange(nodes, px), lagrange(nodes, py)
    dx, dy = lagrange_deriv(nodes, px), lagrange_deriv(nodes, py)
    q = len(nodes)
    V = np.einsum("ka,kb->kba", vx, vy).reshape(len(px), q * q)
    Dxi = np.einsum("ka,kb->kba", dx, vy).reshape(len(px), q * q)
    Deta = np.einsum("ka,kb->kba", vx, dy).reshape(len(px), q * q)
    return V, Dxi, Deta
