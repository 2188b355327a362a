"""Pins for the 1D rules and Lagrange bases of the oracle."""
import numpy as np
import pytest

from oracle.basis import gll_points, gauss_legendre, lagrange, lagrange_deriv, tensor_values


@pytest.mark.parametrize("n", range(1, 8))
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        np.testing.assert_allclose((w * x ** k).sum(), 1.0 / (k + 1), rtol=1e-14)
    assert abs((w * x ** (2 * n)).sum() - 1.0 / (2 * n + 1)) > 1e-12


def test_gll_known_points():
    np.testing.assert_allclose(gll_points(1), [0, 1])
    np.testing.assert_allclose(gll_points(2), [0, 0.5, 1])
    np.testing.assert_allclose(gll_points(3), [0, (1 - 1 / np.sqrt(5)) / 2, (1 + 1 / np.sqrt(5)) / 2, 1],
                               rtol=1e-15)
    np.testing.assert_allclose(gll_points(4), [0, (1 - np.sqrt(3 / 7)) / 2, 0.5, (1 + np.sqrt(3 / 7)) / 2, 1],
                               rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_lagrange_cardinal_and_derivative(q):
    nodes = gll_points(q)
    np.testing.assert_allclose(lagrange(nodes, nodes), np.eye(q + 1), atol=1e-14)
    x = np.linspace(-0.1, 1.1, 13)
    np.testing.assert_allclose(lagrange(nodes, x).sum(axis=1), 1.0, rtol=1e-13)
    np.testing.assert_allclose(lagrange_deriv(nodes, x).sum(axis=1), 0.0, atol=1e-11)
    h = 1e-6
    fd = (lagrange(nodes, x + h) - lagrange(nodes, x - h)) / (2 * h)
    np.testing.assert_allclose(lagrange_deriv(nodes, x), fd, atol=1e-6)
    # reproduces polynomials of degree q: interpolate x^q and differentiate
    f = nodes ** q
    np.testing.assert_allclose(lagrange(nodes, x) @ f, x ** q, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(lagrange_deriv(nodes, x) @ f, q * x ** (q - 1), rtol=1e-10, atol=1e-11)


def test_tensor_ordering():
    nodes = gll_points(2)
    V, Dx, Dy = tensor_values(nodes, np.array([0.0, 1.0, 0.5]), np.array([0.0, 0.0, 1.0]))
    # dof a + 3 b: point (1, 0) is node a=2, b=0 -> dof 2; point (0.5, 1) is a=1, b=2 -> dof 7
    assert V[1, 2] == pytest.approx(1.0) and V[2, 7] == pytest.approx(1.0)
    # f(x, y) = x * y^2 at the nodes: d/dx = y^2, d/dy = 2 x y
    xs, ys = np.meshgrid(nodes, nodes)   # [b][a]
    f = (xs * ys ** 2).ravel()
    assert Dx[2] @ f == pytest.approx(1.0) and Dy[2] @ f == pytest.approx(1.0)
