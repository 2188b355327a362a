"""Pins for the LQn quadrature inputs (S_N angular model of the transport section)."""
import numpy as np
import pytest

from vef_inputs import level_symmetric, LQN_ORDERS

FOUR_PI = 4.0 * np.pi


@pytest.mark.parametrize("N", LQN_ORDERS)
def test_count_and_even_moments(N):
    om, w = level_symmetric(N)
    mu, eta = om[:, 0], om[:, 1]
    assert len(w) == N * (N + 2) // 2
    assert np.all(w > 0)
    np.testing.assert_allclose(np.sum(mu ** 2 + eta ** 2 <= 1.0), len(w))
    # exact sphere integrals of 1, mu^2, mu^4, mu^2 eta^2 (over 4 pi)
    np.testing.assert_allclose(w.sum(), FOUR_PI, rtol=1e-15)
    np.testing.assert_allclose((w * mu ** 2).sum(), FOUR_PI / 3, rtol=1e-14)
    np.testing.assert_allclose((w * eta ** 2).sum(), FOUR_PI / 3, rtol=1e-14)
    np.testing.assert_allclose((w * mu ** 4).sum(), FOUR_PI / 5, rtol=1e-14)
    np.testing.assert_allclose((w * mu ** 2 * eta ** 2).sum(), FOUR_PI / 15, rtol=1e-14)
    # odd moments vanish by symmetry
    for f in (mu, eta, mu * eta, mu ** 3, mu * eta ** 2):
        assert abs((w * f).sum()) < 1e-14


@pytest.mark.parametrize("N", [6, 8, 12, 16])
def test_higher_pure_moments(N):
    """sum w mu^(2k) = 4 pi/(2k+1) for k < N/2 (the LQn construction)."""
    om, w = level_symmetric(N)
    for k in range(N // 2):
        np.testing.assert_allclose((w * om[:, 0] ** (2 * k)).sum(), FOUR_PI / (2 * k + 1), rtol=1e-13)


def test_published_class_weights():
    """LQ8 / LQ12 class weights (published 7-digit tables) come out of the moment
    conditions; the point weight is pi times the per-octant class weight."""
    om, w = level_symmetric(8)
    got = sorted(set(np.round(w / np.pi, 7)))
    assert got == sorted([0.1209877, 0.0907407, 0.0925926])
    om, w = level_symmetric(12)
    got = sorted(set(np.round(w / np.pi, 7)))
    assert got == sorted([0.0707626, 0.0558811, 0.0373377, 0.0502819, 0.0258513]) or \
        np.allclose(got, sorted([0.0707626, 0.0558811, 0.0373377, 0.0502819, 0.0258513]), atol=2e-7)


def test_s4_mu1_is_root_of_fourth_moment():
    om, _ = level_symmetric(4)
    a = np.min(np.abs(om[:, 0])) ** 2
    assert abs(6 * a * a - 4 * a + 0.4) < 1e-15
    np.testing.assert_allclose(np.sqrt(a), 0.3500212, atol=1e-7)
