"""The Taylor-Green advected mesh (input data for the user-control-point path)."""
import numpy as np

from vef_inputs import taylor_green_control_points
from oracle.mesh import control_points
from oracle.transport import Discretization


def test_zero_time_is_the_orthogonal_mesh():
    np.testing.assert_array_equal(taylor_green_control_points(5, 4, 3, T=0.0, steps=1),
                                  control_points(5, 4, 3, 0.0))


def test_advected_mesh_is_valid_continuous_and_keeps_its_area():
    nx, ny, m = 8, 6, 3
    c = taylor_green_control_points(nx, ny, m)
    q = m + 1
    # the normal velocity vanishes on x = 0 and on y = 0: control points there slide along
    # those sides and never leave them
    c0 = control_points(nx, ny, m, 0.0)
    on_x0 = np.isclose(c0[..., 0], 0.0)
    on_y0 = np.isclose(c0[..., 1], 0.0)
    assert np.all(c[on_x0][:, 0] == 0.0) and np.all(c[on_y0][:, 1] == 0.0)
    # neighbours share their face control points exactly (a continuous mesh)
    for j in range(ny):
        for i in range(nx - 1):
            e = j * nx + i
            right = [q - 1 + q * b for b in range(q)]
            left = [q * b for b in range(q)]
            np.testing.assert_array_equal(c[e, right], c[e + 1, left])
    disc = Discretization(nx, ny, m, 0.0, 2, ctrl=c)
    assert disc.mesh.J.min() > 0.0
    # the Taylor-Green velocity is divergence-free: the advected domain keeps area 1 up to
    # the forward Euler and Q3 interpolation errors
    assert abs(np.sum(disc.mesh.wq * disc.mesh.J) - 1.0) < 5e-3
    # and it is strongly distorted (the x = 1 side moves out to x ~ 1.9)
    assert c[..., 0].max() > 1.5
