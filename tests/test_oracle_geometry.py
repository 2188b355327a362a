"""Pins for the oracle's mesh and geometric factors."""
import numpy as np
import pytest

from oracle.mesh import Mesh, OPPOSITE


def test_straight_mesh_jacobian_and_normals():
    g = Mesh(4, 3, 1, 0.0, 3)
    np.testing.assert_allclose(g.J, 1.0 / 12.0, rtol=1e-14)
    # bottom face: n ds = (0, -1) * h_x ; right face: (1, 0) * h_y
    np.testing.assert_allclose(g.nds[:, 0], np.broadcast_to([0.0, -0.25], g.nds[:, 0].shape), atol=1e-15)
    np.testing.assert_allclose(g.nds[:, 1], np.broadcast_to([1.0 / 3.0, 0.0], g.nds[:, 1].shape), atol=1e-15)


@pytest.mark.parametrize("m,nq", [(1, 3), (2, 4), (3, 4), (3, 5)])
def test_curved_mesh_area_and_closed_boundary(m, nq):
    g = Mesh(5, 4, m, 0.05, nq)
    area = (g.wq * g.J).sum(axis=1)
    assert np.all(g.J > 0)
    np.testing.assert_allclose(area.sum(), 1.0, rtol=1e-13)     # boundary of [0,1]^2 is fixed
    # closed curve: sum over faces of int n ds = 0 per element
    closed = np.einsum("k,efkd->ed", g.wf, g.nds)
    np.testing.assert_allclose(closed, 0.0, atol=1e-14)
    # divergence theorem: area = (1/2) oint x . n ds
    half = 0.5 * np.einsum("k,efkd,efkd->e", g.wf, g.xf, g.nds)
    np.testing.assert_allclose(half, area, rtol=1e-12)


def test_shared_faces_match():
    g = Mesh(4, 4, 3, 0.05, 4)
    for e in range(g.E):
        for f in range(4):
            nb = g.nb[e, f]
            if nb < 0:
                continue
            of = g.nbface[e, f]
            assert of == OPPOSITE[f]
            np.testing.assert_allclose(g.xf[e, f], g.xf[nb, of], atol=1e-15)
            np.testing.assert_allclose(g.nds[e, f], -g.nds[nb, of], atol=1e-15)


def test_boundary_face_numbering():
    g = Mesh(3, 2, 1, 0.0, 2)
    bfs = g.boundary_faces()
    assert bfs[0] == (0, 0) and bfs[2] == (2, 0)            # bottom row
    assert bfs[3] == (2, 1) and bfs[4] == (5, 1)            # right column
    assert bfs[5] == (3, 2) and bfs[7] == (5, 2)            # top row
    assert bfs[8] == (0, 3) and bfs[9] == (3, 3)            # left column


def test_sine_map_control_points():
    g = Mesh(4, 4, 3, 0.05, 4)
    # element (1, 1) vertex (0.5, 0.5) is not moved (sin(pi) = 0); (0.25,0.25) moves by alpha
    c = g.ctrl[1 * 4 + 1]
    np.testing.assert_allclose(c[0], [0.25 + 0.05, 0.25 + 0.05], atol=1e-15)
    np.testing.assert_allclose(c[15], [0.5, 0.5], atol=1e-15)
