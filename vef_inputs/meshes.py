"""Mesh control points given to the library as input data (no method arithmetic).

taylor_green_control_points builds the third-order curved mesh the paper uses for its
manufactured-solution study (Sec. "Method of Manufactured Solutions", Fig. tgmesh): the
Gauss-Lobatto control points of an orthogonal nx x ny mesh of [0,1]^2 are advected with the
Taylor-Green vortex velocity v = (sin x cos y, -cos x sin y) by forward Euler steps up to
the final time T (printed: T = 0.3 pi, 300 steps).  The velocity vanishes on x = 0 and
y = 0 but not on x = 1 or y = 1, so those two sides of the domain move with the mesh (the
domain is advected as printed).  Shared control points of neighbouring elements coincide,
so the mesh stays continuous.  Layout [E][(m+1)^2][2], element e = j nx + i, local control
point a + (m+1) b, as vef_mesh_create takes them.
"""
import numpy as np


def _gll(m):
    """m + 1 Gauss-Lobatto points on [0, 1] (Legendre derivative roots and the ends)."""
    if m == 1:
        return np.array([0.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(m).deriv().roots()
    return np.concatenate([[0.0], (np.sort(inner.real) + 1.0) / 2.0, [1.0]])


def taylor_green_control_points(nx, ny, m=3, T=0.3 * np.pi, steps=300):
    g = _gll(m)
    E, q = nx * ny, m + 1
    ctrl = np.zeros((E, q * q, 2))
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            for b in range(q):
                for a in range(q):
                    ctrl[e, a + q * b] = ((i + g[a]) / nx, (j + g[b]) / ny)
    dt = T / steps
    x, y = ctrl[..., 0].copy(), ctrl[..., 1].copy()
    for _ in range(steps):
        vx, vy = np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)
        x, y = x + dt * vx, y + dt * vy
    return np.stack([x, y], axis=-1)
