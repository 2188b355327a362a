"""Structured curved quadrilateral mesh and geometric factors (test infrastructure only).

Mesh (paper Sec. "Description of the Mesh" and Sec. "Solver Performance on Curved
Meshes"): nx x ny elements on [0,1]^2, element e = j*nx + i.  Each element is the
image of the reference square [0,1]^2 under the Q_m map
    x(xi) = sum_c x_{e,c} l_c(xi)
through (m+1)^2 control points at the tensor Gauss-Lobatto points, local index
c = a + (m+1) b.  Control points sit at X = (i + xi_a)/nx, Y = (j + xi_b)/ny and
are moved by the sine distortion
    (X, Y) -> (X, Y) + alpha * sin(2 pi X) sin(2 pi Y) * (1, 1),
which vanishes on the boundary of [0,1]^2.  Shared control points coincide, so the
mesh is continuous.

Geometry (paper Sec. "Integration Transformations"): F = dx/dxi, J = det F,
grad = F^{-T} grad_ref, integrals in reference space with J dxi.  On a face with
reference outward normal n_ref, the physical outward normal times the length
element is n ds = adj(F)^T n_ref ds_ref (equivalently, the tangent rotated
clockwise: the tangent is the counter-clockwise rotation of the normal).

Faces: 0 bottom (eta = 0), 1 right (xi = 1), 2 top (eta = 1), 3 left (xi = 0).
Face points are ordered by increasing reference coordinate along the face, so a
point has the same index k seen from either neighbour.
Boundary faces: bottom row i = 0..nx-1, right column j = 0..ny-1, top row
i = 0..nx-1, left column j = 0..ny-1, in that order (N_bf = 2 nx + 2 ny).
"""
import numpy as np

from .basis import gll_points, gauss_legendre, lagrange, lagrange_deriv, lagrange_deriv2

FACE_NREF = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
OPPOSITE = (2, 3, 0, 1)


def control_points(nx, ny, m, alpha):
    """Control points [E][(m+1)^2][2] of the sine-distorted Q_m mesh."""
    g = gll_points(m)
    E = nx * ny
    ctrl = np.zeros((E, (m + 1) ** 2, 2))
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            for b in range(m + 1):
                for a in range(m + 1):
                    X = (i + g[a]) / nx
                    Y = (j + g[b]) / ny
                    d = alpha * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
                    ctrl[e, a + (m + 1) * b] = (X + d, Y + d)
    return ctrl


def neighbor(nx, ny, e, f):
    """(neighbour element, its face) across face f of element e, or (-1, boundary face)."""
    i, j = e % nx, e // nx
    if f == 0:
        return ((j - 1) * nx + i, 2) if j > 0 else (-1, i)
    if f == 1:
        return (j * nx + i + 1, 3) if i < nx - 1 else (-1, nx + j)
    if f == 2:
        return ((j + 1) * nx + i, 0) if j < ny - 1 else (-1, nx + ny + i)
    return (j * nx + i - 1, 1) if i > 0 else (-1, 2 * nx + ny + j)


def face_ref_points(f, s):
    """Reference coordinates of the points s (along the face) on face f."""
    s = np.asarray(s, dtype=np.float64)
    z, o = np.zeros_like(s), np.ones_like(s)
    return [(s, z), (o, s), (s, o), (z, s)][f]


def map_jacobian(ctrl, m, px, py):
    """Physical points x [E][k][2] and Jacobians F [E][k][2][2] at reference points."""
    g = gll_points(m)
    vx, vy = lagrange(g, px), lagrange(g, py)
    dx, dy = lagrange_deriv(g, px), lagrange_deriv(g, py)
    q = m + 1
    V = np.einsum("ka,kb->kba", vx, vy).reshape(len(px), q * q)
    Dxi = np.einsum("ka,kb->kba", dx, vy).reshape(len(px), q * q)
    Deta = np.einsum("ka,kb->kba", vx, dy).reshape(len(px), q * q)
    x = np.einsum("kc,ecd->ekd", V, ctrl)
    F = np.zeros(x.shape[:2] + (2, 2))
    F[..., :, 0] = np.einsum("kc,ecd->ekd", Dxi, ctrl)   # dx/dxi, dy/dxi
    F[..., :, 1] = np.einsum("kc,ecd->ekd", Deta, ctrl)  # dx/deta, dy/deta
    return x, F


def map_hessian(ctrl, m, px, py):
    """Second derivatives H [E][k][i][j][l] = d^2 x_i / (dxi_j dxi_l) of the Q_m map at
    reference points (xi_0 = xi, xi_1 = eta); symmetric in j, l."""
    g = gll_points(m)
    vx, vy = lagrange(g, px), lagrange(g, py)
    dx, dy = lagrange_deriv(g, px), lagrange_deriv(g, py)
    sx, sy = lagrange_deriv2(g, px), lagrange_deriv2(g, py)
    q = m + 1
    tab = lambda A, B: np.einsum("ka,kb->kba", A, B).reshape(len(px), q * q)
    Dxx, Dxy, Dyy = tab(sx, vy), tab(dx, dy), tab(vx, sy)
    H = np.zeros((ctrl.shape[0], len(px), 2, 2, 2))
    for (j, l), T in (((0, 0), Dxx), ((0, 1), Dxy), ((1, 1), Dyy)):
        H[:, :, :, j, l] = np.einsum("kc,ecd->ekd", T, ctrl)
    H[:, :, :, 1, 0] = H[:, :, :, 0, 1]
    return H


def adjugate(F):
    """adj(F) = det(F) F^{-1} for 2x2 matrices (last two axes)."""
    A = np.empty_like(F)
    A[..., 0, 0] = F[..., 1, 1]
    A[..., 0, 1] = -F[..., 0, 1]
    A[..., 1, 0] = -F[..., 1, 0]
    A[..., 1, 1] = F[..., 0, 0]
    return A


class Mesh:
    """Geometry of the structured Q_m mesh evaluated at the DG quadrature points.

    Attributes (FP64):
      ctrl [E][(m+1)^2][2]; xq [E][nq^2][2] volume points (point k1 + nq k2);
      J [E][nq^2]; adjF [E][nq^2][2][2]; wq [nq^2] reference weights;
      xf [E][4][nq][2] face points; nds [E][4][nq][2] = adj(F)^T n_ref; wf [nq].
    """

    def __init__(self, nx, ny, m, alpha, nq, ctrl=None):
        self.nx, self.ny, self.m, self.alpha, self.nq = nx, ny, m, alpha, nq
        self.E = nx * ny
        self.nbf = 2 * nx + 2 * ny
        self.ctrl = control_points(nx, ny, m, alpha) if ctrl is None else np.asarray(ctrl, np.float64)
        s, w = gauss_legendre(nq)
        self.s1d, self.w1d = s, w
        px = np.tile(s, nq)
        py = np.repeat(s, nq)
        self.ref_vol = (px, py)
        self.wq = np.tile(w, nq) * np.repeat(w, nq)
        self.xq, F = map_jacobian(self.ctrl, m, px, py)
        self.J = F[..., 0, 0] * F[..., 1, 1] - F[..., 0, 1] * F[..., 1, 0]
        self.adjF = adjugate(F)
        self.wf = w
        self.xf = np.zeros((self.E, 4, nq, 2))
        self.nds = np.zeros((self.E, 4, nq, 2))
        for f in range(4):
            fx, fy = face_ref_points(f, s)
            xf, Ff = map_jacobian(self.ctrl, m, fx, fy)
            self.xf[:, f] = xf
            adjT = np.swapaxes(adjugate(Ff), -1, -2)
            self.nds[:, f] = np.einsum("ekij,j->eki", adjT, FACE_NREF[f])
        self.nb = np.zeros((self.E, 4), dtype=np.int64)
        self.nbface = np.zeros((self.E, 4), dtype=np.int64)
        for e in range(self.E):
            for f in range(4):
                self.nb[e, f], self.nbface[e, f] = neighbor(nx, ny, e, f)

    def boundary_faces(self):
        """List of (element, face) for boundary face index 0..N_bf-1."""
        out = [None] * self.nbf
        for e in range(self.E):
            for f in range(4):
                if self.nb[e, f] < 0:
                    out[self.nbface[e, f]] = (e, f)
        return out
