"""Problem builders shared by the tests (manufactured solutions, closed forms)."""
import numpy as np

from oracle import mms
from oracle.mesh import map_jacobian
from oracle.transport import Discretization


def nodal_xy(disc):
    """Physical coordinates of the DG nodes [E][n] (x, y)."""
    p = disc.p
    nd = disc.nodes
    px, py = np.tile(nd, p + 1), np.repeat(nd, p + 1)
    xn, _ = map_jacobian(disc.mesh.ctrl, disc.mesh.m, px, py)
    return xn[..., 0], xn[..., 1]


def boundary_values(disc, omega, fn):
    """inflow [D][N_bf][nq] = fn(x, y, Omega_d) at the boundary face points."""
    g = disc.mesh
    D = len(omega)
    out = np.zeros((D, g.nbf, disc.nq))
    for bf, (e, f) in enumerate(g.boundary_faces()):
        for d in range(D):
            out[d, bf] = fn(g.xf[e, f, :, 0], g.xf[e, f, :, 1], omega[d])
    return out


def l2_error_psi(disc, psi, omega, weights, fn):
    """sqrt(sum_d w_d int (psi_h - psi)^2 dx) with psi exact given by fn."""
    g = disc.mesh
    err = 0.0
    for d in range(len(weights)):
        ex = fn(g.xq[..., 0], g.xq[..., 1], omega[d])
        ap = np.einsum("qj,ej->eq", disc.B, psi[d])
        err += weights[d] * np.sum(g.wq * g.J * (ex - ap) ** 2)
    return np.sqrt(err)


def mms_problem(nx, m, alpha, p, omega, sigma_t=1.0):
    """Pure-absorber-plus-source MMS setup (sigma_s = 0): returns disc and the
    sweep inputs reproducing the paper's manufactured psi."""
    disc = Discretization(nx, nx, m, alpha, p)
    E = disc.mesh.E
    xn, yn = nodal_xy(disc)
    st = np.full(E, sigma_t)
    ss = np.zeros(E)
    src = np.stack([mms.source(xn, yn, omega[d], sigma_t, 0.0, 0.0) for d in range(len(omega))])
    inflow = boundary_values(disc, omega, mms.psi)
    return disc, st, ss, src, inflow


def fit_order(hs, errs):
    """Least-squares slope of log E = log C + p log h (paper's order fit)."""
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]
