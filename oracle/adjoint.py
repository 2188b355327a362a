"""Adjoint transport solves and cross-section gradients (test infrastructure only).

The paper has no adjoint; this follows from its transport equation.  For a
functional R = sum_{e,j} g_{e,j} phi_{e,j} of the scalar flux of one transport
inversion with fixed scattering flux phi_in,
    phi = sum_d w_d psi_d,  L_d psi_d = b_d,
the adjoint directions solve L_d^T lambda_d = w_d g, and
    R = sum_d lambda_d^T b_d,
    dR/dsigma_t,e = - sum_d lambda_{d,e}^T M_e psi_{d,e}     (dL_d/dsigma_t,e = M_e block)
    dR/dsigma_s,e =   sum_d lambda_{d,e}^T M_e phi_in,e / (4 pi)
with M_e the element mass matrix (int_K l_i l_j dx).

region_weights builds g for R = int chi_region phi dx, with the indicator chi
evaluated at the volume quadrature points (physical coordinates).
"""
import numpy as np
import scipy.sparse.linalg as spla


def region_weights(disc, lo=(0.6, 0.6), hi=(0.8, 0.8)):
    """g [E][n] with R = sum g * phi = int_{[lo,hi]} phi dx (quadrature)."""
    g = disc.mesh
    x, y = g.xq[..., 0], g.xq[..., 1]
    chi = ((x >= lo[0]) & (x <= hi[0]) & (y >= lo[1]) & (y <= hi[1])).astype(np.float64)
    return np.einsum("q,eq,eq,qj->ej", g.wq, g.J, chi, disc.B)


def adjoint(disc, omega, weights, sigma_t, sigma_s, psi, g, phi_in=None):
    """Returns (lambda [D][E][n], dR/dsigma_t [E], dR/dsigma_s [E])."""
    sigma_t = np.asarray(sigma_t, np.float64)
    w = np.asarray(weights, np.float64)
    D = len(w)
    E, n = disc.mesh.E, disc.n
    lam = np.zeros((D, E, n))
    dst = np.zeros(E)
    dss = np.zeros(E)
    for d in range(D):
        L, _ = disc.operator(omega[d], sigma_t)
        lam[d] = spla.spsolve(L.T.tocsc(), (w[d] * g).ravel()).reshape(E, n)
        dst -= np.einsum("ei,eij,ej->e", lam[d], disc.M, psi[d])
        if phi_in is not None:
            dss += np.einsum("ei,eij,ej->e", lam[d], disc.M, phi_in) / (4.0 * np.pi)
    return lam, dst, dss
