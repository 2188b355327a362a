"""Source iteration and the VEF fixed-point iteration (test infrastructure only).

Paper Sec. "VEF Algorithm": the transport equation is inverted for a given
scattering source, and the iteration repeats until the scalar flux stops changing.
Here the plain (unaccelerated) form: phi^0 given (default 0), then
    psi^{k} = L^{-1} b(phi^k),  phi^{k+1} = sum_d w_d psi_d^{k},
and the stopping quantity is the max norm of successive differences, the criterion
the paper's nonlinear solver uses (max norm of the difference between iterates).
"""
import numpy as np

from .transport import sweep


def source_iterate(disc, omega, weights, sigma_t, sigma_s, source=None, inflow=None,
                   K=10, phi0=None):
    """Run K source iterations; returns (phi^K [E][n], psi of the last sweep,
    dphi_inf [K] with dphi_inf[k] = max |phi^{k+1} - phi^k|)."""
    phi = np.zeros((disc.mesh.E, disc.n)) if phi0 is None else np.array(phi0, np.float64)
    w = np.asarray(weights, np.float64)
    dinf = np.zeros(K)
    psi = None
    for k in range(K):
        psi = sweep(disc, omega, weights, sigma_t, sigma_s, phi_in=phi, source=source,
                    inflow=inflow)
        new = np.einsum("d,den->en", w, psi)
        dinf[k] = np.max(np.abs(new - phi))
        phi = new
    return phi, psi, dinf


def vef_iterate(disc, omega, weights, sigma_t, sigma_s, source, inflow=None, K=50, tol=1e-6, phi0=None):
    """VEF fixed-point iteration (paper Sec. "VEF Algorithm"): from phi^0 (default 0),
    1) invert the transport equation with the scattering source sigma_s phi^k / (4 pi) + q,
    2) form the Eddington tensor, the boundary factor and J_in from its angular flux,
    3) solve the hybridized RT VEF equations (oracle.hrt) with Q0 = 4 pi q, Q1 = 0 (an
    isotropic source q [E][n] per steradian), and take their scalar flux as phi^{k+1};
    stop when max |phi^{k+1} - phi^k| <= tol (the paper's criterion: the max norm of the
    difference of successive iterates) or after K iterations.
    Returns (phi [E][n], J [E][nJ], iterations, history of the max-norm changes)."""
    from .moments import angular_moments, boundary_closures
    from .hrt import HRT
    hrt = HRT(disc)
    g = disc.mesh
    phi = np.zeros((g.E, disc.n)) if phi0 is None else np.array(phi0, np.float64)
    Q0q = np.einsum("qj,ej->eq", disc.B, 4.0 * np.pi * np.asarray(source, np.float64))
    hist = []
    J = None
    for k in range(K):
        psi = sweep(disc, omega, weights, sigma_t, sigma_s, phi_in=phi, source=source, inflow=inflow)
        phi_tr, _, P = angular_moments(psi, omega, weights)
        Eb, Jin, _ = boundary_closures(disc, psi, omega, weights, inflow)
        Eq, Ef = hrt.eddington_data(phi_tr, P)
        sol = hrt.solve(sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q)
        change = np.max(np.abs(sol["phi"] - phi))
        hist.append(change)
        phi, J = sol["phi"], sol["J"]
        if change <= tol:
            return phi, J, k + 1, np.array(hist)
    return phi, J, K, np.array(hist)
