"""Source iteration (test infrastructure only).

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
