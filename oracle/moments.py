"""Angular moments and VEF closures (test infrastructure only).

Paper Eq. vef_disc: with S_N quadrature {w_d, Omega_d} and finite element
interpolation of psi_d in Y_p,
    E(x)   = sum_d w_d Omega_d (x) Omega_d psi_d(x) / sum_d w_d psi_d(x),
    E_b(x) = sum_d w_d |Omega_d . n| psi_d(x)  / sum_d w_d psi_d(x)     on the boundary.
The VEF data are ratios of DG functions (the remark after Eq. vef_disc): phi and
the second moment P = sum_d w_d Omega_d (x) Omega_d psi_d are DG functions with nodal
coefficients, and E is their ratio evaluated pointwise.  E_b uses the interior trace
and the unit outward normal.  The inflow partial current (paper, text after
Eq. mlbc) is J_in = sum_{Omega_d . n < 0} w_d (Omega_d . n) psi_bar_d.

Outputs: phi [E][n]; J [2][E][n]; P [3][E][n] as (xx, xy, yy); E [3][E][nq^2] at the
volume quadrature points; E_b, J_in [N_bf][nq] at boundary face points.
A denominator sum_d w_d psi_d <= 1e-300 makes E (or E_b) NaN there; `nonpositive`
reports whether that happened (the method assumes psi > 0).
"""
import numpy as np

DENOM_FLOOR = 1e-300


def angular_moments(psi, omega, weights):
    """phi, J, P as DG nodal coefficients (sums over directions of w_d psi_d ...)."""
    w = np.asarray(weights, np.float64)
    mu, eta = omega[:, 0], omega[:, 1]
    phi = np.einsum("d,den->en", w, psi)
    J = np.stack([np.einsum("d,den->en", w * mu, psi), np.einsum("d,den->en", w * eta, psi)])
    P = np.stack([np.einsum("d,den->en", w * mu * mu, psi),
                  np.einsum("d,den->en", w * mu * eta, psi),
                  np.einsum("d,den->en", w * eta * eta, psi)])
    return phi, J, P


def eddington(disc, phi, P):
    """E [3][E][nq^2] = P(x_q) / phi(x_q) at the volume quadrature points."""
    phiq = np.einsum("qj,ej->eq", disc.B, phi)
    Pq = np.einsum("qj,cej->ceq", disc.B, P)
    bad = phiq <= DENOM_FLOOR
    with np.errstate(divide="ignore", invalid="ignore"):
        E = Pq / phiq[None]
    E[:, bad] = np.nan
    return E, bool(bad.any())


def boundary_closures(disc, psi, omega, weights, inflow=None):
    """E_b and J_in [N_bf][nq] at the boundary face quadrature points."""
    g = disc.mesh
    w = np.asarray(weights, np.float64)
    Eb = np.zeros((g.nbf, disc.nq))
    Jin = np.zeros((g.nbf, disc.nq))
    bad = False
    for bf, (e, f) in enumerate(g.boundary_faces()):
        nds = g.nds[e, f]                                        # [nq][2]
        nhat = nds / np.linalg.norm(nds, axis=1)[:, None]
        on = np.einsum("kc,dc->dk", nhat, omega)                 # Omega_d . n  [D][nq]
        trace = np.einsum("ki,di->dk", disc.Bf[f], psi[:, e, :])  # psi_d at face points
        num = np.einsum("d,dk,dk->k", w, np.abs(on), trace)
        den = np.einsum("d,dk->k", w, trace)
        for k in range(disc.nq):
            if den[k] <= DENOM_FLOOR:
                Eb[bf, k] = np.nan
                bad = True
            else:
                Eb[bf, k] = num[k] / den[k]
        if inflow is not None:
            neg = np.where(on < 0.0, on, 0.0)
            Jin[bf] = np.einsum("d,dk,dk->k", w, neg, inflow[:, bf, :])
    return Eb, Jin, bad


def closures(disc, psi, omega, weights, inflow=None):
    """All outputs of the moment/closure pass as a dict."""
    phi, J, P = angular_moments(psi, omega, weights)
    E, bad1 = eddington(disc, phi, P)
    Eb, Jin, bad2 = boundary_closures(disc, psi, omega, weights, inflow)
    return dict(phi=phi, J=J, P=P, E=E, Eb=Eb, Jin=Jin, nonpositive=bad1 or bad2)
