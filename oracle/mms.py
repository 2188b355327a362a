"""Manufactured solution of the paper's MMS section (test infrastructure only).

psi(x, Omega) = (1/(4 pi)) [alpha(x) + Omega . beta(x) + Omega (x) Omega : Theta(x)]
with delta = 1.25, zeta = 0.1, omega = 0.05 and
  alpha     = sin(pi x) sin(pi y) + delta
  beta_1    = beta_2 = s2(x) s2(y),          s2(t) = sin(2 pi (t + omega)/(1 + 2 omega))
  Theta_11  = s3(x) s3(y) / 2,  Theta_22 = s3(x) s3(y) / 4,
  Theta_12  = Theta_21 = s2(x) s2(y),         s3(t) = sin(3 pi (t + zeta)/(1 + 2 zeta))
Moments with exact angular integration:
  phi = alpha + tr(Theta)/3,  J = beta/3,
  P   = alpha/3 I + (1/15) [[3 Theta_11 + Theta_22, 2 Theta_12], [2 Theta_12, Theta_11 + 3 Theta_22]].
The off-diagonal of P is printed as Theta_12/15 in the paper; direct integration
(int mu^2 eta^2 dOmega / 4 pi = 1/15, Theta symmetric) gives 2 Theta_12/15, which is
used here.  In 2D, Omega = (mu, eta) is the x-y projection of the 3D direction.
"""
import numpy as np

DELTA, ZETA, OMEGA_MMS = 1.25, 0.1, 0.05


def _s(t, k, shift):
    a = k * np.pi / (1.0 + 2.0 * shift)
    return np.sin(a * (t + shift)), a * np.cos(a * (t + shift))


def fields(x, y):
    """alpha, beta (2,), Theta (2,2) and their x/y derivatives at points (x, y)."""
    sx, dsx = np.sin(np.pi * x), np.pi * np.cos(np.pi * x)
    sy, dsy = np.sin(np.pi * y), np.pi * np.cos(np.pi * y)
    s2x, d2x = _s(x, 2, OMEGA_MMS)
    s2y, d2y = _s(y, 2, OMEGA_MMS)
    s3x, d3x = _s(x, 3, ZETA)
    s3y, d3y = _s(y, 3, ZETA)
    alpha = sx * sy + DELTA
    da = (dsx * sy, sx * dsy)
    b = s2x * s2y
    db = (d2x * s2y, s2x * d2y)
    t3 = s3x * s3y
    dt3 = (d3x * s3y, s3x * d3y)
    beta = np.stack([b, b])
    dbeta = [np.stack([db[0], db[0]]), np.stack([db[1], db[1]])]
    Theta = np.stack([np.stack([0.5 * t3, b]), np.stack([b, 0.25 * t3])])
    dTheta = [np.stack([np.stack([0.5 * dt3[c], db[c]]), np.stack([db[c], 0.25 * dt3[c]])])
              for c in range(2)]
    return alpha, da, beta, dbeta, Theta, dTheta


def psi(x, y, Om):
    """Exact angular flux for direction Om = (mu, eta)."""
    alpha, _, beta, _, T, _ = fields(x, y)
    mu, eta = Om
    val = alpha + mu * beta[0] + eta * beta[1] + mu * mu * T[0, 0] + 2 * mu * eta * T[0, 1] \
        + eta * eta * T[1, 1]
    return val / (4.0 * np.pi)


def grad_psi(x, y, Om):
    """(d psi/dx, d psi/dy) for direction Om."""
    _, da, _, dbeta, _, dT = fields(x, y)
    mu, eta = Om
    out = []
    for c in range(2):
        v = da[c] + mu * dbeta[c][0] + eta * dbeta[c][1] + mu * mu * dT[c][0, 0] \
            + 2 * mu * eta * dT[c][0, 1] + eta * eta * dT[c][1, 1]
        out.append(v / (4.0 * np.pi))
    return out


def phi(x, y):
    alpha, _, _, _, T, _ = fields(x, y)
    return alpha + (T[0, 0] + T[1, 1]) / 3.0


def current(x, y):
    _, _, beta, _, _, _ = fields(x, y)
    return beta / 3.0


def second_moment(x, y):
    """(P_xx, P_xy, P_yy) with the 2 Theta_12 / 15 off-diagonal."""
    alpha, _, _, _, T, _ = fields(x, y)
    return np.stack([alpha / 3.0 + (3 * T[0, 0] + T[1, 1]) / 15.0,
                     2.0 * T[0, 1] / 15.0,
                     alpha / 3.0 + (T[0, 0] + 3 * T[1, 1]) / 15.0])


def source(x, y, Om, sigma_t, sigma_s, phi_in):
    """q_d = Omega . grad psi + sigma_t psi - sigma_s phi_in / (4 pi)."""
    gx, gy = grad_psi(x, y, Om)
    return Om[0] * gx + Om[1] * gy + sigma_t * psi(x, y, Om) - sigma_s * phi_in / (4.0 * np.pi)
