"""Helpers for the GPU parity tests: one seeded problem, run on the CUDA library and on
the oracle."""
import numpy as np
import torch

from vef_inputs import level_symmetric


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda").contiguous()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def random_problem(nx, ny, m, alpha, p, sn, seed, aniso=False, with_inflow=True, with_phi=True,
                   sigma_range=(-1.0, 2.0)):
    """Seeded heterogeneous problem: returns dict of numpy inputs."""
    rng = np.random.default_rng(seed)
    om, w = level_symmetric(sn)
    E, n, nq = nx * ny, (p + 1) ** 2, p + 2
    D = len(w)
    st = 10.0 ** rng.uniform(sigma_range[0], sigma_range[1], E)
    ss = rng.uniform(0.5, 0.99, E) * st
    phi_in = rng.uniform(0.5, 2.0, (E, n)) if with_phi else None
    q = rng.uniform(0.0, 1.0, (D, E, n) if aniso else (E, n))
    inflow = rng.uniform(0.0, 1.0, (D, 2 * nx + 2 * ny, nq)) if with_inflow else None
    return dict(nx=nx, ny=ny, m=m, alpha=alpha, p=p, omega=om, weights=w, sigma_t=st,
                sigma_s=ss, phi_in=phi_in, source=q, inflow=inflow)
