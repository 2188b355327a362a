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


def _oracle_part(args):
    """Worker: the oracle's direct solve for a subset of the directions."""
    (nx, ny, m, alpha, p), om, w, st, ss, phi_in, source, inflow = args
    from oracle.transport import Discretization, sweep
    disc = Discretization(nx, ny, m, alpha, p)
    return sweep(disc, om, w, st, ss, phi_in=phi_in, source=source, inflow=inflow)


def oracle_sweep_parallel(mesh_args, omega, weights, sigma_t, sigma_s, phi_in=None, source=None,
                          inflow=None, directions=None, procs=None):
    """psi [len(directions)][E][n] from oracle.transport.sweep, the directions split over
    spawned worker processes (each solve is independent of the others; spawn, so that no
    worker inherits a CUDA context).  mesh_args = (nx, ny, m, alpha, p)."""
    import multiprocessing as mp
    import os
    dirs = np.arange(len(weights)) if directions is None else np.asarray(directions)
    procs = procs or max(1, min(len(dirs), os.cpu_count() or 1, 16))
    chunks = [c for c in np.array_split(dirs, procs) if len(c)]

    def sub(a, c):
        return None if a is None else (a[c] if np.ndim(a) == 3 else a)
    jobs = [(tuple(mesh_args), omega[c], weights[c], sigma_t, sigma_s, phi_in, sub(source, c), sub(inflow, c))
            for c in chunks]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_oracle_part, jobs, chunksize=1)
    return np.concatenate(parts, axis=0)
