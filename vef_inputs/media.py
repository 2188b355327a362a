"""Seeded cross sections, sources and named workload descriptions.

The paper's own workloads (crooked pipe, triple-point mesh) need geometry that is
only given in figures, so every workload here is synthetic: structured nx x ny
quadrilateral meshes of [0,1]^2, optionally curved by the sine distortion of the
paper's curved-mesh solver study, with seeded heterogeneous media.
"""
import numpy as np

from .quadrature import level_symmetric


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_media(E, sigma_t, sigma_s):
    """Constant cross sections on every element; float64 arrays of length E."""
    return (np.full(E, float(sigma_t)), np.full(E, float(sigma_s)))


def seeded_media(E, seed, log10_range=(-1.0, 2.0), c_range=(0.9, 0.9999)):
    """Per-element sigma_t = 10^U(log10_range), scattering ratio c = U(c_range),
    sigma_s = c * sigma_t.  Draws sigma_t exponents first, then c."""
    rng = _rng(seed)
    st = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=E)
    c = rng.uniform(c_range[0], c_range[1], size=E)
    return st, c * st


def isotropic_source(E, n, value=1.0):
    """Isotropic source q (per steradian) as nodal DG values [E][n]."""
    return np.full((E, n), float(value))


# Named workloads.  'mesh_order' m = 3 for the curved meshes (the paper's sine and
# Taylor-Green meshes are third order); alpha is the sine-distortion amplitude.
WORKLOADS = {
    "tiny_straight_q1_s4": dict(nx=8, ny=8, mesh_order=1, alpha=0.0, p=1, sn=4,
                                media=("uniform", 1.0, 0.5), source=1.0, iterations=1),
    "sine256_q2_s8": dict(nx=256, ny=256, mesh_order=3, alpha=0.05, p=2, sn=8,
                          media=("seeded", 2), source=1.0, iterations=10),
    "sine512_q3_s12": dict(nx=512, ny=512, mesh_order=3, alpha=0.05, p=3, sn=12,
                           media=("seeded", 3), source=1.0, iterations=1),
    "sine128_q2_s8_adjoint": dict(nx=128, ny=128, mesh_order=3, alpha=0.05, p=2, sn=8,
                                  media=("seeded", 5), source=1.0, iterations=1),
}


def batch_problem(k):
    """Problem k (0..63) of the 64-problem batch: mesh size, order and S_N vary with k."""
    sizes = (16, 32, 64, 128, 256)
    sns = (4, 6, 8, 12, 16)
    n = sizes[k % 5]
    return dict(nx=n, ny=n, mesh_order=3, alpha=0.05, p=1 + (k % 4),
                sn=sns[(k % 5 + k // 5) % 5], media=("seeded", 400 + k), source=1.0,
                iterations=1)


def config_workload(name_or_spec):
    """Materialise a workload: returns a dict with the spec plus omega, weights,
    sigma_t, sigma_s, source [E][n] (isotropic)."""
    spec = dict(WORKLOADS[name_or_spec]) if isinstance(name_or_spec, str) else dict(name_or_spec)
    E = spec["nx"] * spec["ny"]
    n = (spec["p"] + 1) ** 2
    om, w = level_symmetric(spec["sn"])
    if spec["media"][0] == "uniform":
        st, ss = uniform_media(E, spec["media"][1], spec["media"][2])
    else:
        st, ss = seeded_media(E, spec["media"][1])
    spec.update(omega=om, weights=w, sigma_t=st, sigma_s=ss,
                source=isotropic_source(E, n, spec["source"]), E=E, n=n, D=len(w))
    return spec
