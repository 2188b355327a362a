"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the CPU oracle.

This module generates *input data only*: angular quadrature sets (directions and
weights), per-element cross sections, isotropic/anisotropic sources, boundary inflow
arrays and mesh control points (the Taylor-Green advected mesh).  It contains none of the transport method's arithmetic (no mesh
geometry, no element matrices, no sweep, no moments).

Everything is deterministic given a seed (NumPy PCG64).

Layouts (shared by the C-ABI and the oracle):
  omega   [D][2]      direction cosines (mu, eta) of the x-y projection
  weights [D]         angular weights, sum = 4*pi
  sigma_t, sigma_s [E]  per-element total / scattering cross sections, E = nx*ny,
                        element e = j*nx + i
"""
from .quadrature import level_symmetric, LQN_ORDERS
from .media import (uniform_media, seeded_media, isotropic_source, config_workload,
                    WORKLOADS)
from .meshes import taylor_green_control_points

__all__ = ["level_symmetric", "LQN_ORDERS", "uniform_media", "seeded_media",
           "isotropic_source", "config_workload", "WORKLOADS", "taylor_green_control_points"]
