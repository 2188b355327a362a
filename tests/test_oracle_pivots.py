"""The element solves' pivot guard against the element matrices themselves (CPU).

The CUDA factorisation inverts every (element, direction) matrix by Gauss-Jordan
elimination without pivoting and hands a system to a partial-pivoting fallback when a
pivot falls below 2^VEF_PIVOT_FLOOR_LOG2_* times its row's largest entry (include/vef.h).
Gauss-Jordan meets the same pivots as an unpivoted LU factorisation (the diagonal of U).
This scans those pivots for the oracle's element matrices (oracle.transport, the upwind
DG element block A_e = sigma_t M - streaming + outflow faces) over every level-symmetric
set, p = 1..4, void, thin, diffusive and optically thick elements, straight and strongly
curved meshes (a 4x4 mesh with alpha = 0.1 moves control points by 40 % of an element),
and checks that the smallest relative pivot sits over 100 times above both floors, so
the unpivoted path is the one that runs and the fallback is reserved for degenerate input.
The symmetric part sigma_t M + (1/2) sum |Omega.n| face mass is only semidefinite in void
(an interior node has no face trace), which is why this is checked rather than assumed.
"""
import os
import re

import numpy as np
import pytest

from oracle.transport import Discretization
from vef_inputs import level_symmetric, LQN_ORDERS

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vef.h")


def _floor(name):
    m = re.search(r"#define\s+%s\s+\((-?\d+)\)" % name, open(HEADER).read())
    assert m, name
    return 2.0 ** int(m.group(1))


def relative_pivots(A):
    """[E][n]: |pivot_k| / max_j |A_kj| of the unpivoted elimination of each A_e."""
    A = np.array(A, dtype=np.float64)
    E, n, _ = A.shape
    scale = np.abs(A).max(axis=2)
    out = np.empty((E, n))
    for k in range(n):
        piv = A[:, k, k].copy()
        out[:, k] = np.abs(piv) / scale[:, k]
        f = A[:, k + 1:, k] / piv[:, None]
        A[:, k + 1:, k:] -= f[:, :, None] * A[:, k, None, k:]
    return out


def test_scan_reproduces_lu_pivots():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 6, 6)) + 6 * np.eye(6)
    rp = relative_pivots(A)
    import scipy.linalg as sla
    for e in range(5):
        # without pivoting LU's U diagonal: compare with the Schur complements directly
        U = A[e].copy()
        for k in range(6):
            U[k + 1:, k:] -= np.outer(U[k + 1:, k] / U[k, k], U[k, k:])
        np.testing.assert_allclose(rp[e], np.abs(np.diag(U)) / np.abs(A[e]).max(axis=1), rtol=1e-12)
        # and the product of the pivots is |det A|
        assert np.prod(np.abs(np.diag(U))) == pytest.approx(abs(np.linalg.det(A[e])), rel=1e-10)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_smallest_relative_pivot_is_far_above_the_floors(p):
    floor64 = _floor("VEF_PIVOT_FLOOR_LOG2_FP64")
    floor32 = _floor("VEF_PIVOT_FLOOR_LOG2_FP32")
    assert floor64 < floor32 < 1e-3
    worst = np.inf
    for alpha, m in ((0.0, 1), (0.1, 3)):
        disc = Discretization(4, 4, m, alpha, p)
        for sn in LQN_ORDERS:
            om, _ = level_symmetric(sn)
            for sig in (0.0, 1e-3, 1.0, 1e4):
                st = np.full(disc.mesh.E, sig)
                for d in range(len(om)):
                    A, _ = disc.element_matrices(om[d], st)
                    worst = min(worst, relative_pivots(A).min())
    print(f"p = {p}: smallest relative pivot {worst:.3e}")
    assert worst > 1e2 * floor32


def test_a_degenerate_matrix_falls_below_the_floor():
    """A matrix whose leading 2x2 block is singular to rounding: its second pivot is far
    below the FP64 floor, which is the case the fallback exists for."""
    floor64 = _floor("VEF_PIVOT_FLOOR_LOG2_FP64")
    A = np.array([[1.0, 1.0, 0.5], [1.0, 1.0 + 1e-14, 0.2], [0.3, 0.1, 2.0]])
    rp = relative_pivots(A[None])[0]
    assert rp[1] < floor64 < rp[0]
    # partial pivoting (the fallback's elimination) still inverts it accurately
    assert np.linalg.norm(np.linalg.inv(A) @ A - np.eye(3)) < 1e-2


def _inflow_last_order(p, fx, fy):
    """Node order with the nodes of the two inflow faces (x = 0 side unless fx, y = 0 side
    unless fy, after reflection) eliminated last."""
    Q = p + 1
    inner, infl = [], []
    for ibl in range(Q):
        for ial in range(Q):
            ia = p - ial if fx else ial
            ib = p - ibl if fy else ibl
            (infl if (ial == 0 or ibl == 0) else inner).append(ia + Q * ib)
    return inner + infl


@pytest.mark.parametrize("p", [2, 3])
def test_inflow_last_elimination_order_is_unstable_in_void(p):
    """Why the factorisation keeps the natural (upwind-first) order: eliminating the
    inflow-face nodes last would make the solves for W_f = A^{-1} Cin_f short, but on a
    void element the remaining block (streaming only) is singular, so that order meets a
    zero pivot where the natural order's smallest relative pivot stays far from zero."""
    disc = Discretization(4, 4, 1, 0.0, p)
    worst_nat, worst_perm = np.inf, np.inf
    for sn in (4, 8):
        om, _ = level_symmetric(sn)
        st = np.zeros(disc.mesh.E)
        for d in range(len(om)):
            A, _ = disc.element_matrices(om[d], st)
            worst_nat = min(worst_nat, relative_pivots(A).min())
            fx, fy = om[d][0] < 0, om[d][1] < 0
            o = _inflow_last_order(p, fx, fy)
            with np.errstate(divide="ignore", invalid="ignore"):
                rp = relative_pivots(A[:, o][:, :, o])
            worst_perm = min(worst_perm, np.nanmin(np.where(np.isfinite(rp), rp, 0.0)))
    assert worst_nat > 0.05
    assert worst_perm < 1e-12
