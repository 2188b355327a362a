"""Level-symmetric (LQn) S_N angular quadrature restricted to the 2D (x-y) setting.

The transport equation is collocated at discrete directions with weights that
integrate over the unit sphere (paper Sec. "Transport Discretizations", the S_N
angular model).  The paper uses level-symmetric sets (S4 for the MMS and thick
diffusion runs, S12 for the crooked pipe).

Construction (classical LQn):
  * mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2),  i = 1..N/2
  * the octant points are (mu_i, mu_j, mu_k) with i + j + k = N/2 + 2
  * points that are permutations of each other share one weight ("class")
  * class weights solve the even-moment conditions
        sum_octant w mu^(2m) = 1/(2m+1),  m = 0, 2, 3, ..., N/2 - 1
    (m = 1 holds automatically by symmetry).  For N <= 12 the system is square.
    For N = 16 it leaves one free parameter; we take the member of the solution
    set closest (least squares) to the published 7-digit LQ16 weights, so the
    pure moment conditions hold to round-off and the weights match the table.
  * mu_1 is the published LQn value for N >= 6; for N = 4 it is the exact root
    of the mu^4 condition, 6 a^2 - 4 a + 2/5 = 0, a = mu_1^2.

2D reduction: the directions with xi = Omega_z > 0 are kept; each stands for
itself and its mirror image xi < 0, so its weight is doubled.  The weights are
scaled so that sum_d w_d = 4 pi.  D = N (N + 2) / 2.

Direction order: quadrants (+,+), (-,+), (-,-), (+,-); inside a quadrant the
octant points in lexicographic (i, j) order.
"""
import numpy as np

LQN_ORDERS = (4, 6, 8, 12, 16)

_MU1 = {6: 0.2666355, 8: 0.2182179, 12: 0.1672126, 16: 0.1389568}
# Published LQ16 class weights (Lewis & Miller), classes ordered by the sorted
# level-index triple: (1,1,8) (1,2,7) (1,3,6) (1,4,5) (2,2,6) (2,3,5) (2,4,4) (3,3,4).
_LQ16_TABLE = np.array([0.0489872, 0.0413296, 0.0212326, 0.0256207,
                        0.0360486, 0.0144589, 0.0344958, 0.0085179])


def _levels(N):
    L = N // 2
    if N == 4:
        a = (4.0 - np.sqrt(6.4)) / 12.0
        mu1sq = a
    else:
        mu1sq = _MU1[N] ** 2
    return np.sqrt(mu1sq + np.arange(L) * 2.0 * (1.0 - 3.0 * mu1sq) / (N - 2))


def _octant(N):
    L = N // 2
    mus = _levels(N)
    pts = [(i, j, L + 2 - i - j) for i in range(1, L + 1) for j in range(1, L + 1)
           if L + 2 - i - j >= 1]
    classes = sorted(set(tuple(sorted(p)) for p in pts))
    cid = np.array([classes.index(tuple(sorted(p))) for p in pts])
    nc = len(classes)
    rows, rhs = [], []
    for m in [0] + list(range(2, L)):
        r = np.zeros(nc)
        for p, c in zip(pts, cid):
            r[c] += mus[p[0] - 1] ** (2 * m)
        rows.append(r)
        rhs.append(1.0 / (2 * m + 1))
    A = np.array(rows)
    b = np.array(rhs)
    if A.shape[0] == nc:
        w = np.linalg.solve(A, b)
    else:
        # one-parameter family: particular solution + t * null vector, t closest to the table
        w0 = np.linalg.lstsq(A, b, rcond=None)[0]
        null = np.linalg.svd(A)[2][-1]
        t = (_LQ16_TABLE - w0) @ null / (null @ null)
        w = w0 + t * null
    if np.any(w <= 0):
        raise ValueError(f"LQ{N}: non-positive class weight")
    return mus, pts, w[cid]


def level_symmetric(N):
    """Return (omega [D][2], weights [D]) of the 2D LQ_N set, float64, sum w = 4 pi."""
    if N not in LQN_ORDERS:
        raise ValueError(f"unsupported S_N order {N}; choose from {LQN_ORDERS}")
    mus, pts, wpt = _octant(N)
    om, ww = [], []
    for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        for (i, j, _k), w in zip(pts, wpt):
            om.append((sx * mus[i - 1], sy * mus[j - 1]))
            ww.append(w)
    om = np.array(om, dtype=np.float64)
    ww = np.array(ww, dtype=np.float64)
    ww *= 4.0 * np.pi / ww.sum()
    return om, ww
