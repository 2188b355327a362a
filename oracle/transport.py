"""Upwind DG discrete-ordinates transport operator, assembled globally and solved
directly (test infrastructure only).

Paper Eq. transport / trans_bc: Omega . grad psi + sigma_t psi = sigma_s/(4 pi) phi + q
in D, psi = psi_bar on inflow boundary points.  S_N collocation in angle and the DG
space Y_p in space (paper Sec. "Transport Discretizations").  The paper does not
print the DG weak form; this oracle uses the standard once-integrated upwind form,
for every direction d and element K, find psi in Q_p(K) such that for all v:

  - int_K psi (Omega . grad v) dx + int_{dK} (Omega . n) psi_hat v ds
  + int_K sigma_t psi v dx = int_K (sigma_s phi_in / (4 pi) + q_d) v dx,

with psi_hat = psi|_K where Omega . n >= 0 (outflow, including the tangential
case) and psi_hat = the neighbour's trace, or psi_bar on the domain boundary,
where Omega . n < 0.  The choice is made pointwise at every face quadrature point.

In reference coordinates (paper Eq. int_sum and scalar_trans_grad):
  (Omega . grad v) J = (adj(F) Omega) . grad_ref v,  dx = J dxi,  n ds = adj(F)^T n_ref.

The DG basis is the tensor Lagrange basis at the (p+1)^2 Gauss-Lobatto nodes,
local dof a + (p+1) b; the quadrature is tensor Gauss-Legendre with nq = p+2
points per direction on volumes and nq points on faces.  The scattering flux phi_in
and the source q are DG functions in the same space (nodal values).

The result of a sweep is psi_d = L_d^{-1} b_d, computed here by a sparse direct
solve of the global system (no ordering or lagging is involved).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gll_points, tensor_values
from .mesh import Mesh, face_ref_points, OPPOSITE


class Discretization:
    """Mesh plus DG basis tables for order p (nq = p + 2)."""

    def __init__(self, nx, ny, m, alpha, p, ctrl=None):
        self.p = p
        self.n = (p + 1) ** 2
        self.nq = p + 2
        self.mesh = Mesh(nx, ny, m, alpha, self.nq, ctrl=ctrl)
        self.nodes = gll_points(p)
        px, py = self.mesh.ref_vol
        self.B, self.Dxi, self.Deta = tensor_values(self.nodes, px, py)   # [nq^2][n]
        self.Bf = np.zeros((4, self.nq, self.n))                            # face traces
        for f in range(4):
            fx, fy = face_ref_points(f, self.mesh.s1d)
            self.Bf[f] = tensor_values(self.nodes, fx, fy)[0]
        g = self.mesh
        # direction-independent element matrices (for the adjoint gradients)
        self.M = np.einsum("q,eq,qi,qj->eij", g.wq, g.J, self.B, self.B)

    # ------------------------------------------------------------------ operator
    def element_matrices(self, omega, sigma_t):
        """Diagonal blocks A_e [E][n][n] (test index i, trial index j) for one direction."""
        g = self.mesh
        Om = np.asarray(omega, dtype=np.float64)
        Ohat = np.einsum("eqab,b->eqa", g.adjF, Om)                          # adj(F) Omega
        stream = -np.einsum("q,eq,qi,qj->eij", g.wq, Ohat[..., 0], self.Dxi, self.B) \
                 - np.einsum("q,eq,qi,qj->eij", g.wq, Ohat[..., 1], self.Deta, self.B)
        A = sigma_t[:, None, None] * self.M + stream
        c = np.einsum("k,efkd,d->efk", g.wf, g.nds, Om)                      # w (Omega . n ds)
        cout = np.where(c >= 0.0, c, 0.0)
        A += np.einsum("efk,fki,fkj->eij", cout, self.Bf, self.Bf)
        return A, c

    def operator(self, omega, sigma_t):
        """Global sparse L_d (E n x E n) and the face coefficients c [E][4][nq]."""
        g = self.mesh
        n, E = self.n, g.E
        A, c = self.element_matrices(omega, sigma_t)
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        for e in range(E):
            rows.append(e * n + ii.ravel())
            cols.append(e * n + jj.ravel())
            vals.append(A[e].ravel())
            for f in range(4):
                nb = g.nb[e, f]
                if nb < 0:
                    continue
                cin = np.where(c[e, f] < 0.0, c[e, f], 0.0)
                if not np.any(cin):
                    continue
                blk = np.einsum("k,ki,kj->ij", cin, self.Bf[f], self.Bf[OPPOSITE[f]])
                rows.append(e * n + ii.ravel())
                cols.append(nb * n + jj.ravel())
                vals.append(blk.ravel())
        L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(E * n, E * n))
        return L, c

    def rhs(self, c, d, sigma_s, phi_in, source, inflow):
        """b_d [E][n]: volume source plus boundary inflow for direction d.

        source: [E][n] (isotropic) or [D][E][n] (anisotropic); phi_in [E][n] or None;
        inflow [D][N_bf][nq] or None (vacuum)."""
        g = self.mesh
        vol = np.zeros((g.E, self.n))
        if source is not None:
            qd = source if source.ndim == 2 else source[d]
            vol += qd
        if phi_in is not None:
            vol += sigma_s[:, None] * phi_in / (4.0 * np.pi)
        # int J l_i (sum_j vol_j l_j) over the element, by quadrature
        atq = np.einsum("qj,ej->eq", self.B, vol)
        b = np.einsum("q,eq,qi,eq->ei", g.wq, g.J, self.B, atq)
        if inflow is not None:
            for e in range(g.E):
                for f in range(4):
                    if g.nb[e, f] >= 0:
                        continue
                    bf = g.nbface[e, f]
                    cin = np.where(c[e, f] < 0.0, c[e, f], 0.0)
                    b[e] -= np.einsum("k,k,ki->i", cin, inflow[d, bf], self.Bf[f])
        return b


def sweep(disc, omega, weights, sigma_t, sigma_s, phi_in=None, source=None, inflow=None):
    """psi [D][E][n] = L_d^{-1} b_d for every direction (direct sparse solves)."""
    sigma_t = np.asarray(sigma_t, np.float64)
    sigma_s = np.asarray(sigma_s, np.float64)
    D = len(weights)
    psi = np.zeros((D, disc.mesh.E, disc.n))
    for d in range(D):
        L, c = disc.operator(omega[d], sigma_t)
        b = disc.rhs(c, d, sigma_s, phi_in, source, inflow)
        psi[d] = spla.spsolve(L.tocsc(), b.ravel()).reshape(disc.mesh.E, disc.n)
    return psi


def residual(disc, omega, sigma_t, sigma_s, psi, phi_in=None, source=None, inflow=None):
    """r_d = b_d - L_d psi_d [D][E][n] with the globally assembled L_d (used to check a
    candidate solution)."""
    D = psi.shape[0]
    r = np.zeros_like(psi)
    for d in range(D):
        L, c = disc.operator(omega[d], sigma_t)
        b = disc.rhs(c, d, sigma_s, phi_in, source, inflow)
        r[d] = b - (L @ psi[d].ravel()).reshape(b.shape)
    return r


def residual_terms(disc, omega, sigma_t, sigma_s, psi, phi_in=None, source=None, inflow=None,
                   directions=None):
    """Element-by-element r_d = b_d - L_d psi_d and the size of the terms it sums.

    The same upwind system as `operator` / `rhs`, evaluated without assembling L_d: each
    element's block A_e acts on its own psi, and each interior inflow face adds the
    coupling to the neighbour's trace at the face Gauss points.  `size` is the sum of the
    absolute values of every term entering r (|A_e||psi_e| + |couplings| + |b|), the scale
    of its rounding.  directions: indices into omega / psi / source / inflow (default all).
    Returns (r, size), each [len(directions)][E][n]."""
    g = disc.mesh
    sigma_t = np.asarray(sigma_t, np.float64)
    sigma_s = np.asarray(sigma_s, np.float64)
    dirs = range(psi.shape[0]) if directions is None else list(directions)
    r_all = np.zeros((len(dirs), g.E, disc.n))
    s_all = np.zeros_like(r_all)
    for out, d in enumerate(dirs):
        P = psi[d]
        A, c = disc.element_matrices(omega[d], sigma_t)
        b = disc.rhs(c, d, sigma_s, phi_in, source, inflow)
        r = b - np.einsum("eij,ej->ei", A, P)
        size = np.einsum("eij,ej->ei", np.abs(A), np.abs(P)) + np.abs(b)
        for f in range(4):
            nb = g.nb[:, f]
            ok = nb >= 0
            src = np.where(ok, nb, 0)
            cin = np.where(c[:, f] < 0.0, c[:, f], 0.0)
            Bo = disc.Bf[OPPOSITE[f]]
            tr = np.einsum("kj,ej->ek", Bo, P[src])
            atr = np.einsum("kj,ej->ek", np.abs(Bo), np.abs(P[src]))
            r -= np.where(ok[:, None], np.einsum("ek,ki,ek->ei", cin, disc.Bf[f], tr), 0.0)
            size += np.where(ok[:, None],
                             np.einsum("ek,ki,ek->ei", np.abs(cin), np.abs(disc.Bf[f]), atr), 0.0)
        r_all[out] = r
        s_all[out] = size
    return r_all, s_all
