"""Hybridized Raviart-Thomas (HRT) VEF discretisation: element-local elimination and the
reduced system for the Lagrange multiplier (test infrastructure only).

Paper Sec. "Hybridization" ("Extension to VEF", "Implementation Details") on top of the
Raviart-Thomas VEF form of Sec. "Raviart Thomas" (Eqs. A, Ma, D, G, g, f):

  find (J, phi, lambda) in broken RT_p x Y_p x Lambda_p such that for all v, u, mu
    int_G0 [[v . {E n}]] lambda ds - int grad_h v : E phi dx + int sigma_t v . J dx
        + int_Gb (1/E_b) (v . E n)(J . n) ds = int v . Q1 dx + 2 int_Gb (1/E_b) (v . E n) J_in ds,
    int u div_h J dx + int sigma_a u phi dx = int u Q0 dx,
    int_G0 mu [[J . n]] ds = 0.

Matrix form [[A, G, C2], [D, Ma, 0], [C1, 0, 0]] (J, phi, lambda) = (g, f, 0).  A, G, D and
Ma are block diagonal by element; with the element block inverse [[W, X], [Y, Z]] of
[[A, G], [D, Ma]] (Eq. block_inv) the multiplier solves
    H lambda = C1 (W g + X f),   H = C1 W C2,
and the element unknowns follow by block back substitution,
    J = W (g - C2 lambda) + X f,   phi = Y (g - C2 lambda) + Z f.

Discretisation choices (the paper uses MFEM's spaces; these span the same spaces):
  * RT_p on the reference square: x component in Q_{p+1} (xi) x Q_p (eta), y component in
    Q_p (xi) x Q_{p+1} (eta); nodal basis with the p+2 Gauss-Lobatto points in the normal
    direction (the end nodes carry the face's normal flux) and the p+1 Gauss-Legendre
    points in the tangential one; dofs: x part a + (p+2) b, then y part a + (p+1) b.
    Contravariant Piola transform v = F v_hat / J (Eq. piola), gradient of Eq. piola_grad
    written out as grad v = (d v / d xi) F^{-1} with d v / d xi from the map's first and
    second derivatives, divergence div v = div_hat v_hat / J (Eq. piola_div).
  * Y_p: the transport's DG space (tensor Lagrange at Gauss-Lobatto nodes).
  * Lambda_p: degree-p polynomials on each interior face in the face's reference
    coordinate (increasing xi or eta, the same from both sides on the structured mesh),
    Lagrange basis at the p+1 Gauss-Legendre points.
  * Quadrature: the transport's rules (p+2 Gauss-Legendre points per direction), so the
    Eddington tensor enters at the points where the closure pass evaluates it.
  * {E n} on an interior face: the average of the two elements' Eddington tensors (each
    the ratio of its own traces of P and phi) times the normal.
Interior faces are numbered vertical first (between (i, j) and (i+1, j): j (nx-1) + i),
then horizontal (between (i, j) and (i, j+1): (nx-1) ny + j nx + i).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gll_points, gauss_legendre, lagrange, lagrange_deriv
from .mesh import map_jacobian, map_hessian, face_ref_points

FACE_NREF = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])


# ----------------------------------------------------------------- reference spaces
def rt_basis(p, px, py):
    """RT_p reference basis at points: values V [k][nJ][2], d/dxi and d/deta of them
    (same shape), reference divergence [k][nJ]."""
    cl, op = gll_points(p + 1), gauss_legendre(p + 1)[0]
    cx, cy = lagrange(cl, px), lagrange(cl, py)
    ox, oy = lagrange(op, px), lagrange(op, py)
    dcx, dcy = lagrange_deriv(cl, px), lagrange_deriv(cl, py)
    dox, doy = lagrange_deriv(op, px), lagrange_deriv(op, py)
    K = len(px)
    n1 = (p + 2) * (p + 1)
    nJ = 2 * n1
    V = np.zeros((K, nJ, 2))
    Dx = np.zeros((K, nJ, 2))
    Dy = np.zeros((K, nJ, 2))
    for b in range(p + 1):
        for a in range(p + 2):
            i = a + (p + 2) * b                       # x component: closed in xi, open in eta
            V[:, i, 0] = cx[:, a] * oy[:, b]
            Dx[:, i, 0] = dcx[:, a] * oy[:, b]
            Dy[:, i, 0] = cx[:, a] * doy[:, b]
    for b in range(p + 2):
        for a in range(p + 1):
            i = n1 + a + (p + 1) * b                  # y component: open in xi, closed in eta
            V[:, i, 1] = ox[:, a] * cy[:, b]
            Dx[:, i, 1] = dox[:, a] * cy[:, b]
            Dy[:, i, 1] = ox[:, a] * dcy[:, b]
    div = Dx[:, :, 0] + Dy[:, :, 1]
    return V, Dx, Dy, div


def piola(F, J, H, V, Dx, Dy):
    """Physical values v = F v_hat / J [k][nJ][2] and gradients grad v [k][nJ][2][2]
    ((grad v)_{im} = d v_i / d x_m) of Piola-mapped reference functions, from the map's
    Jacobian F [k][2][2], determinant J [k] and second derivatives H [k][i][j][l]."""
    adj = np.stack([np.stack([F[:, 1, 1], -F[:, 0, 1]], -1), np.stack([-F[:, 1, 0], F[:, 0, 0]], -1)], -2)
    Finv = adj / J[:, None, None]
    dF = [H[:, :, :, 0], H[:, :, :, 1]]                 # d F_{ik} / d xi_l, l = 0, 1
    dJ = [np.einsum("kij,kji->k", adj, dF[l]) for l in range(2)]   # Jacobi: dJ = tr(adj F dF)
    v = np.einsum("kij,knj->kni", F, V) / J[:, None, None]
    dv = np.zeros(V.shape + (2,))                       # [k][n][i][l] = d v_i / d xi_l
    for l, D in ((0, Dx), (1, Dy)):
        dv[..., l] = (np.einsum("kij,knj->kni", dF[l], V) + np.einsum("kij,knj->kni", F, D)) / J[:, None, None] \
            - (dJ[l] / J ** 2)[:, None, None] * np.einsum("kij,knj->kni", F, V)
    grad = np.einsum("knil,klm->knim", dv, Finv)
    return v, grad


class HRT:
    """Element-local matrices of the HRT VEF discretisation on the transport
    discretisation's mesh (disc: oracle.transport.Discretization)."""

    def __init__(self, disc):
        self.disc = disc
        g = disc.mesh
        self.p = p = disc.p
        self.n = disc.n
        self.nJ = 2 * (p + 2) * (p + 1)
        self.nl = p + 1                                    # multiplier dofs per face
        nx, ny = g.nx, g.ny
        self.nfaces = (nx - 1) * ny + nx * (ny - 1)
        px, py = g.ref_vol
        self.V, self.Dx, self.Dy, self.div = rt_basis(p, px, py)
        _, F = map_jacobian(g.ctrl, g.m, px, py)
        Hs = map_hessian(g.ctrl, g.m, px, py)
        self.vq, self.gq = [], []
        for e in range(g.E):
            v, gr = piola(F[e], g.J[e], Hs[e], self.V, self.Dx, self.Dy)
            self.vq.append(v)
            self.gq.append(gr)
        # faces: RT values and normal traces at the face points, physical values there
        s = g.s1d
        op = gauss_legendre(p + 1)[0]
        self.lam = lagrange(op, s)                         # [k][t] multiplier basis at face points
        self.vf, self.nflux = [], []
        for f in range(4):
            fx, fy = face_ref_points(f, s)
            Vf, Dfx, Dfy, _ = rt_basis(p, fx, fy)
            _, Ff = map_jacobian(g.ctrl, g.m, fx, fy)
            Jf = Ff[..., 0, 0] * Ff[..., 1, 1] - Ff[..., 0, 1] * Ff[..., 1, 0]
            self.vf.append(np.einsum("ekij,knj->ekni", Ff, Vf) / Jf[..., None, None])   # [E][k][nJ][2]
            self.nflux.append(np.einsum("knj,j->kn", Vf, FACE_NREF[f]))              # v_hat . n_ref
        self.face_id = np.full((g.E, 4), -1, dtype=np.int64)
        for j in range(ny):
            for i in range(nx):
                e = j * nx + i
                if i < nx - 1:
                    self.face_id[e, 1] = j * (nx - 1) + i
                if i > 0:
                    self.face_id[e, 3] = j * (nx - 1) + i - 1
                if j < ny - 1:
                    self.face_id[e, 2] = (nx - 1) * ny + j * nx + i
                if j > 0:
                    self.face_id[e, 0] = (nx - 1) * ny + (j - 1) * nx + i

    # ------------------------------------------------------------- VEF data from moments
    def eddington_data(self, phi, P):
        """E at the volume points [E][nq^2][2][2] and, per face, at the face points from this
        element's traces [E][4][nq][2][2], from the DG moments phi [E][n], P [3][E][n]."""
        d = self.disc

        def ratio(B, ph, PP):
            f = np.einsum("qj,ej->eq", B, ph)
            c = np.einsum("qj,cej->ceq", B, PP) / f[None]
            return np.stack([np.stack([c[0], c[1]], -1), np.stack([c[1], c[2]], -1)], -2)
        Eq = ratio(d.B, phi, P)
        Ef = np.stack([ratio(d.Bf[f], phi, P) for f in range(4)], axis=1)
        return Eq, Ef

    # ------------------------------------------------------------------ element matrices
    def element(self, e, sigma_t, sigma_a, Eq, Ef, Eb, Jin, Q0q, Q1q=None):
        """Local blocks of element e: L = [[A, G], [D, Ma]] ((nJ + n) square), C1 [4 (p+1)][nJ],
        C2 [nJ][4 (p+1)] (zero rows / columns for boundary faces), g [nJ], f [n].
        Eq [E][nq^2][2][2] Eddington tensor at the volume points; Ef [E][4][nq][2][2] at the
        face points from each element's traces; Eb, Jin [N_bf][nq]; Q0q [E][nq^2] and Q1q
        [E][nq^2][2] (or None) the sources at the volume points."""
        d, g = self.disc, self.disc.mesh
        nJ, n, nl = self.nJ, self.n, self.nl
        w = g.wq * g.J[e]                                  # dx weights
        v, gr, B = self.vq[e], self.gq[e], d.B
        A = sigma_t[e] * np.einsum("k,kai,kbi->ab", w, v, v)
        G = -np.einsum("k,kaim,kim,kc->ac", w, gr, Eq[e], B)
        D = np.einsum("k,kc,kb->cb", g.wq, B, self.div)
        Ma = sigma_a[e] * np.einsum("k,kc,kd->cd", w, B, B)
        gv = np.zeros(nJ) if Q1q is None else np.einsum("k,kai,ki->a", w, v, Q1q[e])
        fv = np.einsum("k,kc,k->c", w, B, Q0q[e])
        C1 = np.zeros((4 * nl, nJ))
        C2 = np.zeros((nJ, 4 * nl))
        for f in range(4):
            nds = g.nds[e, f]                              # [nq][2] outward n ds
            vf = self.vf[f][e]                             # [nq][nJ][2]
            if g.nb[e, f] >= 0:
                nb, fo = g.nb[e, f], g.nbface[e, f]
                Eavg = 0.5 * (Ef[e, f] + Ef[nb, fo])
                C2[:, f * nl:(f + 1) * nl] = np.einsum("k,kai,kij,kj,kt->at", g.wf, vf, Eavg, nds, self.lam)
                C1[f * nl:(f + 1) * nl, :] = np.einsum("k,kt,ka->ta", g.wf, self.lam, self.nflux[f])
            else:
                bf = g.nbface[e, f]
                ln = np.linalg.norm(nds, axis=1)
                un = nds / ln[:, None]
                vEn = np.einsum("kai,kij,kj->ka", vf, Ef[e, f], un)
                vn = np.einsum("kai,ki->ka", vf, un)
                A += np.einsum("k,ka,kb->ab", g.wf * ln / Eb[bf], vEn, vn)
                gv += np.einsum("k,ka->a", 2.0 * g.wf * ln * Jin[bf] / Eb[bf], vEn)
        L = np.block([[A, G], [D, Ma]])
        return L, C1, C2, gv, fv

    def _elements(self, sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q, Q1q):
        sigma_t = np.asarray(sigma_t, np.float64)
        sigma_a = sigma_t - np.asarray(sigma_s, np.float64)
        return [self.element(e, sigma_t, sigma_a, Eq, Ef, Eb, Jin, Q0q, Q1q) for e in range(self.disc.mesh.E)]

    def _lam_index(self, e):
        """Global multiplier indices of element e's four faces (-1 for boundary faces)."""
        nl = self.nl
        idx = np.full(4 * nl, -1, dtype=np.int64)
        for f in range(4):
            fid = self.face_id[e, f]
            if fid >= 0:
                idx[f * nl:(f + 1) * nl] = fid * nl + np.arange(nl)
        return idx

    # ------------------------------------------------------------------------- solves
    def solve(self, sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q, Q1q=None):
        """Element-local elimination (paper Sec. "Implementation Details"): returns dict with
        J [E][nJ], phi [E][n], lam [nfaces][p+1], the reduced matrix H (sparse) and rhs r, and
        the element blocks W, X, Y, Z, local H_e and r_e."""
        nJ, nl = self.nJ, self.nl
        els = self._elements(sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q, Q1q)
        N = self.nfaces * nl
        rows, cols, vals = [], [], []
        r = np.zeros(N)
        blocks = []
        for e, (L, C1, C2, gv, fv) in enumerate(els):
            Li = np.linalg.inv(L)
            W, X, Y, Z = Li[:nJ, :nJ], Li[:nJ, nJ:], Li[nJ:, :nJ], Li[nJ:, nJ:]
            He = C1 @ W @ C2
            re = C1 @ (W @ gv + X @ fv)
            idx = self._lam_index(e)
            ok = idx >= 0
            ii, jj = np.meshgrid(idx[ok], idx[ok], indexing="ij")
            rows.append(ii.ravel())
            cols.append(jj.ravel())
            vals.append(He[np.ix_(ok, ok)].ravel())
            np.add.at(r, idx[ok], re[ok])
            blocks.append((W, X, Y, Z, He, re))
        H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
        lam = spla.spsolve(H.tocsc(), r) if N else np.zeros(0)
        E = self.disc.mesh.E
        J = np.zeros((E, nJ))
        phi = np.zeros((E, self.n))
        for e, ((L, C1, C2, gv, fv), (W, X, Y, Z, He, re)) in enumerate(zip(els, blocks)):
            idx = self._lam_index(e)
            le = np.where(idx >= 0, lam[np.maximum(idx, 0)] if N else 0.0, 0.0)
            rhs = gv - C2 @ le
            J[e] = W @ rhs + X @ fv
            phi[e] = Y @ rhs + Z @ fv
        return dict(J=J, phi=phi, lam=lam.reshape(self.nfaces, nl), H=H, r=r, blocks=blocks)

    def solve_full(self, sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q, Q1q=None):
        """The same discrete problem as one global saddle-point system, assembled and solved
        directly (no elimination): returns dict with J, phi, lam."""
        nJ, n, nl = self.nJ, self.n, self.nl
        E = self.disc.mesh.E
        els = self._elements(sigma_t, sigma_s, Eq, Ef, Eb, Jin, Q0q, Q1q)
        m = nJ + n
        N = E * m + self.nfaces * nl
        rows, cols, vals = [], [], []
        b = np.zeros(N)

        def put(r0, c0, M):
            ii, jj = np.nonzero(np.abs(M) > 0)
            rows.append(r0[ii])
            cols.append(c0[jj])
            vals.append(M[ii, jj])
        for e, (L, C1, C2, gv, fv) in enumerate(els):
            loc = e * m + np.arange(m)
            put(loc, loc, L)
            idx = self._lam_index(e)
            ok = idx >= 0
            lg = E * m + idx[ok]
            put(loc[:nJ], lg, C2[:, ok])
            put(lg, loc[:nJ], C1[ok, :])
            b[loc[:nJ]] = gv
            b[loc[nJ:]] = fv
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
        x = spla.spsolve(K.tocsc(), b)
        sol = x[:E * m].reshape(E, m)
        return dict(J=sol[:, :nJ], phi=sol[:, nJ:], lam=x[E * m:].reshape(self.nfaces, nl))

    # --------------------------------------------------------------------- evaluation
    def current_at_points(self, J):
        """Physical current at the volume points [E][nq^2][2] from RT dofs J [E][nJ]."""
        return np.stack([np.einsum("kai,a->ki", self.vq[e], J[e]) for e in range(self.disc.mesh.E)])
