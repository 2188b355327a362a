"""Pins for the oracle's residual checkers, r_d = b_d - L_d psi_d.

`oracle.transport.residual` (globally assembled L_d) and `residual_terms` (element by
element, with the term size) are what the full-size GPU tests measure the CUDA sweep
with, so a residual that returned ~0 for any psi, or dropped a term the tests leave
non-NULL, would make those tests pass vacuously.  Each pin below fails for such a slip:
  * closed-form solutions (psi constant; psi linear when the map is in Q_p) leave no
    residual, with scattering source, anisotropic source and inflow all present: a
    dropped or mis-signed streaming, collision, source, phi_in or inflow term breaks it;
  * summed over an element's dofs (test function v = 1) the residual is that element's
    particle-balance defect, computed here from face traces for an arbitrary psi;
  * the two forms agree for arbitrary psi, and r(psi + delta) - r(psi) = -L delta with a
    dense L;
  * at the oracle's own sweep output (coupled groups present) both vanish.
"""
import numpy as np
import pytest

from oracle.transport import Discretization, sweep, residual, residual_terms
from vef_inputs import level_symmetric
from _problems import nodal_xy, boundary_values

FOUR_PI = 4.0 * np.pi


def _ratio(r, size):
    return np.linalg.norm(r) / np.linalg.norm(size)


def _random_inputs(disc, D, seed, aniso=True):
    g = disc.mesh
    rng = np.random.default_rng(seed)
    st = 10.0 ** rng.uniform(-1.0, 1.0, g.E)
    ss = rng.uniform(0.3, 0.95, g.E) * st
    phi_in = rng.uniform(0.5, 2.0, (g.E, disc.n))
    q = rng.uniform(0.0, 1.0, (D, g.E, disc.n) if aniso else (g.E, disc.n))
    inflow = rng.uniform(0.0, 1.0, (D, g.nbf, disc.nq))
    return st, ss, phi_in, q, inflow


def test_residuals_vanish_at_closed_form_solutions():
    """psi = c (any map) and psi = a + b.x (map order 2 <= p = 2) solve the continuous and
    the discrete problem exactly; with phi_in, an anisotropic source and inflow data, both
    residual forms are rounding-small against the size of their terms."""
    om, w = level_symmetric(6)
    D = len(w)
    # constant solution on a curved Q3 map
    disc = Discretization(4, 3, 3, 0.07, 2)
    E, n = disc.mesh.E, disc.n
    rng = np.random.default_rng(5)
    st = rng.uniform(0.2, 8.0, E)
    ss = rng.uniform(0.0, 0.9, E) * st
    c = 0.8
    phi_in = np.full((E, n), FOUR_PI * c)
    q = np.repeat(((st - ss) * c)[None, :, None], D, axis=0) * np.ones((D, E, n))
    inflow = np.full((D, disc.mesh.nbf, disc.nq), c)
    psi = np.full((D, E, n), c)
    r1 = residual(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    r2, size = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    assert _ratio(r1, size) < 1e-14 and _ratio(r2, size) < 1e-14
    # linear solution on a curved Q2 map with Q2 elements
    disc = Discretization(4, 4, 2, 0.05, 2)
    E, n = disc.mesh.E, disc.n
    a, b = 1.5, np.array([0.6, -0.35])
    st = np.linspace(0.4, 3.0, E)
    ss = 0.45 * st
    xn, yn = nodal_xy(disc)
    lin = a + b[0] * xn + b[1] * yn
    phi_in = FOUR_PI * lin
    src = np.stack([om[d] @ b + st[:, None] * lin - ss[:, None] * phi_in / FOUR_PI for d in range(D)])
    inflow = boundary_values(disc, om, lambda x, y, O: a + b[0] * x + b[1] * y)
    psi = np.broadcast_to(lin, (D, E, n)).copy()
    r1 = residual(disc, om, st, ss, psi, phi_in=phi_in, source=src, inflow=inflow)
    r2, size = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=src, inflow=inflow)
    assert _ratio(r1, size) < 1e-13 and _ratio(r2, size) < 1e-13
    # and a wrong solution does leave a residual of the order of its terms
    r3, size3 = residual_terms(disc, om, st, ss, psi * 1.01, phi_in=phi_in, source=src, inflow=inflow)
    assert _ratio(r3, size3) > 1e-4


def _balance_defect(disc, om_d, st, ss, psi_d, phi_in, q_d, inflow_d):
    """Per element: int (sigma_s phi_in / 4pi + q) - oint (Omega.n) psi_hat - int sigma_t psi,
    from the face traces at the face Gauss points (upwind value where Omega.n < 0)."""
    g = disc.mesh
    out = np.zeros(g.E)
    scale = np.zeros(g.E)
    cface = np.einsum("k,efkx,x->efk", g.wf, g.nds, om_d)
    for e in range(g.E):
        flow = 0.0
        for f in range(4):
            own = disc.Bf[f] @ psi_d[e]
            nb = g.nb[e, f]
            up = disc.Bf[g.nbface[e, f]] @ psi_d[nb] if nb >= 0 else inflow_d[g.nbface[e, f]]
            flow += np.sum(cface[e, f] * np.where(cface[e, f] >= 0.0, own, up))
        absorb = st[e] * np.sum(g.wq * g.J[e] * (disc.B @ psi_d[e]))
        src = np.sum(g.wq * g.J[e] * (disc.B @ (ss[e] * phi_in[e] / FOUR_PI + q_d[e])))
        out[e] = src - flow - absorb
        scale[e] = abs(src) + abs(flow) + abs(absorb)
    return out, scale


def test_element_sums_are_the_particle_balance_defect():
    """For an arbitrary psi (not a solution) the residual summed over an element's dofs is
    the element's balance defect (v = 1 makes the volume streaming term vanish); this pins
    the face, collision, source, scattering and inflow terms of both residual forms."""
    om, w = level_symmetric(4)
    D = len(w)
    disc = Discretization(5, 4, 3, 0.08, 3)
    st, ss, phi_in, q, inflow = _random_inputs(disc, D, seed=17)
    psi = np.random.default_rng(18).uniform(0.2, 2.0, (D, disc.mesh.E, disc.n))
    r1 = residual(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    r2, _ = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    for d in range(D):
        want, scale = _balance_defect(disc, om[d], st, ss, psi[d], phi_in, q[d], inflow[d])
        assert np.max(np.abs(want) / scale) > 1e-3          # psi is far from a solution
        for r in (r1, r2):
            np.testing.assert_array_less(np.abs(r[d].sum(axis=1) - want), 1e-12 * scale)


def test_global_and_elementwise_forms_agree_and_are_linear():
    om, w = level_symmetric(8)
    D = len(w)
    disc = Discretization(4, 5, 3, 0.1, 2)
    st, ss, phi_in, q, inflow = _random_inputs(disc, D, seed=23)
    rng = np.random.default_rng(24)
    psi = rng.uniform(0.0, 2.0, (D, disc.mesh.E, disc.n))
    delta = rng.standard_normal(psi.shape)
    r1 = residual(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    r2, size = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    assert _ratio(r1 - r2, size) < 1e-14
    r3 = residual(disc, om, st, ss, psi + delta, phi_in=phi_in, source=q, inflow=inflow)
    for d in range(D):
        L, _ = disc.operator(om[d], st)
        Ld = (L.toarray() @ delta[d].ravel()).reshape(delta[d].shape)
        np.testing.assert_allclose(r3[d] - r1[d], -Ld, rtol=0, atol=1e-12 * np.abs(Ld).max())


@pytest.mark.parametrize("p", [1, 3])
def test_residuals_vanish_at_the_oracle_sweep(p):
    """Strong distortion (alpha = 0.1) gives coupled element groups; the sweep's direct
    solution leaves both residual forms at rounding level."""
    om, w = level_symmetric(8)
    D = len(w)
    disc = Discretization(6, 5, 3, 0.1, p)
    st, ss, phi_in, q, inflow = _random_inputs(disc, D, seed=30 + p)
    psi = sweep(disc, om, w, st, ss, phi_in=phi_in, source=q, inflow=inflow)
    r1 = residual(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    r2, size = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow)
    assert _ratio(r1, size) < 1e-14 and _ratio(r2, size) < 1e-14
    sub, size_sub = residual_terms(disc, om, st, ss, psi, phi_in=phi_in, source=q, inflow=inflow,
                                   directions=[3, D - 1])
    np.testing.assert_array_equal(sub, r2[[3, D - 1]])
    np.testing.assert_array_equal(size_sub, size[[3, D - 1]])
