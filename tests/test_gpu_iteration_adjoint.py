"""GPU parity of source iteration and of the adjoint sweep's gradients."""
import numpy as np
import pytest

from _gpu import dev, host, rel, random_problem
from oracle.transport import Discretization, sweep as o_sweep
from oracle.iteration import source_iterate as o_iterate
from oracle.adjoint import adjoint as o_adjoint, region_weights
from vef_inputs import level_symmetric, seeded_media

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_source_iteration(lib, precision, tol):
    from paper_2301_04758_gb300.api import Mesh
    nx, m, alpha, p = 10, 3, 0.05, 2
    om, w = level_symmetric(8)
    E, n = nx * nx, (p + 1) ** 2
    st, ss = seeded_media(E, 2)
    q = np.ones((E, n))
    mesh = Mesh(nx, nx, m, p, alpha)
    phi, psi, dphi, info = mesh.source_iterate(dev(st), dev(ss), om, w, 5, source=dev(q),
                                               precision=precision, info=True)
    disc = Discretization(nx, nx, m, alpha, p)
    rphi, rpsi, rd = o_iterate(disc, om, w, st, ss, source=q, K=5)
    assert rel(host(phi), rphi) < tol
    assert rel(host(psi), rpsi) < tol
    assert np.allclose(host(dphi), rd, rtol=1e-8 if precision == "fp64" else 1e-6)


def test_adjoint_gradients_match_oracle(lib):
    from paper_2301_04758_gb300.api import Mesh
    nx, m, alpha, p = 9, 3, 0.08, 2
    om, w = level_symmetric(8)
    E, n = nx * nx, (p + 1) ** 2
    st, ss = seeded_media(E, 5, log10_range=(-1.0, 1.0))
    rng = np.random.default_rng(9)
    phi_in = rng.uniform(0.5, 1.5, (E, n))
    q = np.ones((E, n))
    disc = Discretization(nx, nx, m, alpha, p)
    g = region_weights(disc)
    psi = o_sweep(disc, om, w, st, ss, phi_in=phi_in, source=q)
    lam, dst, dss = o_adjoint(disc, om, w, st, ss, psi, g, phi_in=phi_in)
    mesh = Mesh(nx, nx, m, p, alpha)
    gpsi = mesh.sweep(dev(st), dev(ss), om, w, phi_in=dev(phi_in), source=dev(q))
    gdst, gdss, glam, info = mesh.adjoint(dev(st), dev(ss), om, w, gpsi, dev(g), phi_in=dev(phi_in),
                                          want_lambda=True, info=True)
    assert rel(host(glam), lam) < 1e-12, info
    assert rel(host(gdst), dst) < 1e-12
    assert rel(host(gdss), dss) < 1e-12


@pytest.mark.parametrize("kernel", ["cta", "cluster"])
def test_adjoint_with_coupled_groups(lib, kernel):
    from paper_2301_04758_gb300.api import Mesh
    prob = random_problem(20, 20, 3, 0.1, 2, 8, seed=3, sigma_range=(-1.0, 0.5), with_inflow=False)
    disc = Discretization(20, 20, 3, 0.1, 2)
    g = region_weights(disc, (0.2, 0.3), (0.7, 0.9))
    psi = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"])
    lam, dst, dss = o_adjoint(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                              psi, g, phi_in=prob["phi_in"])
    mesh = Mesh(20, 20, 3, 2, 0.1)
    gdst, gdss, glam, info = mesh.adjoint(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"],
                                          prob["weights"], dev(psi), dev(g),
                                          phi_in=dev(prob["phi_in"]), want_lambda=True, info=True,
                                          kernel=kernel)
    assert info["coupled_groups"] > 0 and info["timed_out"] == 0
    assert rel(host(glam), lam) < 1e-12, info
    assert rel(host(gdst), dst) < 1e-12


@pytest.mark.parametrize("p", [1, 3, 4])
def test_adjoint_other_orders(lib, p):
    """Adjoint sweep against the oracle's adjoint at the other DG orders (curved mesh,
    heterogeneous media, phi_in given)."""
    from paper_2301_04758_gb300.api import Mesh
    prob = random_problem(7, 6, 3, 0.06, p, 4, seed=80 + p, with_inflow=False)
    disc = Discretization(7, 6, 3, 0.06, p)
    g = region_weights(disc, (0.2, 0.2), (0.8, 0.7))
    psi = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"])
    lam, dst, dss = o_adjoint(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                              psi, g, phi_in=prob["phi_in"])
    mesh = Mesh(7, 6, 3, p, 0.06)
    for kernel in ("cta", "cluster"):
        gdst, gdss, glam, info = mesh.adjoint(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"],
                                              prob["weights"], dev(psi), dev(g),
                                              phi_in=dev(prob["phi_in"]), want_lambda=True, info=True,
                                              kernel=kernel)
        assert info["timed_out"] == 0
        assert rel(host(glam), lam) < 1e-12, (kernel, info)
        assert rel(host(gdst), dst) < 1e-12, kernel
        assert rel(host(gdss), dss) < 1e-12, kernel


@pytest.mark.parametrize("slots", ["0", "3"])
def test_adjoint_trace_slot_capacity_fallback(lib, monkeypatch, slots):
    """With the shared-memory slots capped the backward sweep reads the receivers'
    couplings from global memory (the same slots serve the forward and the adjoint)."""
    from paper_2301_04758_gb300.api import Mesh
    monkeypatch.setenv("VEF_TRACE_SLOTS", slots)
    prob = random_problem(12, 10, 3, 0.1, 2, 8, seed=90, with_inflow=False, sigma_range=(-1.0, 0.5))
    disc = Discretization(12, 10, 3, 0.1, 2)
    g = region_weights(disc, (0.1, 0.2), (0.7, 0.8))
    psi = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"])
    lam, dst, dss = o_adjoint(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                              psi, g, phi_in=prob["phi_in"])
    mesh = Mesh(12, 10, 3, 2, 0.1)
    gdst, gdss, glam, info = mesh.adjoint(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"],
                                          prob["weights"], dev(psi), dev(g),
                                          phi_in=dev(prob["phi_in"]), want_lambda=True, info=True)
    assert info["timed_out"] == 0
    assert rel(host(glam), lam) < 1e-12, info
    assert rel(host(gdst), dst) < 1e-12
    assert rel(host(gdss), dss) < 1e-12


def test_region_weights_match_oracle(lib):
    from paper_2301_04758_gb300.api import Mesh
    disc = Discretization(11, 7, 3, 0.06, 3)
    mesh = Mesh(11, 7, 3, 3, 0.06)
    for lo, hi in (((0.6, 0.6), (0.8, 0.8)), ((0.0, 0.0), (1.0, 1.0)), ((0.13, 0.21), (0.47, 0.83))):
        ref = region_weights(disc, lo, hi)
        got = host(mesh.region_weights(lo, hi))
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max() + 1e-18


def test_autograd_transport_phi(lib):
    """phi from transport_phi is differentiable: backward through the adjoint sweep gives
    the oracle's gradients of R = int_region phi."""
    from paper_2301_04758_gb300.api import Mesh
    from paper_2301_04758_gb300.autograd import transport_phi
    nx, m, alpha, p = 9, 3, 0.08, 2
    om, w = level_symmetric(8)
    E, n = nx * nx, (p + 1) ** 2
    st, ss = seeded_media(E, 5, log10_range=(-1.0, 1.0))
    rng = np.random.default_rng(9)
    phi_in = rng.uniform(0.5, 1.5, (E, n))
    q = np.ones((E, n))
    disc = Discretization(nx, nx, m, alpha, p)
    g = region_weights(disc)
    psi = o_sweep(disc, om, w, st, ss, phi_in=phi_in, source=q)
    _, dst, dss = o_adjoint(disc, om, w, st, ss, psi, g, phi_in=phi_in)
    mesh = Mesh(nx, nx, m, p, alpha)
    st_t = dev(st).requires_grad_()
    ss_t = dev(ss).requires_grad_()
    phi = transport_phi(mesh, st_t, ss_t, om, w, phi_in=dev(phi_in), source=dev(q))
    assert rel(host(phi), np.einsum("d,den->en", w, psi)) < 1e-12
    R = (dev(g) * phi).sum()
    R.backward()
    assert rel(host(st_t.grad), dst) < 1e-12
    assert rel(host(ss_t.grad), dss) < 1e-12


def test_adjoint_with_an_fp32_checkpoint(lib):
    """The forward psi kept as an FP32 copy (VEF_CKPT_FP32): the adjoint solution lambda does
    not depend on psi and stays at the oracle's to 1e-12; the gradients of sigma_t carry the
    copy's rounding (relative 2^-24 per value, averaged over the sums) and sit within 1e-6
    of the oracle's; through autograd with ckpt="fp32" the same."""
    from paper_2301_04758_gb300.api import Mesh
    from paper_2301_04758_gb300.autograd import transport_phi
    nx, m, alpha, p = 9, 3, 0.08, 2
    om, w = level_symmetric(8)
    E, n = nx * nx, (p + 1) ** 2
    st, ss = seeded_media(E, 5, log10_range=(-1.0, 1.0))
    rng = np.random.default_rng(9)
    phi_in = rng.uniform(0.5, 1.5, (E, n))
    q = np.ones((E, n))
    disc = Discretization(nx, nx, m, alpha, p)
    g = region_weights(disc)
    psi = o_sweep(disc, om, w, st, ss, phi_in=phi_in, source=q)
    lam, dst, dss = o_adjoint(disc, om, w, st, ss, psi, g, phi_in=phi_in)
    mesh = Mesh(nx, nx, m, p, alpha)
    gpsi = mesh.sweep(dev(st), dev(ss), om, w, phi_in=dev(phi_in), source=dev(q))
    gdst, gdss, glam = mesh.adjoint(dev(st), dev(ss), om, w, gpsi.float(), dev(g), phi_in=dev(phi_in),
                                    want_lambda=True)
    assert rel(host(glam), lam) < 1e-12
    assert rel(host(gdss), dss) < 1e-12          # does not read psi
    e32 = rel(host(gdst), dst)
    assert 1e-10 < e32 < 1e-6, e32               # the copy's rounding, and only that
    st_t = dev(st).requires_grad_()
    ss_t = dev(ss).requires_grad_()
    phi = transport_phi(mesh, st_t, ss_t, om, w, phi_in=dev(phi_in), source=dev(q), ckpt="fp32")
    (dev(g) * phi).sum().backward()
    assert rel(host(st_t.grad), dst) < 1e-6
    assert rel(host(ss_t.grad), dss) < 1e-12
