"""GPU parity: the CUDA sweep (through the C ABI) against the FP64 oracle.

Bar: FP64 path within 1e-12 relative L2 on psi; mixed path within 1e-10 on psi, phi, E.
"""
import numpy as np
import pytest

from _gpu import dev, host, rel, random_problem, oracle_sweep_parallel
from oracle.transport import Discretization, sweep as o_sweep, residual as o_residual, residual_terms

pytestmark = pytest.mark.gpu


def _run(prob, precision="fp64", info=True, **kw):
    from paper_2301_04758_gb300.api import Mesh
    mesh = Mesh(prob["nx"], prob["ny"], prob["m"], prob["p"], prob["alpha"])
    src = prob["source"]
    out = mesh.sweep(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"], prob["weights"],
                     phi_in=None if prob["phi_in"] is None else dev(prob["phi_in"]),
                     source=dev(src), inflow=None if prob["inflow"] is None else dev(prob["inflow"]),
                     precision=precision, info=info, **kw)
    return mesh, out


def _oracle(prob):
    disc = Discretization(prob["nx"], prob["ny"], prob["m"], prob["alpha"], prob["p"])
    psi = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"], inflow=prob["inflow"])
    return disc, psi


def test_tiny_straight_q1_s4(lib):
    """8x8 straight Q1, S4, sigma_t = 1, sigma_s = 0.5, q = 1, vacuum, phi_in = 0."""
    from vef_inputs import config_workload
    wl = config_workload("tiny_straight_q1_s4")
    prob = dict(nx=8, ny=8, m=1, alpha=0.0, p=1, omega=wl["omega"], weights=wl["weights"],
                sigma_t=wl["sigma_t"], sigma_s=wl["sigma_s"], phi_in=None, source=wl["source"],
                inflow=None)
    _, (psi, info) = _run(prob)
    _, ref = _oracle(prob)
    assert rel(host(psi), ref) < 1e-12
    assert info["coupled_groups"] == 0 and info["levels"] == 15   # 2N-1 diagonal wavefront
    assert info["timed_out"] == 0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_curved_heterogeneous_all_orders(lib, p):
    prob = random_problem(7, 5, 3, 0.06, p, 4, seed=10 + p)
    _, (psi, info) = _run(prob)
    _, ref = _oracle(prob)
    assert rel(host(psi), ref) < 1e-12, info


@pytest.mark.parametrize("groups", ["direct", "iterative"])
@pytest.mark.parametrize("sn", [8, 12])
def test_curved_with_coupled_groups(lib, sn, groups):
    """Strong distortion gives faces that are part inflow, part outflow: the coupled
    element groups must be solved to round-off, not lagged.  At S12 the largest groups
    have 8 elements and 42 trace values, so both the shared-memory and the global-memory
    form of the direct solve run; "iterative" forces the inner Gauss-Seidel for all."""
    prob = random_problem(20, 20, 3, 0.1, 2, sn, seed=3, sigma_range=(-1.0, 0.5))
    _, (psi, info) = _run(prob, groups=groups)
    disc, ref = _oracle(prob)
    assert info["coupled_groups"] > 0, info
    assert rel(host(psi), ref) < 1e-12, info
    if groups == "direct":
        assert info["max_inner_iterations"] == 0, info
    else:
        assert info["max_inner_iterations"] >= 2, info


def test_large_groups_mix_direct_and_iterative(lib):
    """alpha = 0.15 on a 16x16 mesh at S16 gives groups of up to ~36 elements whose trace
    systems exceed 128 values: those fall back to the inner iteration while the smaller
    groups of the same sweep are solved directly."""
    prob = random_problem(16, 16, 3, 0.15, 2, 16, seed=21, sigma_range=(-1.0, 0.5))
    _, (psi, info) = _run(prob)
    disc, ref = _oracle(prob)
    assert info["coupled_groups"] > 0, info
    assert info["max_inner_iterations"] >= 2, info
    assert rel(host(psi), ref) < 1e-12, info
    _, (psi_it, _) = _run(prob, groups="iterative")
    assert rel(host(psi), host(psi_it)) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cta_and_cluster_kernels_agree(lib, p):
    """The default sweep (one CTA per direction, upwind traces in shared-memory slots) and
    the cluster sweep both reproduce the oracle on a strongly curved mesh with coupled
    groups, anisotropic source and inflow."""
    prob = random_problem(11, 9, 3, 0.1, p, 8, seed=40 + p, aniso=True, sigma_range=(-1.0, 0.5))
    _, (psi_cta, info) = _run(prob)
    _, (psi_cl, info_cl) = _run(prob, kernel="cluster")
    _, ref = _oracle(prob)
    assert info["coupled_groups"] > 0 and info["timed_out"] == 0 and info_cl["timed_out"] == 0
    assert rel(host(psi_cta), ref) < 1e-12, info
    assert rel(host(psi_cl), ref) < 1e-12, info_cl


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_and_separate_apply_agree(lib, precision):
    """By default the SMs the directions leave free compute y = A^{-1} b inside the sweep
    launch (band flags between the two roles); VEF_APPLY_SEPARATE keeps a launch of its
    own.  Both reproduce the oracle."""
    prob = random_problem(14, 12, 3, 0.1, 2, 8, seed=95, aniso=True, sigma_range=(-1.0, 0.5))
    _, (psi_f, info_f) = _run(prob, precision=precision)
    _, (psi_s, info_s) = _run(prob, precision=precision, apply="separate")
    _, ref = _oracle(prob)
    tol = 1e-12 if precision == "fp64" else 1e-10
    assert info_f["timed_out"] == 0 and info_s["timed_out"] == 0
    assert rel(host(psi_f), ref) < tol, info_f
    assert rel(host(psi_s), ref) < tol, info_s


@pytest.mark.parametrize("slots", ["0", "3"])
def test_trace_slot_capacity_fallback(lib, monkeypatch, slots):
    """With the shared-memory trace slots capped (none, or three live at a time) the
    couplings left over read the donor's psi from global memory; results are unchanged."""
    monkeypatch.setenv("VEF_TRACE_SLOTS", slots)
    prob = random_problem(10, 12, 3, 0.08, 2, 8, seed=50, aniso=True)
    _, (psi, info) = _run(prob)
    _, ref = _oracle(prob)
    assert rel(host(psi), ref) < 1e-12, info


@pytest.mark.parametrize("nx,p,sn", [(30, 4, 4), (120, 1, 4)])
def test_levels_wider_than_a_round(lib, nx, p, sn):
    """Levels of up to nx single-element tasks span several rounds of the CTA sweep
    (14 tasks per round at p = 4, 112 at p = 1), so the ring of round buffers wraps
    inside a level and across levels."""
    prob = random_problem(nx, nx, 3, 0.03, p, sn, seed=60 + p)
    _, (psi, info) = _run(prob)
    _, ref = _oracle(prob)
    assert info["timed_out"] == 0
    assert rel(host(psi), ref) < 1e-12, info


def test_anisotropic_source_and_inflow(lib):
    prob = random_problem(6, 9, 2, 0.05, 2, 8, seed=4, aniso=True)
    _, (psi, _) = _run(prob)
    _, ref = _oracle(prob)
    assert rel(host(psi), ref) < 1e-12


def test_edge_cases_single_element_and_ragged(lib):
    for (nx, ny, p, sn) in [(1, 1, 3, 4), (9, 2, 1, 6), (2, 11, 2, 4)]:
        prob = random_problem(nx, ny, 3, 0.04, p, sn, seed=nx * 7 + ny)
        _, (psi, _) = _run(prob)
        _, ref = _oracle(prob)
        assert rel(host(psi), ref) < 1e-12, (nx, ny)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_void_and_optically_thick_elements(lib, precision):
    """Cross sections from void (sigma_t = 0: the element solve has only the streaming
    and outflow terms, and at p >= 2 the interior node's diagonal entry vanishes) to
    1e4 (thick diffusive elements, sigma_s / sigma_t = 1 - 1e-8) in one curved mesh,
    p = 1..4.  The unpivoted Gauss-Jordan on the element matrix must match the oracle's
    pivoted sparse solve."""
    for p in (1, 2, 3, 4):
        prob = random_problem(6, 5, 3, 0.05, p, 8, seed=60 + p)
        E = 30
        kind = np.arange(E) % 3
        st = np.where(kind == 0, 0.0, np.where(kind == 1, 1e4, prob["sigma_t"]))
        ss = np.where(kind == 0, 0.0, np.where(kind == 1, st * (1 - 1e-8), prob["sigma_s"]))
        prob = dict(prob, sigma_t=st, sigma_s=ss)
        _, (psi, info) = _run(prob, precision=precision)
        _, ref = _oracle(prob)
        assert info["timed_out"] == 0
        assert rel(host(psi), ref) < (1e-12 if precision == "fp64" else 1e-10), (p, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pivot_guard_and_partial_pivoting_fallback(lib, precision):
    """The element systems are inverted without pivoting; the guard sends a system whose
    pivot falls below the relative floor to a partial-pivoting fallback.  On ordinary
    meshes (void and thick elements included) no system goes there; forcing every system
    through the fallback (VEF_PIVOT_ALWAYS) reproduces the oracle, p = 1..4."""
    tol = 1e-12 if precision == "fp64" else 1e-10
    for p in (1, 2, 3, 4):
        prob = random_problem(6, 5, 3, 0.1, p, 8, seed=80 + p, aniso=True, sigma_range=(-1.0, 0.5))
        kind = np.arange(30) % 4
        prob["sigma_t"] = np.where(kind == 0, 0.0, np.where(kind == 1, 1e4, prob["sigma_t"]))
        prob["sigma_s"] = np.where(kind == 0, 0.0, np.where(kind == 1, prob["sigma_t"] * 0.999, prob["sigma_s"]))
        _, ref = _oracle(prob)
        _, (psi, info) = _run(prob, precision=precision)
        assert info["pivoted_tasks"] == 0 and info["timed_out"] == 0, info
        assert rel(host(psi), ref) < tol, (p, info)
        _, (psi_pv, info_pv) = _run(prob, precision=precision, pivot="always")
        assert info_pv["pivoted_tasks"] == 30 * len(prob["weights"]), info_pv
        assert rel(host(psi_pv), ref) < tol, (p, info_pv)


def test_maximum_direction_count(lib):
    """D = 1023, the largest direction set a call takes (10 bits of direction index in a
    packed task code), on a small curved mesh: 1023 direction CTAs leave no SMs for the
    fused apply, so the separate apply launch runs.  psi and the closures match the oracle,
    and D = 1024 is refused."""
    import ctypes
    from oracle.moments import closures
    from paper_2301_04758_gb300 import _lib
    rng = np.random.default_rng(1023)
    D = 1023
    z, ph = rng.uniform(0.02, 0.98, D), rng.uniform(0.0, 2 * np.pi, D)
    om = np.stack([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph)], axis=1)
    w = np.full(D, 4 * np.pi / D)
    prob = random_problem(3, 2, 3, 0.05, 2, 4, seed=5, with_inflow=False)
    prob = dict(prob, omega=om, weights=w)
    mesh, (psi, info) = _run(prob)
    disc, ref = _oracle(prob)
    assert info["timed_out"] == 0
    assert rel(host(psi), ref) < 1e-12
    out = mesh.moments(psi, om, w)
    rc = closures(disc, ref, om, w)
    for k in ("phi", "J", "E", "Eb"):
        assert rel(host(out[k]), rc[k]) < 1e-12, k
    om2 = np.ascontiguousarray(np.concatenate([om, om[:1]]), dtype=np.float64)
    w2 = np.full(D + 1, 4 * np.pi / (D + 1))
    st = lib.vef_sweep(mesh.handle, None, None, None, None, 0, None,
                       om2.ctypes.data_as(ctypes.c_void_p), w2.ctypes.data_as(ctypes.c_void_p), D + 1,
                       None, None, None, None)
    assert st == _lib.VEF_ERR_INVALID_ARG and b"1..1023" in lib.vef_last_error()


def test_axis_aligned_and_single_direction(lib):
    """Directions parallel to straight faces (Omega . n = 0 on two faces: outflow by
    convention, zero weight) and a one-direction set."""
    prob = random_problem(5, 4, 1, 0.0, 2, 4, seed=8)
    prob["omega"] = np.array([[1.0, 0.0], [0.0, -1.0], [-0.6, 0.8]])
    prob["weights"] = np.array([1.0, 2.0, 3.0])
    prob["inflow"] = prob["inflow"][:3]
    _, (psi, _) = _run(prob)
    _, ref = _oracle(prob)
    assert rel(host(psi), ref) < 1e-12
    one = dict(prob, omega=prob["omega"][2:], weights=prob["weights"][2:], inflow=prob["inflow"][2:])
    _, (psi1, _) = _run(one)
    _, ref1 = _oracle(one)
    assert rel(host(psi1), ref1) < 1e-12


def test_mixed_precision_defect_correction(lib):
    from oracle.moments import closures
    prob = random_problem(12, 12, 3, 0.08, 3, 8, seed=21)
    mesh, (psi, info) = _run(prob, precision="mixed")
    disc, ref = _oracle(prob)
    assert info["passes"] >= 2 and info["rel_residual"] <= 1e-13, info
    assert rel(host(psi), ref) < 1e-10
    out = mesh.moments(psi, prob["omega"], prob["weights"])
    rc = closures(disc, ref, prob["omega"], prob["weights"])
    assert rel(host(out["phi"]), rc["phi"]) < 1e-10
    assert rel(host(out["E"]), rc["E"]) < 1e-10


@pytest.mark.parametrize("kernel", ["cta", "cluster"])
def test_mixed_p3_correction_takes_y_from_the_residual(lib, kernel):
    """At p = 3 the FP64 residual kernel also forms the correction sweep's y = A^{-1} r,
    and the correction sweep skips its apply: through the single-CTA and the cluster sweep,
    with an anisotropic source, inflow and coupled groups, to the default tolerance (several
    passes, each residual forming the next y) and with two fixed passes, psi matches the
    FP64 oracle."""
    prob = random_problem(11, 9, 3, 0.1, 3, 8, seed=47, aniso=True, sigma_range=(-1.0, 0.5))
    _, ref = _oracle(prob)
    for kw in (dict(), dict(tol=-1.0, max_passes=2)):
        _, (psi, info) = _run(prob, precision="mixed", kernel=kernel, **kw)
        assert info["timed_out"] == 0 and info["passes"] >= 2 and info["coupled_groups"] > 0, info
        assert rel(host(psi), ref) < 1e-10, (kw, info)


def test_mixed_precision_q3_s12_against_the_oracle(lib):
    """The precision workload's recipe (sine alpha 0.05, Q3 map, DG Q3, S12, seed-3 media,
    q = 1, vacuum) on a 48x48 mesh: the mixed-precision sweep (FP32 factorisation and
    sweeps inside FP64 defect correction), as the benchmark runs it (two passes, no final
    residual) and to its default tolerance, against the FP64 oracle: psi, phi, J and E each
    within 1e-10 relative L2."""
    from oracle.moments import closures
    from vef_inputs import level_symmetric, seeded_media
    from paper_2301_04758_gb300.api import Mesh
    N, p = 48, 3
    om, w = level_symmetric(12)
    st, ss = seeded_media(N * N, 3)
    q = np.ones((N * N, 16))
    disc = Discretization(N, N, 3, 0.05, p)
    ref = oracle_sweep_parallel((N, N, 3, 0.05, p), om, w, st, ss, source=q)
    rc = closures(disc, ref, om, w)
    mesh = Mesh(N, N, 3, p, 0.05)
    for kw in (dict(), dict(tol=-1.0, max_passes=2)):
        psi, info = mesh.sweep(dev(st), dev(ss), om, w, source=dev(q), precision="mixed", info=True, **kw)
        assert info["timed_out"] == 0 and info["passes"] >= 2, info
        out = mesh.moments(psi, om, w)
        assert rel(host(psi), ref) < 1e-10, kw
        for k in ("phi", "J", "E"):
            assert rel(host(out[k]), rc[k]) < 1e-10, (k, kw)


@pytest.mark.parametrize("p,sn", [(2, 8), (3, 12)])
def test_taylor_green_mesh_from_user_control_points(lib, p, sn):
    """The paper's third-order Taylor-Green mesh (an orthogonal mesh advected by the vortex
    to T = 0.3 pi, 300 forward Euler steps; its x = 1 and y = 1 sides move with it), given
    to vef_mesh_create as control points: the faces tilt enough that many are partly inflow
    and partly outflow, so the sweep solves coupled element groups; psi matches the oracle
    on the same control points."""
    from vef_inputs import taylor_green_control_points
    from paper_2301_04758_gb300.api import Mesh
    nx = ny = 10
    ctrl = taylor_green_control_points(nx, ny, 3)
    prob = random_problem(nx, ny, 3, 0.0, p, sn, seed=120 + p, aniso=True)
    mesh = Mesh(nx, ny, 3, p, 0.0, ctrl=ctrl)
    psi, info = mesh.sweep(dev(prob["sigma_t"]), dev(prob["sigma_s"]), prob["omega"], prob["weights"],
                           phi_in=dev(prob["phi_in"]), source=dev(prob["source"]),
                           inflow=dev(prob["inflow"]), info=True)
    disc = Discretization(nx, ny, 3, 0.0, p, ctrl=ctrl)
    ref = o_sweep(disc, prob["omega"], prob["weights"], prob["sigma_t"], prob["sigma_s"],
                  phi_in=prob["phi_in"], source=prob["source"], inflow=prob["inflow"])
    assert info["coupled_groups"] > 0 and info["timed_out"] == 0, info
    assert rel(host(psi), ref) < 1e-12, info
    from oracle.moments import closures
    out = mesh.moments(psi, prob["omega"], prob["weights"], inflow=dev(prob["inflow"]))
    rc = closures(disc, ref, prob["omega"], prob["weights"], inflow=prob["inflow"])
    for k in ("phi", "J", "E", "Eb", "Jin"):
        assert rel(host(out[k]), rc[k]) < 1e-12, k


def test_invalid_arguments_are_rejected(lib):
    import ctypes
    from paper_2301_04758_gb300 import _lib
    from paper_2301_04758_gb300.api import Mesh
    h = ctypes.c_void_p()
    assert lib.vef_mesh_create(0, 4, 1, 1, 0.0, None, ctypes.byref(h)) == _lib.VEF_ERR_INVALID_ARG
    assert lib.vef_mesh_create(4, 4, 1, 7, 0.0, None, ctypes.byref(h)) == _lib.VEF_ERR_INVALID_ARG
    mesh = Mesh(3, 3, 1, 1, 0.0)
    st = lib.vef_sweep(mesh.handle, None, None, None, None, 0, None, None, None, 0, None, None,
                       None, None)
    assert st == _lib.VEF_ERR_INVALID_ARG


@pytest.mark.slow
def test_full_size_sine256_q2_s8_global_residual(lib):
    """At the benchmark size (256^2, Q2, S8, seeded media) the GPU psi satisfies the
    oracle's global upwind system to rounding: ||b - L psi|| is compared with the size of
    the terms the residual sums, || |L| |psi| || + ||b||.  The streaming terms are O(h psi)
    while b is O(h^2 q), so ||b|| alone understates the rounding floor by about 1/h.  Each
    element solve applies an explicit inverse (condition number <= 18 on this mesh) to a sum
    of up to 21 terms, so the bound allows a few hundred ulps of the term size."""
    from vef_inputs import config_workload
    wl = config_workload("sine256_q2_s8")
    from paper_2301_04758_gb300.api import Mesh
    mesh = Mesh(256, 256, 3, 2, 0.05)
    psi, info = mesh.sweep(dev(wl["sigma_t"]), dev(wl["sigma_s"]), wl["omega"], wl["weights"],
                           source=dev(wl["source"]), info=True)
    assert info["timed_out"] == 0
    disc = Discretization(256, 256, 3, 0.05, 2)
    P = host(psi)
    for d in (0, 13, 27, 39):
        om = wl["omega"][d:d + 1]
        r = o_residual(disc, om, wl["sigma_t"], wl["sigma_s"], P[d:d + 1], source=wl["source"])
        L, c = disc.operator(om[0], wl["sigma_t"])
        b = disc.rhs(c, 0, wl["sigma_s"], None, wl["source"], None)
        scale = np.linalg.norm(abs(L) @ np.abs(P[d].ravel())) + np.linalg.norm(b)
        assert np.linalg.norm(r) / scale < 1e-13, d
    # forward error: the oracle's direct solve of sampled directions, element by element
    sample = (0, 13, 27, 39)
    ref = oracle_sweep_parallel((256, 256, 3, 0.05, 2), wl["omega"], wl["weights"], wl["sigma_t"],
                                wl["sigma_s"], source=wl["source"], directions=sample)
    for k, d in enumerate(sample):
        assert rel(P[d], ref[k]) < 1e-12, d


@pytest.mark.slow
def test_full_size_sine512_q3_s12_fp64_and_mixed(lib):
    """The precision workload at full size (512^2, Q3, S12: 84 directions, 22 M element
    systems of order 16), as bench.py launches it: on sampled directions the FP64 sweep
    satisfies the upwind system to rounding of the summed terms (as in the 256^2 test),
    and the mixed-precision sweep (FP32 solves inside FP64 defect correction, target
    ||r|| / ||b|| <= 1e-13) to the same order of magnitude."""
    from vef_inputs import config_workload
    from paper_2301_04758_gb300.api import Mesh
    wl = config_workload("sine512_q3_s12")
    mesh = Mesh(512, 512, 3, 3, 0.05)
    st, ss, q = dev(wl["sigma_t"]), dev(wl["sigma_s"]), dev(wl["source"])
    P64, info = mesh.sweep(st, ss, wl["omega"], wl["weights"], source=q, info=True)
    assert info["timed_out"] == 0 and info["coupled_groups"] > 0, info
    P64 = host(P64)
    Pmx, infm = mesh.sweep(st, ss, wl["omega"], wl["weights"], source=q, precision="mixed", info=True)
    assert infm["rel_residual"] <= 1e-13, infm
    Pmx = host(Pmx)
    del mesh
    disc = Discretization(512, 512, 3, 0.05, 3)
    for P, bound in ((P64, 1e-13), (Pmx, 1e-12)):
        r, size = residual_terms(disc, wl["omega"], wl["sigma_t"], wl["sigma_s"], P,
                                 source=wl["source"], directions=(0, 41, 83))
        for k in range(3):
            assert np.linalg.norm(r[k]) / np.linalg.norm(size[k]) < bound, (k, bound)
