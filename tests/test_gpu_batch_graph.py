"""Batched sweeps, the autotuner and CUDA-graph capture (GPU, through the C ABI)."""
import numpy as np
import pytest
import torch

from _gpu import dev, host, rel
from vef_inputs import level_symmetric, seeded_media

pytestmark = pytest.mark.gpu

SPECS = [(9, 1, 4), (12, 2, 8), (7, 3, 6), (5, 4, 12), (16, 2, 16), (10, 1, 8)]   # (N, p, S_N)


def _problems():
    from paper_2301_04758_gb300.api import Mesh
    probs = []
    for k, (N, p, sn) in enumerate(SPECS):
        mesh = Mesh(N, N, 3, p, 0.05)
        om, w = level_symmetric(sn)
        st, ss = seeded_media(N * N, 400 + k)
        rng = np.random.default_rng(k)
        phi = rng.uniform(0.5, 1.5, (N * N, (p + 1) ** 2))
        q = np.ones((N * N, (p + 1) ** 2))
        probs.append(dict(mesh=mesh, om=om, w=w, st=dev(st), ss=dev(ss), phi=dev(phi), q=dev(q)))
    return probs


def test_batch_matches_single_sweeps_and_tuning_keeps_results(lib):
    from paper_2301_04758_gb300.api import Batch
    probs = _problems()
    single = [P["mesh"].sweep(P["st"], P["ss"], P["om"], P["w"], phi_in=P["phi"], source=P["q"]) for P in probs]
    single = [host(x) for x in single]
    batch = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    args = ([P["st"] for P in probs], [P["ss"] for P in probs])
    kw = dict(phi_in=[P["phi"] for P in probs], source=[P["q"] for P in probs])
    out, info = batch.sweep(*args, info=True, **kw)
    assert info["timed_out"] == 0
    for a, b in zip(out, single):
        assert rel(host(a), b) < 1e-15
    tiles = batch.tune()
    assert set(tiles) == {1, 2, 3, 4}
    out2 = batch.sweep(*args, **kw)
    torch.cuda.synchronize()
    for a, b in zip(out2, single):
        assert rel(host(a), b) < 1e-15


def test_mixed_order_batch_and_graph_replay_match_the_oracle(lib):
    """A batch of three problems of different DG order and direction set (Q1 S4 4x4, Q3 S8
    6x5, Q2 S6 5x7 on sine-curved Q3 maps, each with its own seeded media, phi_in, source
    and inflow) swept in one call and replayed from a CUDA graph: every problem's psi
    matches the FP64 oracle within 1e-12 relative L2."""
    from paper_2301_04758_gb300.api import Mesh, Batch
    from oracle.transport import Discretization, sweep as o_sweep
    specs = [(4, 4, 1, 4), (6, 5, 3, 8), (5, 7, 2, 6)]
    probs, refs = [], []
    for k, (nx, ny, p, sn) in enumerate(specs):
        om, w = level_symmetric(sn)
        E, n, nq = nx * ny, (p + 1) ** 2, p + 2
        st, ss = seeded_media(E, 700 + k)
        rng = np.random.default_rng(710 + k)
        phi = rng.uniform(0.5, 1.5, (E, n))
        q = rng.uniform(0.0, 1.0, (E, n))
        inflow = rng.uniform(0.0, 1.0, (len(w), 2 * nx + 2 * ny, nq))
        disc = Discretization(nx, ny, 3, 0.05, p)
        refs.append(o_sweep(disc, om, w, st, ss, phi_in=phi, source=q, inflow=inflow))
        probs.append(dict(mesh=Mesh(nx, ny, 3, p, 0.05), om=om, w=w, st=dev(st), ss=dev(ss), phi=dev(phi),
                          q=dev(q), inflow=dev(inflow)))
    batch = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    args = ([P["st"] for P in probs], [P["ss"] for P in probs])
    kw = dict(phi_in=[P["phi"] for P in probs], source=[P["q"] for P in probs],
              inflow=[P["inflow"] for P in probs])
    psi, info = batch.sweep(*args, info=True, **kw)
    assert info["timed_out"] == 0
    for a, ref in zip(psi, refs):
        assert rel(host(a), ref) < 1e-12
    for a in psi:
        a.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.sweep(*args, psi=psi, stream=s, **kw)
    g.replay()
    torch.cuda.synchronize()
    for a, ref in zip(psi, refs):
        assert rel(host(a), ref) < 1e-12


def test_tuner_cache_and_factor_reuse(lib, tmp_path, monkeypatch):
    """With VEF_TUNE_CACHE set, the tuner's choices go to the file, a new batch of the same
    problems reads them back (an order found there is not timed again, so edited choices
    come back as written), every form reproduces the single sweeps, and a sweep keeping the
    previous factorisation (sigma_t unchanged) gives the same psi."""
    from paper_2301_04758_gb300.api import Batch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("VEF_TUNE_CACHE", str(cache))
    probs = _problems()
    single = [host(P["mesh"].sweep(P["st"], P["ss"], P["om"], P["w"], phi_in=P["phi"], source=P["q"]))
              for P in probs]
    args = ([P["st"] for P in probs], [P["ss"] for P in probs])
    kw = dict(phi_in=[P["phi"] for P in probs], source=[P["q"] for P in probs])
    batch = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    batch.sweep(*args, **kw)
    tiles = batch.tune()
    lines = [l.split() for l in cache.read_text().splitlines()]
    assert len(lines) == 4 and sorted(int(t) for _, t in lines) == sorted(tiles.values())
    # rewrite every choice: the single-CTA form for p = 1, 2, a cluster shape for p = 3, 4
    want = {}
    with open(cache, "w") as f:
        for key, _ in lines:
            p = int(key.split("-p")[-1].split("-")[0])
            want[p] = 1 if p <= 2 else 204
            f.write(f"{key} {want[p]}\n")
    batch2 = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    out = batch2.sweep(*args, **kw)
    assert batch2.tune() == want
    out_reuse = batch2.sweep(*args, reuse=True, **kw)
    torch.cuda.synchronize()
    for a, r, b in zip(out, out_reuse, single):
        assert rel(host(a), b) < 1e-15 and rel(host(r), b) < 1e-15
    assert len(cache.read_text().splitlines()) == 4   # nothing re-timed, nothing appended


def test_tuning_right_after_an_unsynchronised_sweep(lib):
    """The first batched sweep returns without synchronising and the tuner starts at once:
    the argument tables still being copied for that sweep must not change under it, and
    every later sweep must reproduce the single-problem sweeps."""
    from paper_2301_04758_gb300.api import Mesh, Batch
    specs = [(48, 3, 12), (40, 4, 8), (64, 2, 16), (56, 1, 6)]
    probs = []
    for k, (N, p, sn) in enumerate(specs):
        mesh = Mesh(N, N, 3, p, 0.05)
        om, w = level_symmetric(sn)
        st, ss = seeded_media(N * N, 500 + k)
        probs.append(dict(mesh=mesh, om=om, w=w, st=dev(st), ss=dev(ss),
                          q=dev(np.ones((N * N, (p + 1) ** 2)))))
    single = [host(P["mesh"].sweep(P["st"], P["ss"], P["om"], P["w"], source=P["q"])) for P in probs]
    batch = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    args = ([P["st"] for P in probs], [P["ss"] for P in probs])
    psi = batch.sweep(*args, source=[P["q"] for P in probs])        # no info: returns at once
    batch.tune()
    for _ in range(2):
        batch.sweep(*args, source=[P["q"] for P in probs], psi=psi)
    torch.cuda.synchronize()
    for a, b in zip(psi, single):
        assert rel(host(a), b) < 1e-15


def test_batch_sweep_replays_from_a_cuda_graph(lib):
    from paper_2301_04758_gb300.api import Batch
    probs = _problems()
    batch = Batch([P["mesh"] for P in probs], [P["om"] for P in probs], [P["w"] for P in probs])
    args = ([P["st"] for P in probs], [P["ss"] for P in probs])
    kw = dict(phi_in=[P["phi"] for P in probs], source=[P["q"] for P in probs])
    psi = batch.sweep(*args, **kw)              # first call allocates
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.sweep(*args, psi=psi, stream=s, **kw)
    # new cross sections, replay, compare with a direct call
    for P in probs:
        P["st"].mul_(1.5)
    g.replay()
    torch.cuda.synchronize()
    got = [host(x).copy() for x in psi]
    ref = batch.sweep(*args, **kw)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert rel(a, host(b)) < 1e-15


def test_source_iteration_replays_from_a_cuda_graph(lib):
    from paper_2301_04758_gb300.api import Mesh
    om, w = level_symmetric(8)
    N, p = 24, 2
    mesh = Mesh(N, N, 3, p, 0.05)
    st, ss = seeded_media(N * N, 2)
    st, ss = dev(st), dev(ss)
    q = dev(np.ones((N * N, 9)))
    phi, psi, dphi = mesh.source_iterate(st, ss, om, w, 4, source=q)
    ref = host(phi).copy()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out = mesh.source_iterate(st, ss, om, w, 4, source=q, psi=psi, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert rel(host(out[0]), ref) < 1e-15
