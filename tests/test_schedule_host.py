"""The sweep's dependency scheduler on the host (vef_schedule_host, no GPU): wavefronts on
straight meshes, the Omega . n = 0 convention, a planted two-element cycle, and on randomly
tilted face normals the strongly connected components and levels of an independent graph
library."""
import ctypes

import numpy as np
import pytest

from vef_inputs import level_symmetric


def _lib():
    from paper_2301_04758_gb300 import _lib
    return _lib, _lib.load()


def _straight_nds(nx, ny, p):
    """Outward n ds of the unit square cut into nx x ny rectangles, at p + 2 points per face;
    faces 0..3 towards j-1, i+1, j+1, i-1."""
    nq = p + 2
    hx, hy = 1.0 / nx, 1.0 / ny
    face = np.array([[0.0, -hx], [hy, 0.0], [0.0, hx], [-hy, 0.0]])
    return np.ascontiguousarray(np.broadcast_to(face[None, :, None, :], (nx * ny, 4, nq, 2)))


def _schedule(nx, ny, p, nds, omega):
    _l, lib = _lib()
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    D, E = len(omega), nx * ny
    levels = np.zeros(D, np.int32)
    groups = np.zeros(D, np.int64)
    level = np.zeros((D, E), np.int32)
    size = np.zeros((D, E), np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = lib.vef_schedule_host(nx, ny, p, ptr(nds), ptr(omega), D, ptr(levels), ptr(groups), ptr(level), ptr(size))
    assert st == _l.VEF_OK, lib.vef_last_error()
    return levels, groups, level, size


def test_straight_mesh_gives_the_quadrant_wavefront():
    nx, ny, p = 7, 4, 2
    om, _ = level_symmetric(4)
    levels, groups, level, size = _schedule(nx, ny, p, _straight_nds(nx, ny, p), om)
    e = np.arange(nx * ny)
    i, j = e % nx, e // nx
    for d, (mu, eta) in enumerate(om):
        key = (i if mu > 0 else nx - 1 - i) + (j if eta > 0 else ny - 1 - j)
        assert levels[d] == nx + ny - 1 and groups[d] == 0
        assert np.array_equal(level[d], key) and np.all(size[d] == 1)


def test_faces_parallel_to_the_direction_couple_nothing():
    """Omega . n = 0 on the faces parallel to an axis-aligned direction: neither inflow nor
    outflow, so each row (column) of elements is an independent chain."""
    nx, ny, p = 5, 3, 1
    om = np.array([[1.0, 0.0], [0.0, -1.0]])
    levels, groups, level, _ = _schedule(nx, ny, p, _straight_nds(nx, ny, p), om)
    e = np.arange(nx * ny)
    assert levels.tolist() == [nx, ny] and groups.tolist() == [0, 0]
    assert np.array_equal(level[0], e % nx)
    assert np.array_equal(level[1], ny - 1 - e // nx)


def test_planted_two_element_cycle_becomes_one_group():
    """Tilt the face shared by elements 0 and 1 of a 3 x 1 row so that it is inflow for
    element 0 at one Gauss point and for element 1 at the others: the two form one coupled
    group at level 0 and element 2, downstream, comes next."""
    nx, ny, p = 3, 1, 1
    nds = _straight_nds(nx, ny, p).copy()
    tilt = np.array([[1.0, -20.0], [1.0, 0.0], [1.0, 0.0]])   # Omega . v = -1.2, 0.8, 0.8
    nds[0, 1] = tilt
    nds[1, 3] = -tilt
    levels, groups, level, size = _schedule(nx, ny, p, nds, [[0.8, 0.1]])
    assert levels[0] == 2 and groups[0] == 1
    assert size[0].tolist() == [2, 2, 1] and level[0].tolist() == [0, 0, 1]


def test_random_tilts_match_an_independent_graph_library():
    nx_ = pytest.importorskip("networkx")
    nx, ny, p = 9, 7, 2
    nq, E = p + 2, nx * ny
    rng = np.random.default_rng(17)
    nds = _straight_nds(nx, ny, p).copy()
    nds += rng.normal(0.0, 0.03, nds.shape)   # ~25 % of h: many small groups, 15-22 levels
    for e in range(E):   # shared faces carry one n ds, seen with opposite signs from each side
        i, j = e % nx, e // nx
        if i + 1 < nx:
            nds[e + 1, 3] = -nds[e, 1]
        if j + 1 < ny:
            nds[e + nx, 0] = -nds[e, 2]
    om, _ = level_symmetric(8)
    levels, groups, level, size = _schedule(nx, ny, p, nds, om)
    nb = lambda e, f: [e - nx if e >= nx else -1, e + 1 if e % nx < nx - 1 else -1,
                       e + nx if e < E - nx else -1, e - 1 if e % nx > 0 else -1][f]
    assert groups.sum() > 100 and size.max() > 2 and levels.min() > 10   # cycles, yet a deep DAG
    for d, o in enumerate(om):
        g = nx_.DiGraph()
        g.add_nodes_from(range(E))
        for e in range(E):
            for f in range(4):
                w = nb(e, f)
                if w >= 0 and np.any(nds[e, f] @ o > 0.0):   # e has outflow into w
                    g.add_edge(e, w)
        comps = list(nx_.strongly_connected_components(g))
        cid = {e: k for k, c in enumerate(comps) for e in c}
        assert [len(comps[cid[e]]) for e in range(E)] == size[d].tolist()
        assert groups[d] == sum(len(c) > 1 for c in comps)
        cg = nx_.condensation(g, comps)
        lev = {}
        for c in nx_.topological_sort(cg):
            lev[c] = max((lev[u] + 1 for u in cg.predecessors(c)), default=0)
        assert [lev[cid[e]] for e in range(E)] == level[d].tolist()
        assert levels[d] == max(lev.values()) + 1


def test_arguments_are_checked():
    _l, lib = _lib()
    nds = _straight_nds(2, 2, 1)
    om = np.array([[0.5, 0.5]])
    out = np.zeros(4, np.int64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.vef_schedule_host(2, 2, 0, ptr(nds), ptr(om), 1, ptr(out), ptr(out), None, None) == _l.VEF_ERR_INVALID_ARG
    assert lib.vef_schedule_host(2, 2, 1, ptr(nds), ptr(om), 0, ptr(out), ptr(out), None, None) == _l.VEF_ERR_INVALID_ARG
    assert lib.vef_schedule_host(2, 2, 1, None, ptr(om), 1, ptr(out), ptr(out), None, None) == _l.VEF_ERR_INVALID_ARG
    assert lib.vef_schedule_host(0, 2, 1, ptr(nds), ptr(om), 1, ptr(out), ptr(out), None, None) == _l.VEF_ERR_INVALID_ARG


def test_degenerate_meshes_and_the_largest_direction_set():
    """One element: one level for every direction.  A 1 x 9 strip: the sweep runs along
    the strip, so a direction going up or down has 9 levels.  1023 directions (the most a
    call takes) on a 4 x 3 straight mesh: every one a quadrant wavefront or, on an axis,
    a chain."""
    rng = np.random.default_rng(5)
    ph = rng.uniform(0.0, 2 * np.pi, 1023)
    r = np.sqrt(rng.uniform(0.0, 1.0, 1023))
    om = np.stack([r * np.cos(ph), r * np.sin(ph)], axis=1)
    levels, groups, _, _ = _schedule(1, 1, 3, _straight_nds(1, 1, 3), om[:5])
    assert levels.tolist() == [1] * 5 and groups.tolist() == [0] * 5
    levels, groups, level, _ = _schedule(1, 9, 1, _straight_nds(1, 9, 1), [[0.3, 0.7], [0.3, -0.7]])
    assert levels.tolist() == [9, 9] and level[0].tolist() == list(range(9))
    assert level[1].tolist() == list(range(8, -1, -1))
    levels, groups, _, _ = _schedule(4, 3, 4, _straight_nds(4, 3, 4), om)
    assert np.all(levels == 6) and np.all(groups == 0)
