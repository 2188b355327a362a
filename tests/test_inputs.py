"""The seeded input generators shared by the oracle tests, the GPU tests and the bench:
reproducible, inside the stated ranges, and shaped like the named workloads."""
import numpy as np
import pytest

from vef_inputs import WORKLOADS, config_workload, level_symmetric, seeded_media
from vef_inputs.media import batch_problem


def test_seeded_media_is_reproducible_and_in_range():
    st, ss = seeded_media(4096, 2)
    st2, ss2 = seeded_media(4096, 2)
    assert np.array_equal(st, st2) and np.array_equal(ss, ss2)
    assert not np.array_equal(st, seeded_media(4096, 3)[0])
    assert st.dtype == np.float64 and st.shape == (4096,)
    assert st.min() >= 0.1 and st.max() <= 100.0
    c = ss / st
    assert c.min() >= 0.9 and c.max() <= 0.9999
    # sigma_t spans the decades evenly: about a third of the draws per decade
    counts = np.histogram(np.log10(st), bins=[-1, 0, 1, 2])[0]
    assert np.all(np.abs(counts / 4096 - 1 / 3) < 0.05)


@pytest.mark.parametrize("name,E,D,n", [("tiny_straight_q1_s4", 64, 12, 4), ("sine256_q2_s8", 65536, 40, 9),
                                        ("sine512_q3_s12", 262144, 84, 16),
                                        ("sine128_q2_s8_adjoint", 16384, 40, 9)])
def test_named_workloads(name, E, D, n):
    wl = config_workload(name)
    assert (wl["E"], wl["D"], wl["n"]) == (E, D, n)
    assert wl["omega"].shape == (D, 2) and wl["weights"].shape == (D,)
    assert wl["sigma_t"].shape == (E,) and wl["source"].shape == (E, n)
    np.testing.assert_allclose(wl["weights"].sum(), 4 * np.pi, rtol=1e-14)
    assert np.all(wl["sigma_s"] < wl["sigma_t"])
    assert set(WORKLOADS) >= {name}


def test_batch_problems_cover_sizes_orders_and_quadratures():
    probs = [batch_problem(k) for k in range(64)]
    assert {p["nx"] for p in probs} == {16, 32, 64, 128, 256}
    assert {p["p"] for p in probs} == {1, 2, 3, 4}
    assert {p["sn"] for p in probs} == {4, 6, 8, 12, 16}
    assert len({p["media"][1] for p in probs}) == 64        # one seed per problem
    # each DG order meets four of the five quadratures, so every per-order launch mixes
    # direction counts (and mesh sizes)
    for order in (1, 2, 3, 4):
        same = [p for p in probs if p["p"] == order]
        assert len({p["sn"] for p in same}) == 4 and len({p["nx"] for p in same}) >= 4


def test_level_symmetric_direction_counts():
    for N, D in ((4, 12), (6, 24), (8, 40), (12, 84), (16, 144)):
        om, w = level_symmetric(N)
        assert om.shape == (D, 2) and np.all(w > 0)
        assert np.all(np.hypot(om[:, 0], om[:, 1]) < 1.0)    # projections of xi > 0 directions
