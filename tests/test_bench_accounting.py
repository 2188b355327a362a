"""bench.py's work model and roofline arithmetic, on the host (no GPU).

The per-unit counts are the ones the bench line's roofline divides by; the event times
below are a 256x256 Q2 S8 run's per-class totals over 5 timed steps of 10 source
iterations (FP64: 1 factorisation + 10 fused apply-and-sweep launches per step; mixed: 21
FP32 sweeps and 21 FP64 residuals per step), and a 512x512 Q3 S12 run's over 3 steps of
one inversion, so the reported fractions can be checked by hand.
"""
import pytest

import bench

E, D, P = 256 * 256, 40, 2
PROF64 = {"factor": (5, 40.78), "sweep": (50, 121.40), "source": (150, 5.47), "moments": (15, 3.21)}
PROF32 = {"factor": (10, 34.56), "sweep": (105, 178.10), "residual": (105, 78.15), "source": (255, 15.39)}


def test_per_unit_work_at_p2():
    n = 9
    assert bench.flops_sweep(P) == 2 * 2 * n * 3 == 108
    assert bench.flops_apply(P) == 2 * n * n == 162
    # record prefix 16 + 2 W slots of 9x3 doubles (448 after padding), y row 72 -> 80,
    # 16 bytes of slot ids, psi 72
    assert bench.bytes_sweep(P) == 448 + 80 + 16 + 72 == 616
    assert bench.bytes_apply(P, D) == pytest.approx(648 + 80 + 72 / D)
    # FP32: the same counts in 4-byte words (232 -> 240, 36 -> 48)
    assert bench.bytes_sweep(P, word=4) == 240 + 48 + 16 + 36
    assert bench.flops_residual(P) == 2 * 81 + 4 * 9 + 36
    assert bench.bytes_residual(P, D) == pytest.approx(8 * 117 + 72 + 48 + 72 / D + 72)
    assert bench.flops_factor(P) == 2845


def test_roofline_report_by_hand():
    roof, main, roof32, main32 = bench.roofline_report(PROF64, PROF32, P, D, E, 5, 10, 6792.4, 1053.9,
                                                       traffic_of=lambda k: 123.0)
    units = E * D
    # FP64 sweep launch: (108 + 162) flop per unit over 121.40 / 50 ms, against 1258.56 GFLOP/s
    t = 121.40 / 50 * 1e-3
    assert main["kernel"] == "sweep" and main["bound"] == "alu" and main["traffic"] == 123.0
    assert main["achieved"] == pytest.approx(270 * units / t / 1e12, rel=1e-3)
    assert main["frac"] == pytest.approx(270 * units / t / 1.25856e12, rel=1e-3)
    assert main["peak_measured_fma_tflops"] == pytest.approx(1.0539, abs=1e-4)
    assert roof["factor"]["bound"] == "alu"
    # mixed: the FP32 sweep is bound by its bytes; 105 - 50 of its launches are corrections
    corr = 55 / 105
    by = (340 + (324 + 48 + 72 / D) + corr * 72 * (1 - 1 / D)) * units
    t32 = 178.10 / 105 * 1e-3
    assert main32["kernel"] == "sweep" and main32["bound"] == "hbm" and main32["traffic"] is None
    assert main32["achieved"] == pytest.approx(by / t32 / 1e9, rel=1e-3)
    assert main32["frac"] == pytest.approx(by / t32 / 1e9 / 6792.4, rel=1e-3)
    assert roof32["residual"]["bound"] == "alu" and roof32["residual"]["peak"] == pytest.approx(1.25856)


def test_classes_without_launches_are_left_out():
    roof, main, roof32, main32 = bench.roofline_report({"sweep": (0, 0.0)}, {}, P, D, E, 1, 10, 6792.4, 1e3,
                                                       traffic_of=lambda k: None)
    assert roof == {} and main is None and roof32 == {} and main32 is None


def test_per_unit_work_at_p3_single_inversion():
    n, q, nq = 16, 4, 5
    assert bench.flops_residual_mf(3) == 6 * n * n + 3 * n + 4 * nq * (4 + 2 * q) + 4 * q * 2 * nq + 4 * n == 2048
    assert bench.bytes_residual_mf(3, 84) == pytest.approx(8 * n + 2 * 8 * q + 8 * n + (3 * 8 * n * n + 8 * 40 + 8 * n) / 84)
    assert bench.flops_factor(3) == 11728
    assert bench.bytes_factor(3, 84) == pytest.approx(8 * 3 * n * n / 84 + 16 + 8 * (n * n + 2 * n * q))


def test_roofline_of_a_single_inversion_step():
    """512^2 Q3 S12, one inversion per step: the FP64 step is dominated by the factorisation
    (reported against the FP64 ALU peak); the mixed step's residual is the matrix-free form."""
    E3, D3, P3 = 512 * 512, 84, 3
    prof64 = {"factor": (3, 888.3), "sweep": (3, 99.1), "group": (3, 30.0), "moments": (9, 22.7)}
    prof32 = {"factor": (3, 75.0), "sweep": (6, 80.0), "residual": (3, 150.0), "moments": (9, 22.7)}
    roof, main, roof32, main32 = bench.roofline_report(prof64, prof32, P3, D3, E3, 3, 1, 6792.4, 1053.9,
                                                       traffic_of=lambda k: None)
    units = E3 * D3
    assert main["kernel"] == "factor" and main["bound"] == "alu"
    # a single inversion's factorisation also forms y = A^{-1} b: + 2 n^2 = 512 flop
    assert main["achieved"] == pytest.approx((11728 + 512) * units / (888.3 / 3 * 1e-3) / 1e12, rel=1e-3)
    assert roof["sweep"]["flops_per_launch"] == bench.flops_sweep(P3) * units
    assert "group" not in roof                    # no work model: never the reported kernel
    # 6 FP64 FMAs per psi value: far above GB300's FP64 ridge (~0.19 flop/B), so ALU-bound
    assert bench.flops_moments(P3, D3) == pytest.approx(12 * 16 + 25 * (8 * 16 + 3) / D3)
    assert roof["moments"]["bound"] == "alu"
    assert main32["kernel"] == "residual" and main32["bound"] == "alu"
    assert main32["achieved"] == pytest.approx(2048 * units / (150.0 / 3 * 1e-3) / 1e12, rel=1e-3)
    # FP32 factorisation: 11728 flop at the FP32 peak take less time than writing its
    # ~1.6 KB record at the HBM rate, so it is bound by the record bytes
    assert roof32["factor"]["bound"] == "hbm" and roof32["factor"]["peak"] == pytest.approx(6792.4)


def test_committed_traffic_summaries_parse():
    """The DRAM-traffic summaries behind roofline.traffic list their kernel class with a
    workload and a source hash in the form src_hash() produces."""
    import os
    for kernel, name in bench.TRAFFIC_FILES.items():
        path = os.path.join(os.path.dirname(bench.__file__), "profiles", name)
        if not os.path.exists(path):
            continue
        rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
        mine = [r for r in rows if r[0] == kernel]
        assert mine and all(r[1] in bench.BENCH_WORKLOADS for r in mine)
        for r in mine:
            assert float(r[2]) > 0 and len(r[3]) == len(bench.src_hash(kernel))
