"""bench.py's work model and roofline arithmetic, on the host (no GPU).

The per-unit counts are the ones the bench line's roofline divides by; the event times
below are a 256x256 Q2 S8 run's per-class totals over 5 timed steps (FP64: 1 factorisation
+ 10 fused apply-and-sweep launches per step; mixed: 21 FP32 sweeps and 21 FP64
residuals per step), so the reported fractions can be checked by hand.
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
    roof, main, roof32, main32 = bench.roofline_report(PROF64, PROF32, P, D, E, 5, 6792.4, 1053.9,
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
    roof, main, roof32, main32 = bench.roofline_report({"sweep": (0, 0.0)}, {}, P, D, E, 1, 6792.4, 1e3,
                                                       traffic_of=lambda k: None)
    assert roof == {} and main is None and roof32 == {} and main32 is None


def test_committed_traffic_summary_parses():
    """The DRAM-traffic summary behind roofline.traffic lists the sweep launch of the bench
    workload with a source hash in the form src_hash() produces."""
    import os
    path = os.path.join(os.path.dirname(bench.__file__), "profiles",
                        "sweep_cta_kernel_dram_traffic_sine128_q2_s8.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    sweep = [r for r in rows if r[0] == "sweep" and r[1] == bench.WORKLOAD]
    assert len(sweep) == 1
    assert float(sweep[0][2]) > 0 and len(sweep[0][3]) == len(bench.src_hash("sweep"))
