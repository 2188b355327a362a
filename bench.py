#!/usr/bin/env python
"""Benchmark: DG S_N sweep + VEF closure pass on one GB300 (or N replicas).

Default workload (one "step"): the 512 x 512 sine-curved (alpha = 0.05, third-order map)
mesh of [0,1]^2, DG Q3, level-symmetric S12 (84 directions), per-element sigma_t
log-uniform in [0.1, 100] and sigma_s/sigma_t uniform in [0.9, 0.9999] (seed 3),
isotropic source 1, vacuum inflow: one transport inversion (local factorisation of every
(element, direction) system, then the wavefront sweep) followed by the closure pass (phi,
J, E, E_b, J_in).  Metric: angular-DOF updates per second = E (p+1)^2 D / step time, in
FP64 (`value`) and in mixed precision beside it (`mixed`: FP32 factorisation and sweeps
inside FP64 defect correction, two passes), with the mixed path's psi / phi / J / E / E_b
errors against FP64.  Inputs live in HBM for `value`; `e2e` adds the host->device copy
of the step's inputs and the device->host copy of its outputs through the same C-ABI
calls.  `--workload sine256_q2_s8` runs the 256 x 256 Q2 S8 source-iteration workload
(10 inversions per step) instead.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# workloads this script times: (transport inversions per step, description)
BENCH_WORKLOADS = {
    "sine512_q3_s12": (1, "512x512 sine-curved Q3 mesh (alpha 0.05), DG Q3, S12 (84 dirs), seeded "
                          "sigma_t/sigma_s (seed 3), q=1, vacuum; one transport inversion (local "
                          "factorisation + sweep) + closures per step"),
    "sine256_q2_s8": (10, "256x256 sine-curved Q3 mesh (alpha 0.05), DG Q2, S8 (40 dirs), seeded "
                          "sigma_t/sigma_s (seed 2), q=1, vacuum; 10 source iterations (one "
                          "factorisation, 10 sweeps) + closures per step"),
}
WORKLOAD = "sine512_q3_s12"
# the headline: FP64 throughput of the whole step, the mixed-precision step beside it with
# its errors against FP64, and each path's roofline
METRIC = "sweep angular-DOF updates/s, mixed vs FP64 at phi,E rel.err<=1e-10; % roofline"
MIXED_ERR_BOUND = 1e-10
MIXED_PASSES = 2
# FP64 peak from unit counts: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2070 MHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=WORKLOAD, choices=tuple(BENCH_WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-only", type=int, default=0, metavar="NX",
                    help="profiling driver: build an NX x NX mesh with the workload's recipe and run "
                         "--steps sweeps (factorisation included); prints the wall time and the "
                         "per-kernel-class times of the calls after the first")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="NX",
                    help="profiling driver: the adjoint workload's recipe on an NX x NX mesh, one forward "
                         "sweep, then --steps adjoint sweeps (no timing line)")
    ap.add_argument("--order", type=int, default=2, help="--sweep-only: DG order p")
    ap.add_argument("--sn", type=int, default=8, help="--sweep-only: level-symmetric order N")
    ap.add_argument("--seed", type=int, default=2, help="--sweep-only: media seed")
    ap.add_argument("--precision", default="fp64", choices=("fp64", "mixed"), help="--sweep-only: precision")
    ap.add_argument("--apply", default="fused", choices=("fused", "separate"),
                    help="--sweep-only: y = A^-1 b inside the sweep launch or as its own launch")
    ap.add_argument("--suite", default="", choices=("", "batch", "adjoint", "hrt", "vef"),
                    help="other workloads (one JSON line each, not the headline): batch = the "
                         "64-problem batch; adjoint = 128x128 Q2 S8 adjoint gradients with a "
                         "central-difference check; hrt = the hybridized RT VEF solve after a "
                         "128x128 Q2 S8 sweep; vef = the VEF fixed-point iteration on a 64x64 "
                         "thick-diffusion-limit problem")
    ap.add_argument("--mixed-tol", type=float, default=-1.0,
                    help="mixed precision: relative residual target of the defect correction, or < 0 "
                         "for a fixed %d passes" % MIXED_PASSES)
    ap.add_argument("--cpu-sample", type=int, default=64, metavar="NX",
                    help="mesh size of the oracle's bounded CPU sample (the workload's recipe)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ accounting
def flops_factor(p, inflow_faces=2.0):
    """Algorithmic flops of one (element, direction) factorisation (FMA = 2 flops):
    assembly sigma_t M - mu Gx - eta Gy (5 n^2), four faces' outflow/inflow face
    matrices (4 [4 nq + 5 (p+1)^2 nq + (p+1)^2]), in-place Gauss-Jordan inversion
    (n [(n-1) + (n-1)(2n-1)]) and W_f = A^{-1} Cin_f per interior inflow face (2 n (p+1)^2)."""
    n, q, nq = (p + 1) ** 2, p + 1, p + 2
    return (5 * n * n + 4 * (4 * nq + 5 * q * q * nq + q * q)
            + n * ((n - 1) + (n - 1) * (2 * n - 1)) + inflow_faces * 2 * n * q * q)


def flops_apply(p):
    """Per (element, direction) flops of the dependency-free apply: y = A^{-1} b (2 n^2)."""
    n = (p + 1) ** 2
    return 2 * n * n


def bytes_apply(p, D, word=8):
    """Per (element, direction) apply bytes: A^{-1} read, y row written (16-byte padded),
    the direction-independent rhs read once per element (/ D)."""
    n = (p + 1) ** 2
    pad = lambda b: (b + 15) // 16 * 16
    return word * n * n + pad(word * n) + 8 * n / D


def flops_sweep(p, inflow_faces=2.0):
    """Per (element, direction) sweep flops: psi = y - sum_f W_f u_f (2 n (p+1) per
    interior inflow face)."""
    n = (p + 1) ** 2
    return inflow_faces * 2 * n * (p + 1)


def bytes_sweep(p, word=8, inflow_faces=2.0):
    """Per (element, direction) sweep DRAM bytes of the single-CTA sweep: the staged record
    prefix (16 bytes of element info + two W slots), the padded y row, the 16 bytes of
    trace-slot ids, and psi written (the upwind face values pass through shared memory;
    inflow_faces is kept for the flop count's signature)."""
    n = (p + 1) ** 2
    pad = lambda b: (b + 15) // 16 * 16
    return pad(16 + 2 * word * n * (p + 1)) + pad(word * n) + 16 + word * n


def flops_residual(p):
    """Per (element, direction) flops of the FP64 residual r = b - L psi (mixed path): the
    element matrix times psi (2 n^2), the upwind couplings of two interior inflow faces
    (2 x 2 (p+1)^2) and the two squared norms (4 n)."""
    n, q = (p + 1) ** 2, p + 1
    return 2 * n * n + 2 * 2 * q * q + 4 * n


def bytes_residual(p, D):
    """Per (element, direction) bytes of the FP64 residual: the stored FP64 element matrix
    and four face couplings (n^2 + 4 (p+1)^2 words), psi read, the upwind face values of
    two faces, the direction-independent rhs (/ D) and r written."""
    n, q = (p + 1) ** 2, p + 1
    return 8 * (n * n + 4 * q * q) + 8 * n + 2 * 8 * q + 8 * n / D + 8 * n


def flops_residual_mf(p):
    """Per (element, direction) flops of the matrix-free FP64 residual (a single inversion's
    defect correction): the volume operator from M, Gx, Gy (3 n^2 FMAs and their 3 n
    combinations), the 4 (p+2) face points (Omega . n ds: 3, one trace: 2 (p+1), the product:
    1), the face-node rows (4 faces x (p+1) rows x 2 (p+2)) and the two squared norms (4 n)."""
    n, q, nq = (p + 1) ** 2, p + 1, p + 2
    return 6 * n * n + 3 * n + 4 * nq * (4 + 2 * q) + 4 * q * 2 * nq + 4 * n


def bytes_residual_mf(p, D):
    """Per (element, direction) bytes of the matrix-free residual: psi read, two upwind
    faces' node values, r written, and the per-element M, Gx, Gy, normals and right-hand side
    read once per element (/ D)."""
    n, q, nq = (p + 1) ** 2, p + 1, p + 2
    return 8 * n + 2 * 8 * q + 8 * n + (3 * 8 * n * n + 8 * 4 * nq * 2 + 8 * n) / D


def bytes_factor(p, D, word=8):
    """Per (element, direction) bytes of the factorisation: the per-element M, Gx, Gy read
    once per element (/ D), the record written (16 bytes of element info, A^{-1} and two W
    slots)."""
    n, q = (p + 1) ** 2, p + 1
    return 8.0 * 3 * n * n / D + 16 + word * (n * n + 2 * n * q)


def flops_moments(p, D):
    """Per (element, direction) flops of the moment and closure pass: six FP64 FMAs per psi
    value for the nodal phi, J, P (12 n), and, once per element (/ D), the Eddington tensor
    at the (p+2)^2 Gauss points (four interpolations of n terms and three quotients)."""
    n, nq2 = (p + 1) ** 2, (p + 2) ** 2
    return 12 * n + nq2 * (8 * n + 3) / D


def bytes_moments(p, D, nq2=None):
    """Per (element, direction) bytes of the moment and closure pass: psi read once; the
    nodal phi, J, P (six fields) and the Eddington tensor written once per element (/ D)."""
    n = (p + 1) ** 2
    nq2 = nq2 or (p + 2) ** 2
    return 8 * n + (8 * 6 * n + 8 * 3 * nq2) / D


HBM_MEASURED = "MEASURED_PEAKS.json hbm_gbs (measured)"
HBM_FALLBACK = "fallback: 6.8 TB/s, an earlier GB300 copy measurement (MEASURED_PEAKS.json absent)"
FP64_SRC = "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2070 MHz"
FP32_SRC = "derived: 152 SM x 128 FP32 FMA/clk x 2 flop x 2070 MHz"


def roofline_entries(prof, work, units, hbm_gbs, hbm_src=HBM_MEASURED):
    """Roofline of each kernel class from its live CUDA-event times.

    prof: {class: (launches, ms)}; work: {class: (flops per unit, bytes per unit, ALU peak
    in GFLOP/s, how that peak was obtained)}; units: (element, direction) units one launch
    processes.  The bound is whichever of the flops at the ALU peak and the bytes at the
    measured HBM bandwidth takes longer; achieved = that quantity / the average launch time."""
    roof = {}
    for k, (fl_u, by_u, alu_gflops, alu_src) in work.items():
        cnt, tms = prof.get(k, (0, 0.0))
        if not cnt or tms <= 0.0:
            continue
        avg = tms / cnt
        fl, by = fl_u * units, by_u * units
        if fl / (alu_gflops * 1e9) >= by / (hbm_gbs * 1e9):
            r = {"bound": "alu", "achieved": fl / (avg * 1e-3) / 1e12, "peak": alu_gflops / 1e3,
                 "unit": "TFLOP/s", "peak_source": alu_src}
        else:
            r = {"bound": "hbm", "achieved": by / (avg * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                 "peak_source": hbm_src}
        r.update(frac=r["achieved"] / r["peak"], avg_ms=avg, flops_per_launch=fl, bytes_per_launch=by,
                 tflops=fl / (avg * 1e-3) / 1e12, gbps=by / (avg * 1e-3) / 1e9)
        roof[k] = r
    return roof




SWEEP_REGION = ("// upwind correction of row i for face f of member record r",
                "// -------------------------------------------------------------- FP64 residual (mixed)")
# committed ncu summaries of DRAM traffic per kernel class: lines
#   <class> <workload> <bytes per launch at the workload's full size> <source hash>
TRAFFIC_FILES = {"sweep": "sweep_cta_kernel_dram_traffic_sine128_q2_s8.txt",
                 "factor": "factor_elem_kernel_dram_traffic_sine96_q3_s12.txt"}


def src_hash(kernel):
    """Hash of the source a kernel is built from (its region of sweep.cu plus device.cuh for
    the sweep; its files for the factorisation)."""
    csrc = os.path.join(ROOT, "paper_2301_04758_gb300", "csrc")
    h = hashlib.sha256()
    if kernel == "sweep":
        src = open(os.path.join(csrc, "sweep.cu")).read()
        a, b = src.index(SWEEP_REGION[0]), src.index(SWEEP_REGION[1])
        h.update(src[a:b].encode())
        h.update(open(os.path.join(csrc, "device.cuh"), "rb").read())
    else:
        for nm in ("factor_impl.cuh", "device.cuh"):
            h.update(open(os.path.join(csrc, nm), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, workload=None):
    """DRAM bytes per launch from the committed ncu summary of that kernel class on the
    workload, if the kernel source is unchanged since the capture (else None)."""
    workload = workload or WORKLOAD
    name = TRAFFIC_FILES.get(kernel)
    path = os.path.join(ROOT, "profiles", name) if name else None
    if not path or not os.path.exists(path):
        return None
    want = src_hash(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
            return float(parts[2]) if parts[3] == want else None
    return None


# ----------------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = [l.strip().split(",") for l in open(self.tmp.name) if l.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], 0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------------- our arm
def max_over_ranks(values, world, device="cpu"):
    """Each timing's maximum over the ranks (one all-reduce of the list); the identity on
    one rank.  Every rank runs its own replica of the workload, so the job takes as long
    as its slowest rank."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def job_rate(units_per_step, steps, ms, world):
    """Whole-job throughput: `world` replicas each process `units_per_step` per step, and
    `ms` (the maximum over the ranks) covers `steps` steps."""
    return world * units_per_step * steps / (ms * 1e-3)


def dominant_roofline(prof, roof, traffic_of):
    """The bench line's roofline object: the kernel class with the most event time among
    those with a work model, its DRAM traffic per launch from traffic_of (or None)."""
    timed = [k for k in roof if prof.get(k, (0, 0.0))[0]]
    if not timed:
        return None
    k = max(timed, key=lambda c: prof[c][1])
    r = roof[k]
    return {"bound": r["bound"], "achieved": round(r["achieved"], 4), "peak": round(r["peak"], 4),
            "unit": r["unit"], "frac": round(r["frac"], 4), "traffic": traffic_of(k), "kernel": k,
            "peak_source": r["peak_source"]}


def roofline_report(prof64, prof32, p, D, E, steps, K, hbm_gbs, fp64_meas_gflops, traffic_of=None,
                    hbm_src=HBM_MEASURED, residual_stored=None):
    """Rooflines of the FP64 and the mixed step from their per-class (launches, ms) event
    times over `steps` timed steps of K transport inversions each: returns (FP64 per-class
    entries, FP64 dominant, mixed per-class entries, mixed dominant).  The mixed residual is
    the stored-system form under source iteration (K > 1), else the matrix-free form."""
    n = (p + 1) ** 2
    traffic_of = traffic_of or ncu_traffic
    if residual_stored is None:
        residual_stored = K > 1
    # y = A^{-1} b: for a single inversion (K == 1) the factorisation forms it (2 n^2 flop and
    # the y row written); under source iteration the sweep launch applies A^{-1} on the SMs
    # its directions leave free, and the work counts with the sweep
    fused = K == 1
    ypad = (8 * n + 15) // 16 * 16
    work = {"factor": (flops_factor(p) + (flops_apply(p) if fused else 0),
                       bytes_factor(p, D) + (ypad if fused else 0), FP64_PEAK_GFLOPS, FP64_SRC),
            "sweep": (flops_sweep(p) + (0 if fused else flops_apply(p)),
                      bytes_sweep(p) + (0 if fused else bytes_apply(p, D)), FP64_PEAK_GFLOPS, FP64_SRC),
            "moments": (flops_moments(p, D), bytes_moments(p, D), FP64_PEAK_GFLOPS, FP64_SRC)}
    roof = roofline_entries(prof64, work, E * D, hbm_gbs, hbm_src)
    roofline = dominant_roofline(prof64, roof, traffic_of)
    if roofline:
        roofline["peak_measured_fma_tflops"] = round(fp64_meas_gflops / 1e3, 4)

    # mixed path: FP32 factorisation and sweeps (one plain sweep per inversion, the rest
    # defect corrections, whose fused apply reads the FP64 residual row of each unit instead
    # of the per-element rhs) and the FP64 residual
    s32 = prof32.get("sweep", (0, 0.0))[0]
    corr = max(s32 - K * steps, 0) / s32 if s32 else 0.0
    res = ((flops_residual(p), bytes_residual(p, D)) if residual_stored
           else (flops_residual_mf(p), bytes_residual_mf(p, D)))
    # mixed: a single inversion's first FP32 sweep has its y from the factorisation; the
    # correction sweeps apply A^{-1} to the residual themselves
    ypad32 = (4 * n + 15) // 16 * 16
    work32 = {"factor": (flops_factor(p) + (flops_apply(p) if fused else 0),
                         bytes_factor(p, D, word=4) + (ypad32 if fused else 0), FP32_PEAK_GFLOPS, FP32_SRC),
              "sweep": (flops_sweep(p) + flops_apply(p) * (corr if fused else 1.0),
                        bytes_sweep(p, word=4) + bytes_apply(p, D, word=4) * (corr if fused else 1.0)
                        + corr * 8.0 * n * (1 - 1 / D),
                        FP32_PEAK_GFLOPS, FP32_SRC),
              "residual": res + (FP64_PEAK_GFLOPS, FP64_SRC),
              "moments": (flops_moments(p, D), bytes_moments(p, D), FP64_PEAK_GFLOPS, FP64_SRC)}
    roof32 = roofline_entries(prof32, work32, E * D, hbm_gbs, hbm_src)
    roofline32 = dominant_roofline(prof32, roof32, lambda k: None)
    return roof, roofline, roof32, roofline32


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2301_04758_gb300 import build as vbuild
    vbuild.build()
    from paper_2301_04758_gb300.api import Mesh, fma_peak
    from vef_inputs import config_workload

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    K, desc = BENCH_WORKLOADS[args.workload]
    wl = config_workload(args.workload)
    om, w = wl["omega"], wl["weights"]
    E, n, D, p = wl["E"], wl["n"], wl["D"], wl["p"]
    updates = E * n * D * K
    mesh = Mesh(wl["nx"], wl["ny"], wl["mesh_order"], p, wl["alpha"])
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev).contiguous()
    st, ss, q = T(wl["sigma_t"]), T(wl["sigma_s"]), T(wl["source"])
    psi = torch.empty(D, E, n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    outputs = ("phi", "J", "E", "Eb", "Jin")
    mixed_kw = (dict(tol=-1.0, max_passes=MIXED_PASSES) if args.mixed_tol < 0
                else dict(tol=args.mixed_tol))

    def step(precision, st_=None, ss_=None, q_=None):
        st_ = st if st_ is None else st_
        ss_ = ss if ss_ is None else ss_
        q_ = q if q_ is None else q_
        kw = mixed_kw if precision == "mixed" else {}
        if K == 1:
            ps = mesh.sweep(st_, ss_, om, w, source=q_, psi=psi, precision=precision, **kw)
        else:
            _, ps, _ = mesh.source_iterate(st_, ss_, om, w, K, source=q_, precision=precision, psi=psi, **kw)
        return mesh.moments(ps, om, w, outputs=outputs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(precision, steps):
        for _ in range(args.warmup):
            step(precision)
        torch.cuda.synchronize()
        mesh.sync()
        mesh.profile(True)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            res = step(precision)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = mesh.profile_read()
        mesh.profile(False)
        mesh.sync()
        return ms, prof, res

    clocks = Clocks(local_rank)
    clocks.start()
    ms64, prof64, res64 = timed("fp64", args.steps)
    clk = clocks.stop()
    res64 = {k: v.clone() for k, v in res64.items()}
    psi64 = psi.clone() if K == 1 else None
    clocks2 = Clocks(local_rank)
    clocks2.start()
    ms32, prof32, res32 = timed("mixed", args.steps)
    clk2 = clocks2.stop()

    # errors of the mixed path against the FP64 path (same inputs), each output separately
    def relerr(a, b):
        return float(torch.linalg.norm((a - b).flatten()) / torch.linalg.norm(b.flatten()))
    mixed_err = {k: relerr(res32[k], res64[k]) for k in ("phi", "J", "E", "Eb")}
    if psi64 is not None:
        mixed_err["psi"] = relerr(psi, psi64)
    del psi64

    # end to end through the public API: pinned host inputs -> device, outputs -> host
    h_st = torch.tensor(wl["sigma_t"], dtype=torch.float64).pin_memory()
    h_ss = torch.tensor(wl["sigma_s"], dtype=torch.float64).pin_memory()
    h_q = torch.tensor(wl["source"], dtype=torch.float64).pin_memory()
    d_st, d_ss, d_q = torch.empty_like(st), torch.empty_like(ss), torch.empty_like(q)
    outs_host = None

    def e2e_step():
        nonlocal outs_host
        d_st.copy_(h_st, non_blocking=True)
        d_ss.copy_(h_ss, non_blocking=True)
        d_q.copy_(h_q, non_blocking=True)
        out = step("fp64", d_st, d_ss, d_q)
        if outs_host is None:
            outs_host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
        for k, v in out.items():
            outs_host[k].copy_(v, non_blocking=True)
        return out

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        out = e2e_step()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = t0.elapsed_time(t1)
    h2d = 8 * (2 * E + E * n)
    d2h = sum(8 * v.numel() for v in out.values())

    ms64, ms32, ms_e2e = max_over_ranks([ms64, ms32, ms_e2e], world, dev)
    steps = args.steps
    value = job_rate(updates, steps, ms64, world)
    mixed_value = job_rate(updates, steps, ms32, world)
    e2e_value = job_rate(updates, steps, ms_e2e, world)

    # roofline of the dominant kernel (FP64 run), from the live per-kernel CUDA events
    fp64_meas = fma_peak("fp64") / 1e9
    hbm_peak, hbm_src = 6800.0, HBM_FALLBACK
    try:
        hbm_peak, hbm_src = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), HBM_MEASURED
    except (OSError, KeyError, ValueError):
        pass
    roof, roofline, roof32, roofline32 = roofline_report(
        prof64, prof32, p, D, E, args.steps, K, hbm_peak, fp64_meas,
        traffic_of=lambda k: ncu_traffic(k, args.workload), hbm_src=hbm_src)
    launches = sum(v[0] for v in prof64.values())

    line = {
        "metric": METRIC,
        "value": value, "unit": "angular-DOF updates/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms64 / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "name": args.workload,
                   "nx": wl["nx"], "ny": wl["ny"], "p": p, "mesh_order": wl["mesh_order"], "directions": D,
                   "transport_inversions_per_step": K, "angular_dof_updates_per_step": updates,
                   "l2": "inputs larger than L2 (factor records %.0f GB)" % (
                       E * D * bytes_factor(p, D) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "mixed": {"value": mixed_value, "ms_per_step": ms32 / steps,
                  "speedup_vs_fp64": ms64 / ms32,
                  "dtype": "f32 factorisation and sweeps + f64 defect correction",
                  "defect_correction": (f"{MIXED_PASSES} passes (FP32 sweep, FP64 residual, FP32 "
                                        "correction sweep)" if args.mixed_tol < 0 else
                                        f"to ||r||/||b|| <= {args.mixed_tol}"),
                  "rel_err_vs_fp64": mixed_err, "rel_err_bound": MIXED_ERR_BOUND,
                  "within_bound": all(mixed_err[k] <= MIXED_ERR_BOUND for k in ("phi", "E")),
                  "clocks": clk2,
                  "roofline": roofline32, "roofline_kernels": roof32,
                  "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof32.items() if v[0]}},
        "e2e": {"value": e2e_value, "unit": "angular-DOF updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e / steps},
        "roofline": roofline,
        "roofline_kernels": roof,
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof64.items() if v[0]},
        "gpu_launches": launches,
        "clocks": clk,
    }
    _, info = mesh.sweep(st, ss, om, w, source=q, info=True, psi=psi)
    line["info"] = {"levels": info["levels"], "coupled_groups": info["coupled_groups"],
                    "lagged_face_points": info["lagged_face_points"],
                    "max_inner_iterations": info["max_inner_iterations"]}
    return line


# ------------------------------------------------------------ oracle (CPU) arm
# The oracle is timed on a bounded sample: an NX x NX mesh built with the workload's recipe
# (same map, order, direction set and media recipe), one transport inversion for some of
# its directions.  Worker processes are started with `spawn` and one BLAS / OpenMP thread
# each, so `cores` is the number of processes that ran.
_ORACLE = {}


def _directions(workload):
    from vef_inputs import WORKLOADS, level_symmetric
    return level_symmetric(WORKLOADS[workload]["sn"])


def _oracle_setup(workload, nx):
    import numpy as np
    from oracle.transport import Discretization
    from vef_inputs import WORKLOADS, seeded_media
    spec = WORKLOADS[workload]
    om, w = _directions(workload)
    E, n = nx * nx, (spec["p"] + 1) ** 2
    st, ss = seeded_media(E, spec["media"][1])
    disc = Discretization(nx, nx, spec["mesh_order"], spec["alpha"], spec["p"])
    q = np.full((E, n), float(spec["source"]))
    _ORACLE.update(disc=disc, om=om, w=w, st=st, ss=ss, q=q, n=n, E=E)
    return True


def _oracle_solve(dirs):
    """One transport inversion of the sample for the directions `dirs`: (updates, seconds)."""
    from oracle.transport import sweep
    o = _ORACLE
    t = time.perf_counter()
    sweep(o["disc"], o["om"][dirs], o["w"][dirs], o["st"], o["ss"], source=o["q"])
    return o["E"] * o["n"] * len(dirs), time.perf_counter() - t


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


class OraclePool:
    """`cores` spawned worker processes, each holding the sample's discretisation."""

    def __init__(self, workload, nx, cores):
        import multiprocessing as mp
        keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in keep:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_setup, initargs=(workload, nx))
        finally:
            for k, v in keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.cores = cores

    def run(self, per_worker, D):
        """Every worker solves `per_worker` directions (round robin over the set); returns
        (updates, wall seconds)."""
        jobs = [[(k * per_worker + j) % D for j in range(per_worker)] for k in range(self.cores)]
        t = time.perf_counter()
        res = self.pool.map(_oracle_solve, jobs, chunksize=1)
        return sum(r[0] for r in res), time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def sample_desc(workload, nx, cores, per_worker):
    K, _ = BENCH_WORKLOADS[workload]
    from vef_inputs import WORKLOADS as W
    spec = W[workload]
    return (f"oracle (FP64 NumPy/SciPy, global sparse direct solve per direction) on a {nx}x{nx} mesh "
            f"built with the {spec['nx']}x{spec['ny']} workload's recipe (sine alpha {spec['alpha']}, "
            f"Q{spec['mesh_order']} map, DG Q{spec['p']}, S{spec['sn']}, seed-{spec['media'][1]} media, "
            f"q=1, vacuum): {per_worker} direction(s) per process on {cores} process(es)")


def cpu_baseline(workload, nx, per_worker=2):
    """The oracle's rate on one core and on all host cores (bounded samples)."""
    D = len(_directions(workload)[1])
    all_cores = host_cores()
    out = {"unit": "angular-DOF updates/s", "kind": "oracle", "host_cpu": _cpu_model(),
           "nproc": os.cpu_count()}
    for cores in (1, all_cores):
        pool = OraclePool(workload, nx, cores)
        try:
            pool.run(1, D)                       # warm: imports and first solve
            upd, sec = pool.run(per_worker, D)
        finally:
            pool.close()
        out["1_core" if cores == 1 else "all_cores"] = {
            "value": upd / sec, "cores": cores, "seconds": sec,
            "sample": sample_desc(workload, nx, cores, per_worker)}
    out.update(value=out["all_cores"]["value"], cores=all_cores, sample=out["all_cores"]["sample"])
    return out


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only; each step is one inversion of one
    direction per process of the bounded sample, on every host core."""
    if rank != 0:
        return None
    D = len(_directions(args.workload)[1])
    cores = host_cores()
    pool = OraclePool(args.workload, args.cpu_sample, cores)
    try:
        for _ in range(max(1, args.warmup)):
            pool.run(1, D)
        rates, secs = [], []
        for _ in range(args.steps):
            upd, sec = pool.run(1, D)
            rates.append(upd / sec)
            secs.append(sec)
    finally:
        pool.close()
    value = statistics.median(rates)
    desc = sample_desc(args.workload, args.cpu_sample, cores, 1)
    return {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "angular-DOF updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "name": args.workload, "sample_nx": args.cpu_sample,
                       "directions_per_step": cores},
            "cpu_baseline": {"value": value, "unit": "angular-DOF updates/s", "cores": cores,
                             "kind": "oracle", "sample": desc, "host_cpu": _cpu_model()},
            "e2e": {"value": value, "unit": "angular-DOF updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ other workloads
def _cuda_time(fn, reps=1):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        out = fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def suite_batch(args):
    """The 64-problem batch: problem k (seed 400 + k) has N in {16,32,64,128,256} (k mod 5),
    p = 1 + (k mod 4), S_N in {4,6,8,12,16} (k mod 5 shifted by k // 5), sine mesh alpha 0.05,
    Q3 map, q = 1, vacuum.  One batched FP64 inversion of all 64 (the sweep forms as tuned),
    timed with its factorisations, with the factorisations kept (sigma_t unchanged, as in the
    outer iterations of the VEF method) and as a CUDA-graph replay; beside it the same 64
    problems inverted one call after another."""
    import torch
    from paper_2301_04758_gb300.api import Mesh, Batch
    from vef_inputs.media import batch_problem
    from vef_inputs import level_symmetric, seeded_media
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    meshes, oms, ws, sts, sss, qs = [], [], [], [], [], []
    updates = 0
    for k in range(64):
        spec = batch_problem(k)
        N, p = spec["nx"], spec["p"]
        meshes.append(Mesh(N, N, spec["mesh_order"], p, spec["alpha"]))
        om, w = level_symmetric(spec["sn"])
        oms.append(om)
        ws.append(w)
        st, ss = seeded_media(N * N, spec["media"][1])
        sts.append(T(st))
        sss.append(T(ss))
        qs.append(torch.ones(N * N, (p + 1) ** 2, dtype=torch.float64, device="cuda"))
        updates += N * N * (p + 1) ** 2 * len(w)
    reps = max(1, args.steps)
    # one problem after another, each its own call (schedules built and warm first)
    psis = [m.sweep(st, ss, om, w, source=q) for m, st, ss, om, w, q in zip(meshes, sts, sss, oms, ws, qs)]
    one_by_one = lambda reuse: [m.sweep(st, ss, om, w, source=q, psi=ps, reuse=reuse)
                                for m, st, ss, om, w, q, ps in zip(meshes, sts, sss, oms, ws, qs, psis)]
    ms_single, _ = _cuda_time(lambda: one_by_one(False), reps=reps)
    ms_single_reuse, _ = _cuda_time(lambda: one_by_one(True), reps=reps)
    t0 = time.perf_counter()
    batch = Batch(meshes, oms, ws)
    build_s = time.perf_counter() - t0
    psi = batch.sweep(sts, sss, source=qs)
    ms_default, _ = _cuda_time(lambda: batch.sweep(sts, sss, source=qs, psi=psi), reps=reps)
    tiles = batch.tune()
    ms, _ = _cuda_time(lambda: batch.sweep(sts, sss, source=qs, psi=psi), reps=reps)
    ms_reuse, _ = _cuda_time(lambda: batch.sweep(sts, sss, source=qs, psi=psi, reuse=True), reps=reps)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.sweep(sts, sss, source=qs, psi=psi, stream=s)
    ms_g, _ = _cuda_time(g.replay, reps=reps)
    rate = lambda t: updates / (t * 1e-3)
    return {"suite": "batch", "workload": "64 problems, N 16..256, Q1..Q4, S4..S16, sine alpha 0.05, seeds 400+k",
            "problems": 64, "angular_dof_updates_per_inversion": updates,
            "batched": {"ms": ms, "angular_dof_updates_per_s": rate(ms), "tuned_tiles": tiles,
                        "ms_before_tuning": ms_default},
            "batched_factors_kept": {"ms": ms_reuse, "angular_dof_updates_per_s": rate(ms_reuse)},
            "graph_replay": {"ms": ms_g, "angular_dof_updates_per_s": rate(ms_g)},
            "one_call_per_problem": {"ms": ms_single, "angular_dof_updates_per_s": rate(ms_single),
                                     "ms_factors_kept": ms_single_reuse,
                                     "angular_dof_updates_per_s_factors_kept": rate(ms_single_reuse)},
            "schedule_build_s": build_s}


def flops_hrt_local(p):
    """Algorithmic flops of one element's hybridized RT elimination: the element-dependent
    local blocks (A: 2 (p+2)^2 NJ^2 with NJ = 2 (p+2)(p+1); G: (p+2)^2 NJ (n + 8); the
    divergence block D is the same reference matrix on every element, formed once), the
    Gauss-Jordan inverse of the (NJ + n) system (2 m^3), and H_e = C1 (W C2), r_e (2 NJ^2 NL4
    + 2 NL4^2 NJ + 2 NJ m + 2 NL4 NJ, NL4 = 4 (p+1))."""
    n, nq2 = (p + 1) ** 2, (p + 2) ** 2
    nJ = 2 * (p + 2) * (p + 1)
    m, nl4 = nJ + n, 4 * (p + 1)
    return (2 * nq2 * nJ * nJ + nq2 * nJ * (n + 8) + 2 * m ** 3
            + 2 * nJ * nJ * nl4 + 2 * nl4 * nl4 * nJ + 2 * nJ * m + 2 * nl4 * nJ)


def suite_hrt(args):
    """Hybridized RT VEF solve after one transport inversion: 128 x 128 sine-curved Q3 mesh,
    DG Q2 (RT_2 current), S8, seed-2 media, q = 1, vacuum: the sweep's closures give E, E_b,
    J_in; the solve eliminates every element's local system on the GPU, solves the
    multiplier system (BiCGStab, two-level Schwarz: element patches and a coarse bilinear
    space) and recovers phi and J."""
    import torch
    from paper_2301_04758_gb300.api import Mesh
    from vef_inputs import level_symmetric, seeded_media
    N, p = 128, 2
    om, w = level_symmetric(8)
    st, ss = seeded_media(N * N, 2)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    mesh = Mesh(N, N, 3, p, 0.05)
    st_d, ss_d = T(st), T(ss)
    q = torch.ones(N * N, (p + 1) ** 2, dtype=torch.float64, device="cuda")
    psi = mesh.sweep(st_d, ss_d, om, w, source=q)
    mom = mesh.moments(psi, om, w, outputs=("phi", "P", "Eb", "Jin"))
    Q0 = q * (4.0 * 3.141592653589793)      # Q0 = int q dOmega for the isotropic q = 1
    solve = lambda: mesh.hrt_solve(st_d, ss_d, mom["phi"], mom["P"], mom["Eb"], mom["Jin"], Q0, tol=1e-8,
                                   max_iter=20000, check=False)
    solve()   # warm
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 5))
    mesh.profile(True)
    t0 = time.perf_counter()
    for _ in range(reps):
        phi, J, lam, info = solve()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / reps
    prof = mesh.profile_read()
    mesh.profile(False)
    launches, ms = prof["hrt"]
    # the class times the local elimination and the recovery; the elimination dominates
    local_ms = ms / reps
    fl = flops_hrt_local(p) * N * N
    return {"suite": "hrt", "workload": "128x128 sine-curved Q3 mesh, DG Q2 / RT_2, S8 closures, seed-2 media",
            "elements": N * N, "multipliers": info["multipliers"], "bicgstab_iterations": info["iterations"],
            "rel_residual": info["rel_residual"], "bicgstab_converged_to_1e-8": info["converged"],
            "wall_ms_per_solve": wall * 1e3,
            "local_elimination_and_recovery_ms": local_ms,
            "local_roofline": {"bound": "alu", "achieved": fl / (local_ms * 1e-3) / 1e12,
                               "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                               "frac": fl / (local_ms * 1e-3) / 1e12 / (FP64_PEAK_GFLOPS / 1e3),
                               "flops_per_element": flops_hrt_local(p), "peak_source": FP64_SRC}}


def suite_vef(args):
    """The VEF fixed-point iteration (sweep, closures, hybridized RT VEF solve per iteration)
    on the thick-diffusion-limit recipe at a larger size: 64 x 64 orthogonal mesh, DG Q2,
    S8, sigma_t = 1/eps, sigma_s = 1/eps - eps, q = eps, eps = 1e-2, vacuum, tolerance 1e-6
    on the max norm of successive scalar fluxes."""
    import torch
    from paper_2301_04758_gb300.api import Mesh
    from vef_inputs import level_symmetric
    N, p, eps = 64, 2, 1e-2
    om, w = level_symmetric(8)
    mesh = Mesh(N, N, 1, p, 0.0)
    E, n = mesh.E, mesh.n
    st = torch.full((E,), 1.0 / eps, dtype=torch.float64, device="cuda")
    ss = torch.full((E,), 1.0 / eps - eps, dtype=torch.float64, device="cuda")
    q = torch.full((E, n), eps, dtype=torch.float64, device="cuda")
    mesh.vef_iterate(st, ss, om, w, source=q, tol=1e-6, hrt_tol=1e-10)     # warm (schedules, buffers)
    torch.cuda.synchronize()
    mesh.profile(True)
    t0 = time.perf_counter()
    phi, J, psi, dphi, info = mesh.vef_iterate(st, ss, om, w, source=q, tol=1e-6, hrt_tol=1e-10)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    prof = mesh.profile_read()
    mesh.profile(False)
    its = info["iterations"]
    return {"suite": "vef", "workload": "64x64 orthogonal mesh, DG Q2 / RT_2, S8, thick diffusion limit eps = 1e-2",
            "iterations": its, "converged": info["converged"], "last_change": info["last_change"],
            "hrt_bicgstab_iterations": info["hrt_iterations"], "wall_ms": wall * 1e3,
            "wall_ms_per_iteration": wall * 1e3 / max(its, 1),
            "angular_dof_updates_per_s": E * n * len(w) * its / wall,
            "kernels_ms": {k: round(v[1], 3) for k, v in prof.items() if v[0]},
            "dphi": [float(x) for x in dphi.cpu()]}


def suite_adjoint(args):
    """128 x 128 sine mesh, Q2, S8, seed-5 media: forward sweep, adjoint sweep and the
    gradients of R = int_[0.6,0.8]^2 phi; central differences (relative step 1e-6) on 64
    seeded elements per cross section."""
    import numpy as np
    import torch
    from paper_2301_04758_gb300.api import Mesh
    from vef_inputs import config_workload
    wl = config_workload("sine128_q2_s8_adjoint")
    om, w = wl["omega"], wl["weights"]
    E, n = wl["E"], wl["n"]
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    st_h, ss_h = wl["sigma_t"].copy(), wl["sigma_s"].copy()
    rng = np.random.Generator(np.random.PCG64(5))
    phi_in = T(rng.uniform(0.5, 1.5, (E, n)))
    q = T(wl["source"])
    mesh = Mesh(128, 128, 3, 2, 0.05)
    g = mesh.region_weights((0.6, 0.6), (0.8, 0.8))
    st, ss = T(st_h), T(ss_h)

    def R_of(st_, ss_):
        psi = mesh.sweep(st_, ss_, om, w, phi_in=phi_in, source=q)
        return float((g * mesh.moments(psi, om, w, outputs=("phi",))["phi"]).sum())

    psi = mesh.sweep(st, ss, om, w, phi_in=phi_in, source=q)
    ms_f, _ = _cuda_time(lambda: mesh.sweep(st, ss, om, w, phi_in=phi_in, source=q, psi=psi), reps=3)
    ms_a, (dst, dss, _) = _cuda_time(lambda: mesh.adjoint(st, ss, om, w, psi, g, phi_in=phi_in), reps=3)
    worst, checked = {}, 0
    for rel_step in (1e-6, 1e-4):
        worst[rel_step] = 0.0
        for arr_h, grad in ((st_h, dst), (ss_h, dss)):
            gh = grad.cpu().numpy()
            # seeded sample among elements whose gradient is not negligible (central
            # differences of R resolve about 1e-10 R / h; tiny gradients are FD noise)
            big = np.flatnonzero(np.abs(gh) >= 1e-2 * np.abs(gh).max())
            sample = rng.choice(big, min(32, len(big)), replace=False)
            checked += len(sample)
            for e in sample:
                h = rel_step * arr_h[e]
                arr_h[e] += h
                Rp = R_of(T(st_h), T(ss_h))
                arr_h[e] -= 2 * h
                Rm = R_of(T(st_h), T(ss_h))
                arr_h[e] += h
                fd = (Rp - Rm) / (2 * h)
                worst[rel_step] = max(worst[rel_step], abs(fd - gh[e]) / abs(gh[e]))
    return {"suite": "adjoint", "workload": "128x128 sine-curved Q3 mesh, DG Q2, S8, seed-5 media; "
            "R = int over [0.6,0.8]^2 of phi", "forward_sweep_ms": ms_f, "adjoint_ms": ms_a,
            "fd_samples": checked, "fd_max_rel_diff_step_1e-6": worst[1e-6],
            "fd_max_rel_diff_step_1e-4": worst[1e-4],
            "fd_note": "central differences, relative steps 1e-6 and 1e-4, elements with |dR/dsigma| >= 1e-2 max"}


def sweep_only(args):
    """Small driver for ncu captures: NX x NX sine mesh (alpha 0.05, Q3 map), DG order
    --order (default 2), S_N --sn (default 8), media of seed --seed (default 2), q = 1; runs
    --steps sweeps (each with its factorisation) in --precision (mixed: the benchmark's fixed
    passes), with the apply --apply, through the public API."""
    import torch

    from paper_2301_04758_gb300 import build as vbuild
    vbuild.build()
    from paper_2301_04758_gb300.api import Mesh
    from vef_inputs import level_symmetric, seeded_media
    N, p = args.sweep_only, args.order
    n = (p + 1) ** 2
    om, w = level_symmetric(args.sn)
    st, ss = seeded_media(N * N, args.seed)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    mesh = Mesh(N, N, 3, p, 0.05)
    q = torch.ones(N * N, n, dtype=torch.float64, device="cuda")
    psi = torch.empty(len(w), N * N, n, dtype=torch.float64, device="cuda")
    kw = dict(tol=-1.0, max_passes=MIXED_PASSES) if args.precision == "mixed" else {}
    st_d, ss_d = T(st), T(ss)
    for s in range(args.steps):
        if s == 1:   # the first call builds the schedule: time the others
            torch.cuda.synchronize()
            mesh.profile(True)
            t0 = time.perf_counter()
        mesh.sweep(st_d, ss_d, om, w, source=q, psi=psi, precision=args.precision, apply=args.apply, **kw)
    torch.cuda.synchronize()
    mesh.sync()
    if args.steps > 1:
        k = args.steps - 1
        prof = {c: round(v[1] / k, 3) for c, v in mesh.profile_read().items() if v[0]}
        print(json.dumps({"sweep_only": f"{N}x{N} Q{p} S{args.sn} {args.precision} apply={args.apply}",
                          "ms_per_call": (time.perf_counter() - t0) / k * 1e3, "kernels_ms": prof}))
        mesh.profile(False)


def adjoint_only(args):
    """Small driver for ncu captures of the backward sweep: NX x NX sine mesh (alpha 0.05,
    Q3 map), Q2, S8, seed-5 media, phi_in seeded, q = 1, R = int over [0.6,0.8]^2 of phi;
    one forward sweep, then --steps adjoint sweeps through the public API."""
    import numpy as np
    import torch

    from paper_2301_04758_gb300 import build as vbuild
    vbuild.build()
    from paper_2301_04758_gb300.api import Mesh
    from vef_inputs import level_symmetric, seeded_media
    N, p = args.adjoint_only, 2
    n = (p + 1) ** 2
    om, w = level_symmetric(8)
    st, ss = seeded_media(N * N, 5)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    rng = np.random.Generator(np.random.PCG64(5))
    phi_in = T(rng.uniform(0.5, 1.5, (N * N, n)))
    mesh = Mesh(N, N, 3, p, 0.05)
    q = torch.ones(N * N, n, dtype=torch.float64, device="cuda")
    g = mesh.region_weights((0.6, 0.6), (0.8, 0.8))
    psi = mesh.sweep(T(st), T(ss), om, w, phi_in=phi_in, source=q)
    for _ in range(args.steps):
        mesh.adjoint(T(st), T(ss), om, w, psi, g, phi_in=phi_in)
    torch.cuda.synchronize()
    mesh.sync()


def main():
    args = parse()
    if args.sweep_only:
        sweep_only(args)
        return
    if args.adjoint_only:
        adjoint_only(args)
        return
    if args.suite:
        from paper_2301_04758_gb300 import build as vbuild
        vbuild.build()
        fn = {"batch": suite_batch, "adjoint": suite_adjoint, "hrt": suite_hrt, "vef": suite_vef}[args.suite]
        print(json.dumps(fn(args)))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
