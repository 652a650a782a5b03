#!/usr/bin/env python3
"""Benchmark of the even-odd Wilson-Dirac CG hot path on GB300.

One step = one complete FP64-class (double-word) even-odd CG solve of
D x = b to a true relative residual of 1e-10 on a 24^3x48 lattice
(links exp(i*0.3*H), kappa = 0.12, antiperiodic time, Gaussian source):
source preparation, CG on Mhat^dag Mhat, reconstruction.  Gauge field and
source are resident in HBM when the timed region starts.

value = Dslash GB/s of the whole job: algorithmic bytes of every hop launch
in the timed solves (1536 B per output site, +192 B when the hop also reads
an axpy operand) divided by the wall time of the solves, summed over ranks.
gflops = the same solves in the Wilson hop's conventional 1320 flops per
output site (spin projection, SU(3) times half-spinor, reconstruction and
accumulation over the 8 directions; axpy terms not counted) per second.
e2e   = the same quantity through jqcd_cg_solve with host buffers in pinned
memory (copy of b in, copy of x out, inside the timed region).
roofline = the double-word hop kernel timed alone on the same lattice (mean of
back-to-back launches, CUDA events on its stream), reported against HBM: its
algorithmic bytes per launch over the measured copy bandwidth (the metric's
"Dslash GB/s vs HBM peak").  Its FP32-datapath fraction (error-free
double-word arithmetic: FP32 lane operations per second against SMs x 128
lanes x clock) rides along under roofline.alu.  roofline.traffic is ncu's
DRAM bytes per launch from the committed profile summary, used only while
the kernel sources hash to the captured value (roofline.traffic_source).
cg = CG seconds to 1e-10 per solver mode (double-word, plain FP64, mixed FP32
and FP16 inner) on the workload and on 32^3x64, each workload solution's
error against the FP64 oracle's solution (err_vs_oracle) and each 32^3x64
solution's against the plain FP64 GPU solve's (err_vs_f64).
cpu_baseline = the FP64 CPU oracle's complete solve of the workload system
on the host cores (its solution gives err_vs_oracle); --impl reference = the
oracle's CG iterations on the same system.

Multi-GPU (torchrun): each rank solves its own replica (independent problems,
weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 48)
KAPPA = 0.12
EPS = 0.3
TOL = 1e-10
METRIC = "Dslash GB/s vs HBM peak; CG s to 1e-10 mixed vs FP64; serve p50/p99"
HOP_BYTES = {"dw": 1536, "f64": 1536, "f32": 576, "f16n": 488}  # per output site
AXPY_BYTES = {"dw": 192, "f64": 192, "f32": 96, "f16n": 52}
HOP_FLOPS_PER_SITE = 1320  # conventional Wilson hop count per output site (axpy not counted)
# The sources hop_dwp_kernel is compiled from: its translation unit and the
# headers it reaches (dslash.cu also includes hop_lp.cuh and cg_steps.cuh,
# which serve the low-precision kernels only).  The committed ncu traffic is
# reported only while their hash matches the one the capture was taken at.
HOP_KERNEL_SOURCES = ["dslash.cu", "hop_dwp.cuh", "hop_dw.cuh", "hop.cuh", "dw2.cuh", "dw.cuh",
                      "fields.cuh", "lattice.cuh", "reduce.cuh", "kernels.h", "pdl.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jqcd", choices=["jqcd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config2", action="store_true",
                    help="skip the 32^3x64 mixed-vs-double-word CG comparison")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="leave out the per-mode err_vs_oracle of the workload solves")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-solve batch")
    ap.add_argument("--serve-host", default="pinned", choices=["pinned", "pageable"],
                    help="host memory of the serving stream's sources and solutions")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the serving run (0 skips it)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def vol(dims):
    v = 1
    for d in dims:
        v *= d
    return v


def sample_description(iters):
    return (f"oracle textbook CG on {DIMS[0]}^3x{DIMS[3]}, {iters} iteration(s) "
            f"({iters + 2} applications of Mhat^dag Mhat incl. start and true residual)")


def time_oracle_cg(U, b, iters, threads=0):
    """Oracle CG run for `iters` iterations on `threads` threads (0: all it
    uses by default); returns (GB/s of hop bytes, seconds, threads used)."""
    import oracle
    rhs = oracle.zero_parity(DIMS, b, 1)
    before = oracle.set_threads(0)
    used = oracle.set_threads(threads) if threads > 0 else before
    try:
        t0 = time.perf_counter()
        oracle.cg(DIMS, U, rhs, KAPPA, eo=True, tol=1e-30, maxiter=iters)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(before)
    vh = vol(DIMS) // 2
    hop_bytes = (iters + 2) * vh * (4 * 1536 + 2 * 192)
    return hop_bytes / dt / 1e9, dt, used


def time_oracle_solve(U, b, tol):
    """The oracle's complete even-odd solve of the workload system D x = b to
    `tol` on all the threads it uses by default.  Returns (GB/s of hop bytes
    at the GPU's accounting, seconds, threads, x, CG iterations, system
    residual).  Hop bytes: source preparation (3 hops), (iters + 2)
    applications of Mhat^dag Mhat (start and true residual included) and the
    reconstruction (1 hop)."""
    import oracle
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    x, iters, res, _, _ = oracle.solve(DIMS, U, b, KAPPA, eo=True, tol=tol)
    dt = time.perf_counter() - t0
    vh = vol(DIMS) // 2
    hop_bytes = (iters + 2) * vh * (4 * 1536 + 2 * 192) + vh * (4 * 1536 + 3 * 192)
    return hop_bytes / dt / 1e9, dt, threads, x, iters, res


def kernel_hash():
    h = hashlib.sha256()
    for f in HOP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2409_03030_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the double-word hop from the committed ncu
    summary, or None when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "hop_dw_24x24x24x48.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP32 lane operations (add, mul or fma, each on one lane) per output site of
# the plain double-word hop, counted from its arithmetic: per hop, projection
# 6 x 9, mat-vec 2 x 3 x (2 x 17 + 2) (offset-grid sums: 5 + 6 + 6 per sum of
# three products, 2 to join A + iB) and reconstruction 2 x 3 x 17 packed
# two-lane operations; epilogue 12 x 10 packed; times 2 lanes; plus the grid
# bounds, 2 x 5 + 1 scalar per hop.  The backward links are conjugated by
# flipping sign bits, which is no floating-point operation.
DW_HOP_LANE_OPS = 2 * (8 * (6 * 9 + 2 * 3 * (2 * 17 + 2) + 2 * 3 * 17) + 12 * 10) + 8 * (2 * 5 + 1)
NOMINAL_HBM_GBS = 7900.0


def alu_peak_tops(device=0):
    """FP32 lane operations per second of the GPU: SMs x 128 FP32 lanes x
    the maximum SM clock (MEASURED_PEAKS.json, else the device's own)."""
    import torch
    props = torch.cuda.get_device_properties(device)
    mhz = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            mhz = json.load(fh).get("sm_max_mhz")
    if not mhz:
        mhz = getattr(props, "clock_rate", 2070000) / 1000.0
    return props.multi_processor_count * 128 * float(mhz) * 1e6 / 1e12


def reduce_over_ranks(max_values, sum_values, device):
    """Across all ranks: elementwise max of max_values and sum of sum_values
    (lists of floats).  One rank: returned unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(max_values), list(sum_values)
    tm = torch.tensor(list(max_values), dtype=torch.float64, device=device)
    ts = torch.tensor(list(sum_values), dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm.tolist(), ts.tolist()


def parse_clock_lines(lines):
    """nvidia-smi CSV rows (clocks.sm, clocks.max.sm, power, active mask,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm.append(float(parts[0]))
            mx.append(float(parts[1]))
        except ValueError:
            continue
        for n, v in zip(names, parts[4:8]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.idx = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.idx, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_lines(out.splitlines())


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2409_03030_gb300 import synth
    U = synth.gauge(DIMS, "expi", eps=EPS, seed=1)
    b = synth.gaussian_spinor(DIMS, seed=2)
    iters = 1
    for _ in range(args.warmup):
        time_oracle_cg(U, b, iters)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, threads = time_oracle_cg(U, b, iters)
        vals.append(v)
        times.append(dt)
    total = sum(times)
    value = sum(v * t for v, t in zip(vals, times)) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": threads,
                         "kind": "oracle", "sample": sample_description(iters)},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    del oracle


def workload_config():
    return {"workload": "even-odd Wilson-Dirac CG to 1e-10 true residual, 24^3x48, "
                        "FP64-class double-word arithmetic",
            "lattice": list(DIMS), "kappa": KAPPA, "links": f"exp(i*{EPS}*H), seeded",
            "source": "Gaussian, seeded", "tol": TOL, "boundary": "periodic xyz, antiperiodic t",
            "l2": "inputs larger than L2 (double-word gauge field 382 MB)",
            "parallelism": "replicas"}


def bench_force(ctx, jqcd, synth, np, torch, stream, g, b):
    """Fermion action and force on the workload lattice (kappa 0.12): the
    per-link kernel alone on resident X, Y (1536 algorithmic bytes per site:
    X, Y once, 4 links in, 4 matrices out), and the whole action + force
    (two even-odd solves to 1e-10, the dot product, the kernel) from a host
    pseudofermion, double-word and mixed FP16."""
    X = synth.gaussian_spinor(DIMS, seed=81)
    with torch.cuda.stream(stream):
        xe, xo = g.pack(X, jqcd.PREC_DW, stream=stream)
        ye, yo = g.pack(b, jqcd.PREC_DW, stream=stream)
        out = torch.empty(g.linkfield_bytes(), dtype=torch.uint8, device=xe.device)
    for _ in range(3):
        g.fermi_force_dev(KAPPA, xe, xo, ye, yo, out, stream=stream)
    stream.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    a0.record(stream)
    for _ in range(n):
        g.fermi_force_dev(KAPPA, xe, xo, ye, yo, out, stream=stream)
    a1.record(stream)
    stream.synchronize()
    us = a0.elapsed_time(a1) / n * 1e3
    V = vol(DIMS)
    hbm, _ = peaks()
    res = {"kernel": "force_kernel (U dS/dU, double-word)", "us": round(us, 1),
           "gbs": round(V * 1536 / us / 1e3, 1), "hbm_frac": round(V * 1536 / us / 1e3 / hbm, 4)}
    for name, mode in [("dw", jqcd.CG_DW), ("mixed_f16", jqcd.CG_MIXED_F16)]:
        g.fermi_force(b, KAPPA, tol=TOL, mode=mode)  # warm-up
        t0 = time.perf_counter()
        S, _, info, st = g.fermi_force(b, KAPPA, tol=TOL, mode=mode)
        res[f"action_force_{name}"] = {"s": round(time.perf_counter() - t0, 4),
                                       "gpu_s": round(info["gpu_seconds"], 4),
                                       "iters": info["iters"], "action": S, "status": st}
    return res


def bench_hmc(ctx, jqcd, synth, np):
    """One HMC trajectory (the paper's MD step: 10 leapfrog steps of length
    1/10, plaquette action beta 5.5, two-flavour Wilson fermions kappa 0.12,
    solves to 1e-10) on a 16^4 exp(i 0.3 H) field, double-word and mixed-FP16
    solves; random numbers seeded on the host."""
    d = (16, 16, 16, 16)
    U = synth.gauge(d, "expi", eps=EPS, seed=61)
    rng = np.random.default_rng(62)
    normals = rng.normal(size=(4,) + tuple(reversed(d)) + (8,))
    xi = synth.gaussian_spinor(d, seed=63)
    out = {"workload": "16^4, beta 5.5, kappa 0.12, 10 MD steps, tau 1, tol 1e-10"}
    for name, mode in [("dw", jqcd.CG_DW), ("mixed_f16", jqcd.CG_MIXED_F16)]:
        g = ctx.gauge_upload(d, U)
        g.hmc_trajectory(normals, xi, 0.0, 5.5, kappa=KAPPA, n_md=2, tol=TOL, mode=mode)  # warm-up
        g.free()
        g = ctx.gauge_upload(d, U)
        info, st = g.hmc_trajectory(normals, xi, 0.0, 5.5, kappa=KAPPA, n_md=10, tol=TOL, mode=mode)
        out[name] = {"s": round(info["seconds"], 4), "cg_iters": info["cg_iters"], "dH": info["dH"],
                     "plaquette": info["plaquette"], "status": st}
        g.free()
    return out


def bench_staggered(jqcd, synth, torch, stream, g):
    """Staggered operator on the workload lattice and links: the double-word
    hop alone (algorithmic bytes per output site: colour vector in once, 8
    double-word links, out = 1248 B) and the even-odd solve of D x = b to
    1e-10 at m = 0.05."""
    b = synth.gaussian_colour(DIMS, seed=91)
    with torch.cuda.stream(stream):
        be, bo = g.stag_pack(b, stream=stream)
        out = g.stag_empty()
    for _ in range(5):
        g.stag_dslash_eo(0, 0, bo, None, out, stream=stream)
    stream.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 40
    a0.record(stream)
    for _ in range(n):
        g.stag_dslash_eo(0, 0, bo, None, out, stream=stream)
    a1.record(stream)
    stream.synchronize()
    us = a0.elapsed_time(a1) / n * 1e3
    vh = vol(DIMS) // 2
    hbm, _ = peaks()
    gbs = vh * 1248 / us / 1e3
    with torch.cuda.stream(stream):
        xe, xo = g.stag_empty(), g.stag_empty()
    g.stag_solve_dev(be, bo, xe, xo, 0.05, tol=TOL, stream=stream)  # warm-up
    info, st = g.stag_solve_dev(be, bo, xe, xo, 0.05, tol=TOL, stream=stream)
    return {"hop_us": round(us, 1), "hop_gbs": round(gbs, 1), "hop_hbm_frac": round(gbs / hbm, 4),
            "solve": {"mass": 0.05, "s": round(info["gpu_seconds"], 4), "iters": info["iters"],
                      "true_rel_resid": info["true_rel_resid"], "full_rel_resid": info["full_rel_resid"],
                      "status": st}}


def bench_multishift(jqcd, g, stream, rhs_even):
    """Multi-shift CG on the workload lattice: eight RHMC-like shifts of
    Mhat^dag Mhat to 1e-10 in one Krylov space, against the same eight
    systems solved one at a time (a one-shift solve each)."""
    shifts = [1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3]
    xs = [g.empty(jqcd.PREC_DW) for _ in shifts]
    g.cg_multishift_dev(rhs_even, xs, KAPPA, shifts, tol=TOL, stream=stream)  # warm-up
    infos, st = g.cg_multishift_dev(rhs_even, xs, KAPPA, shifts, tol=TOL, stream=stream)
    t_multi = infos[0]["gpu_seconds"]
    t_single, it_single = 0.0, []
    for i, sg in enumerate(shifts):
        inf1, _ = g.cg_multishift_dev(rhs_even, [xs[i]], KAPPA, [sg], tol=TOL, stream=stream)
        t_single += inf1[0]["gpu_seconds"]
        it_single.append(inf1[0]["iters"])
    return {"workload": "8 shifts 1e-4..0.3 of Mhat^dag Mhat, 24^3x48, kappa 0.12, tol 1e-10, double-word",
            "multishift_s": round(t_multi, 4), "separate_s": round(t_single, 4),
            "speedup": round(t_single / t_multi, 2), "iters": [i["iters"] for i in infos],
            "iters_separate": it_single,
            "max_true_rel_resid": max(i["true_rel_resid"] for i in infos), "status": st,
            "hop_gbs": round(infos[0]["hop_bytes"] / t_multi / 1e9, 1)}


def bench_batch(ctx, jqcd, synth, np):
    """12 point sources on 24^3x48 + 12 Gaussian sources on 16^4 (kappa 0.12,
    exp(i 0.3 H) links, tol 1e-10): one jqcd_cg_solve_batch call vs the same
    24 solves one after another through jqcd_cg_solve, with FP16 inner
    solves; `f32_inner` repeats it with FP32 inner solves (FP32/FP64 mixed)."""
    dA, dB = (24, 24, 24, 48), (16, 16, 16, 16)
    gA = ctx.gauge_upload(dA, synth.gauge(dA, "expi", eps=EPS, seed=31))
    gB = ctx.gauge_upload(dB, synth.gauge(dB, "expi", eps=EPS, seed=32))
    bs = [synth.point_source(dA, s, c) for s in range(4) for c in range(3)]
    bs += [synth.gaussian_spinor(dB, seed=100 + i) for i in range(12)]
    gauges = [gA] * 12 + [gB] * 12
    # pinned host buffers, reused by both ways of solving (no page faults in the timing)
    bs = [pinned_copy(b) for b in bs]
    outs = [pinned_copy(np.zeros_like(b)) for b in bs]
    out = batch_vs_sequential(ctx, jqcd, gauges, bs, outs, gA, jqcd.CG_MIXED_F16)
    out["workload"] = ("12 point sources 24^3x48 + 12 Gaussian 16^4, kappa 0.12, tol 1e-10, "
                       "mixed FP16, one batch (pinned host buffers, reused)")
    f32 = batch_vs_sequential(ctx, jqcd, gauges, bs, outs, gA, jqcd.CG_MIXED_F32)
    out["f32_inner"] = {k: f32[k] for k in ("batch_s", "sequential_s", "speedup", "sequential_gpu_s",
                                            "max_true_rel_resid", "iters", "status")}
    gA.free()
    gB.free()
    return out


def batch_vs_sequential(ctx, jqcd, gauges, bs, outs, gA, mode):
    """Best of three alternating repetitions of one batch call and of the same
    solves one after another."""
    ctx.cg_solve_batch(gauges, bs, [KAPPA] * 24, [TOL] * 24, mode=mode, out=outs)  # warm-up + autotune
    gA.cg_solve(bs[0], KAPPA, tol=TOL, mode=mode, out=outs[0])  # warm-up
    reps = 3  # both ways alternate; each is reported as the best of its repetitions
    tb, ts, tsg = [], [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        xs, infos, st = ctx.cg_solve_batch(gauges, bs, [KAPPA] * 24, [TOL] * 24, mode=mode, out=outs)
        tb.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        gpu = 0.0
        for g, b, o in zip(gauges, bs, outs):
            gpu += g.cg_solve(b, KAPPA, tol=TOL, mode=mode, out=o)[1]["gpu_seconds"]
        ts.append(time.perf_counter() - t0)
        tsg.append(gpu)
    t_batch, t_seq = min(tb), min(ts)
    out = {"batch_s": round(t_batch, 4), "sequential_s": round(t_seq, 4),
           "speedup": round(t_seq / t_batch, 3), "solves_per_s": round(24 / t_batch, 2),
           "repetitions": reps, "batch_all_s": [round(v, 4) for v in tb],
           "sequential_all_s": [round(v, 4) for v in ts],
           "sequential_gpu_s": round(min(tsg), 4),  # device time of the 24 solves proper
           "max_true_rel_resid": max(i["true_rel_resid"] for i in infos),
           "iters": [infos[0]["iters"], infos[12]["iters"]], "status": st}
    return out


def pinned_copy(a):
    """Copy of a complex128 array in pinned (page-locked) host memory."""
    import torch
    t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
    t.numpy()[...] = a
    return t.numpy()


def bench_serve(ctx, jqcd, synth, np, n_req, rate=20.0, host="pinned"):
    """Poisson arrivals (seeded, mean `rate`/s) of solves with volume drawn from
    {8^4, 16^4, 24^3x48, 32^3x64}, kappa ~ U[0.10, 0.122], tol in {1e-8,
    1e-10, 1e-12}, Gaussian sources, gauge fields pre-generated (eps 0.3).
    Latency = scheduled arrival -> completion seen by the client.  host:
    "pinned" (sources and solution buffers page-locked, as a serving front
    end holds them) or "pageable" (plain numpy arrays)."""
    vols = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64)]
    gauges = [ctx.gauge_upload(d, synth.gauge(d, "expi", eps=EPS, seed=70 + i))
              for i, d in enumerate(vols)]
    n_src, n_x = 3, 8
    keep = pinned_copy if host == "pinned" else (lambda a: a)
    srcs = [[keep(synth.gaussian_spinor(d, seed=800 + 10 * i + j)) for j in range(n_src)]
            for i, d in enumerate(vols)]
    xpool = [[keep(np.zeros(synth.spinor_shape(d), np.complex128)) for _ in range(n_x)] for d in vols]
    free = [list(range(n_x)) for _ in vols]
    rng = np.random.default_rng(20261202)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    vol = rng.integers(0, 4, n_req)
    kap = rng.uniform(0.10, 0.122, n_req)
    tol = rng.choice([1e-8, 1e-10, 1e-12], n_req)
    src = rng.integers(0, n_src, n_req)
    mode = jqcd.CG_MIXED_F16
    ctx.serve_start(64 << 30, max_slots=32, mode=mode)
    inflight = {}  # ticket -> (request index, volume, x index)
    lat, done, nxt, worst_res = [], 0, 0, 0.0
    lat_vol = [[] for _ in vols]
    t0 = time.perf_counter()
    while done < n_req:
        now = time.perf_counter() - t0
        while nxt < n_req and arrivals[nxt] <= now and free[vol[nxt]]:
            v = int(vol[nxt])
            xi = free[v].pop()
            st, t = ctx.serve_submit(gauges[v], srcs[v][src[nxt]], xpool[v][xi], float(kap[nxt]),
                                     float(tol[nxt]), mode=mode)
            if st != 0:
                raise RuntimeError(f"serve_submit status {st}")
            inflight[t] = (nxt, v, xi)
            nxt += 1
        for t in list(inflight):
            st, info = ctx.serve_poll(t)
            if st == jqcd.PENDING:
                continue
            i, v, xi = inflight.pop(t)
            if st != 0:
                raise RuntimeError(f"request {i} finished with status {st}")
            lat.append(time.perf_counter() - t0 - arrivals[i])
            lat_vol[v].append(lat[-1])
            worst_res = max(worst_res, info["true_rel_resid"] / tol[i])
            free[v].append(xi)
            done += 1
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    stats = ctx.serve_stop()
    lat = np.sort(np.array(lat))
    out = {"workload": f"{n_req} Poisson requests at {rate}/s, volumes 8^4/16^4/24^3x48/32^3x64, "
                       "kappa U[0.10,0.122], tol {1e-8,1e-10,1e-12}, mixed FP16, budget 64 GiB, "
                       f"{host} host buffers",
           "p50_s": round(float(np.percentile(lat, 50)), 5),
           "p99_s": round(float(np.percentile(lat, 99)), 5),
           "mean_s": round(float(lat.mean()), 5),
           "solves_per_s": round(n_req / wall, 2), "offered_per_s": rate,
           "arrival_span_s": round(float(arrivals[-1]), 3), "wall_s": round(wall, 3),
           "stable": bool(wall < arrivals[-1] + 2.0),
           "server_p50_s": round(stats["p50_s"], 5), "server_p99_s": round(stats["p99_s"], 5),
           "peak_active": stats["peak_active"], "peak_queue": stats["peak_queue"],
           "peak_slot_bytes": stats["peak_hbm_bytes"],
           "max_true_resid_over_tol": worst_res,
           "by_volume": {"x".join(map(str, d)): {
               "n": len(lv), "p50_s": round(float(np.percentile(lv, 50)), 5) if lv else None,
               "p99_s": round(float(np.percentile(lv, 99)), 5) if lv else None}
               for d, lv in zip(vols, lat_vol)}}
    for g in gauges:
        g.free()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    from paper_2409_03030_gb300 import jqcd, synth

    vh = vol(DIMS) // 2
    U = synth.gauge(DIMS, "expi", eps=EPS, seed=1)
    b = synth.gaussian_spinor(DIMS, seed=2 + rank)
    ctx = jqcd.Context(local)
    g = ctx.gauge_upload(DIMS, U)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        be, bo = g.pack(b, jqcd.PREC_DW, stream=stream)
        xe, xo = g.empty(jqcd.PREC_DW), g.empty(jqcd.PREC_DW)
    stream.synchronize()

    def solve():
        info, st = g.cg_solve_dev(be, bo, xe, xo, KAPPA, tol=TOL, eo=True, mode=jqcd.CG_DW,
                                  stream=stream)
        return info

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        solve()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = jqcd.jqcd_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [solve() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = jqcd.jqcd_kernel_launches() - l0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    hop_bytes = sum(i["hop_bytes"] for i in infos)
    hop_flops = sum(i["hop_count"] for i in infos) * (vol(DIMS) // 2) * HOP_FLOPS_PER_SITE
    (ms_max,), (bytes_sum, flops_sum) = reduce_over_ranks([ms], [hop_bytes, hop_flops], "cuda")
    value = bytes_sum / (ms_max * 1e-3) / 1e9
    gflops = flops_sum / (ms_max * 1e-3) / 1e9
    dw_s = ms / args.steps * 1e-3

    # end to end through the host-buffer C ABI call, pinned host memory
    shape = b.shape
    b_pin = torch.empty(shape, dtype=torch.complex128, pin_memory=True)
    b_pin.numpy()[...] = b
    x_pin = torch.zeros(shape, dtype=torch.complex128, pin_memory=True)
    bn, xn = b_pin.numpy(), x_pin.numpy()
    p = g.params(KAPPA, TOL, 20000, True, jqcd.CG_DW)
    import ctypes
    info = jqcd.jqcd_solve_info()
    bptr = bn.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    xptr = xn.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    e2e_steps = max(3, args.steps // 2)
    for _ in range(2):
        ctx.check(jqcd.jqcd_cg_solve(ctx.h, g.id, ctypes.byref(p), bptr, xptr, ctypes.byref(info)),
                  "cg_solve")
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_bytes = 0.0
    for _ in range(e2e_steps):
        ctx.check(jqcd.jqcd_cg_solve(ctx.h, g.id, ctypes.byref(p), bptr, xptr, ctypes.byref(info)),
                  "cg_solve")
        e2e_bytes += info.hop_bytes
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    (e2e_s,), (e2e_bytes,) = reduce_over_ranks([e2e_s], [e2e_bytes], "cuda")
    e2e_value = e2e_bytes / e2e_s / 1e9

    # dominant kernel alone: double-word hop, plus the other precisions
    def time_hop(prec, n=40, gg=None, src=None):
        gg = g if gg is None else gg
        src = b if src is None else src
        with torch.cuda.stream(stream):
            pe, po = gg.pack(src, prec, stream=stream)
            out = gg.empty(prec)
        for _ in range(5):
            gg.dslash_eo(prec, 0, 0, po, None, out, stream=stream)
        stream.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            gg.dslash_eo(prec, 0, 0, po, None, out, stream=stream)
        a1.record(stream)
        stream.synchronize()
        return a0.elapsed_time(a1) / n

    precs = [("dw", jqcd.PREC_DW), ("f64", jqcd.PREC_F64), ("f32", jqcd.PREC_F32),
             ("f16n", jqcd.PREC_F16N)]

    def hop_sweep(gg, dims, src):
        vhs = vol(dims) // 2
        return {name: round(vhs * HOP_BYTES[name] / (time_hop(code, gg=gg, src=src) * 1e-3) / 1e9, 1)
                for name, code in precs}

    hop_ms = {name: time_hop(code) for name, code in precs}
    sweep = {"x".join(map(str, DIMS)): {k: round(vh * HOP_BYTES[k] / (v * 1e-3) / 1e9, 1)
                                        for k, v in hop_ms.items()}}
    d16 = (16, 16, 16, 16)
    g16 = ctx.gauge_upload(d16, synth.gauge(d16, "expi", eps=EPS, seed=21))
    sweep["16x16x16x16 (L2-resident)"] = hop_sweep(g16, d16, synth.gaussian_spinor(d16, seed=22))
    g16.free()
    hbm, peak_kind = peaks()
    dw_achieved = vh * HOP_BYTES["dw"] / (hop_ms["dw"] * 1e-3) / 1e9
    alu_achieved = vh * DW_HOP_LANE_OPS / (hop_ms["dw"] * 1e-3) / 1e12
    alu_peak = alu_peak_tops(local)
    traffic = profiled_traffic()

    # CG to 1e-10: double-word vs mixed precision, on the workload lattice and
    # on the 32^3x64 configuration (exp(i 0.4 H) links, kappa 0.122)
    def time_solves(gg, be_, bo_, xe_, xo_, kappa, mode, n):
        gg.cg_solve_dev(be_, bo_, xe_, xo_, kappa, tol=TOL, eo=True, mode=mode, stream=stream)
        t = []
        info = None
        for _ in range(n):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            info, _ = gg.cg_solve_dev(be_, bo_, xe_, xo_, kappa, tol=TOL, eo=True, mode=mode,
                                      stream=stream)
            a1.record(stream)
            stream.synchronize()
            t.append(a0.elapsed_time(a1) * 1e-3)
        return statistics.median(t), info

    def cg_table(gg, be_, bo_, kappa, n, keep=None):
        """Per mode: median solve time, iterations, residuals.  keep: dict
        that receives each mode's solution (host, canonical order)."""
        xe_, xo_ = gg.empty(jqcd.PREC_DW), gg.empty(jqcd.PREC_DW)
        out = {}
        for name, mode in [("dw", jqcd.CG_DW), ("f64", jqcd.CG_F64),
                           ("mixed_f32", jqcd.CG_MIXED_F32), ("mixed_f16", jqcd.CG_MIXED_F16)]:
            t, info = time_solves(gg, be_, bo_, xe_, xo_, kappa, mode, n)
            out[name] = {"s": round(t, 5), "iters": info["iters"],
                         "reliable_updates": info["reliable_updates"],
                         "true_rel_resid": info["true_rel_resid"],
                         "full_rel_resid": info["full_rel_resid"]}
            if keep is not None:
                keep[name] = gg.unpack(xe_, xo_, jqcd.PREC_DW, stream=stream)
        for m in ("mixed_f16", "mixed_f32"):
            out[f"speedup_{m}_vs_f64"] = round(out["f64"]["s"] / out[m]["s"], 3)
            out[f"speedup_{m}_vs_dw"] = round(out["dw"]["s"] / out[m]["s"], 3)
        out["speedup_dw_vs_f64"] = round(out["f64"]["s"] / out["dw"]["s"], 3)
        return out

    work_solutions = {}
    cg_work = cg_table(g, be, bo, KAPPA, 3, keep=work_solutions)
    cg_c2 = None
    c2_solutions = {}
    d2 = (32, 32, 32, 64)
    if not args.no_config2:
        g2 = ctx.gauge_upload(d2, synth.gauge(d2, "expi", eps=0.4, seed=11))
        b2 = synth.gaussian_spinor(d2, seed=12)
        with torch.cuda.stream(stream):
            b2e, b2o = g2.pack(b2, jqcd.PREC_DW, stream=stream)
        stream.synchronize()
        cg_c2 = cg_table(g2, b2e, b2o, 0.122, 3, keep=c2_solutions)
        sweep["32x32x32x64"] = hop_sweep(g2, d2, synth.gaussian_spinor(d2, seed=12))
        cg_c2["workload"] = "32^3x64, exp(i*0.4*H) links, kappa 0.122, even-odd, tol 1e-10"
        g2.free()

    force = bench_force(ctx, jqcd, synth, np, torch, stream, g, b)
    multishift = bench_multishift(jqcd, g, stream, be)
    staggered = bench_staggered(jqcd, synth, torch, stream, g)
    hmc = bench_hmc(ctx, jqcd, synth, np)
    def with_clocks(fn):
        """fn() with the SM clocks sampled while it runs (added as "clocks")."""
        smp = ClockSampler(local)
        smp.start()
        out = fn()
        clk = smp.stop()
        if out is not None:
            out["clocks"] = clk
        return out

    batch = with_clocks(lambda: bench_batch(ctx, jqcd, synth, np)) if not args.no_batch else None
    serve = (with_clocks(lambda: bench_serve(ctx, jqcd, synth, np, args.serve_requests,
                                             host=args.serve_host))
             if args.serve_requests > 0 else None)

    # 32^3x64: each mode's solution against the plain FP64 GPU solve's
    if cg_c2 is not None and "f64" in c2_solutions:
        x64 = c2_solutions["f64"]
        n64 = float(np.linalg.norm(x64))
        for name, xs in c2_solutions.items():
            if name != "f64":
                cg_c2[name]["err_vs_f64"] = float(np.linalg.norm(xs - x64)) / n64
    c2_solutions = None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle solves the bench's own system (tol 1e-12), after every GPU
        # timing of the run; its solution also gives each GPU mode's error
        v, dt, threads, xo, it_o, res_o = time_oracle_solve(U, b, 1e-12)
        v1, dt1s, _ = time_oracle_cg(U, b, 1, threads=1)  # one thread, one iteration
        cpu = {"value": round(v, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": (f"oracle even-odd solve of the workload system to 1e-12 "
                          f"(textbook CG, {it_o} iterations, system residual {res_o:.2e}), "
                          f"{dt:.1f} s"),
               "single_thread": {"value": round(v1, 3), "unit": "GB/s", "cores": 1,
                                 "sample": sample_description(1) + f", {dt1s:.1f} s"},
               "gpu_speedup": {"vs_all_cores": round(value / v, 1),
                               "vs_one_core": round(value / v1, 1)}}
        if not args.no_oracle_error:
            nrm = float(np.linalg.norm(xo))
            for name, xs in work_solutions.items():
                cg_work[name]["err_vs_oracle"] = float(np.linalg.norm(xs - xo)) / nrm
            cg_work["err_definition"] = ("||x - x_oracle|| / ||x_oracle|| over the whole lattice, "
                                         "x_oracle the FP64 oracle's solution of D x = b to 1e-12 "
                                         "(the cpu_baseline solve)")
    work_solutions = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "gflops": round(gflops, 1),
            "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2 (double-word, FP64-class)", "data": "synthetic",
            "config": workload_config(),
            "roofline": {"bound": "hbm", "achieved": round(dw_achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(dw_achieved / hbm, 4), "traffic": traffic,
                         "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per "
                                            "launch, profiles/hop_dw_24x24x24x48.md (kernel "
                                            "sources hash-matched); not measured in this run"
                                            if traffic is not None else None),
                         "kernel": "hop_dwp_kernel (double-word plain hop)",
                         "bytes_per_site": HOP_BYTES["dw"],
                         "frac_nominal": round(dw_achieved / NOMINAL_HBM_GBS, 4),
                         "peak_kind": f"{peak_kind} copy bandwidth (burst); nominal 7.9 TB/s",
                         "alu": {"achieved": round(alu_achieved, 2), "peak": round(alu_peak, 2),
                                 "unit": "Tops/s (FP32 lane operations)",
                                 "frac": round(alu_achieved / alu_peak, 4), "ops_per_site": DW_HOP_LANE_OPS,
                                 "peak_kind": "SMs x 128 FP32 lanes x maximum SM clock"}},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": int(b.nbytes), "d2h_bytes_per_step": int(b.nbytes)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cg": {"dw_s": round(dw_s, 5), "dw_iters": infos[-1]["iters"],
                   "dw_true_rel_resid": infos[-1]["true_rel_resid"],
                   "dw_full_rel_resid": infos[-1]["full_rel_resid"],
                   "modes_24x24x24x48": cg_work, "modes_32x32x32x64": cg_c2},
            "dslash_gbs": {k: round(vh * HOP_BYTES[k] / (v * 1e-3) / 1e9, 1)
                           for k, v in hop_ms.items()},
            "dslash_gflops": {k: round(vh * HOP_FLOPS_PER_SITE / (v * 1e-3) / 1e9, 1)
                              for k, v in hop_ms.items()},
            "dslash_sweep_gbs": sweep,
            "dslash_link_reals": {"dw": 18, "f64": 18, "f32": 12, "f16n": 12},
            "force": force,
            "multishift": multishift,
            "staggered": staggered,
            "hmc": hmc,
            "batch": batch,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    g.free()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    del np


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
