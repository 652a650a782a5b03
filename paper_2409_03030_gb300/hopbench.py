"""Time one operator kernel alone: python -m paper_2409_03030_gb300.hopbench.

--op wilson (default): the even-odd Wilson hop in --prec; --op staggered: the
double-word staggered hop; --op force: the U dS/dU kernel of the fermion
force.  Prints one JSON line with the mean launch time (CUDA events on the
launching stream, after warm-up) and the algorithmic bandwidth (bytes per
output site: Wilson double-word/FP64 1536, FP32 576, FP16+norm 488, plus one
spinor when the axpy operand is read; staggered 1248 (+48); force 1536 per
site of the whole lattice).

--op cg: --iters whole even-odd CG solves (--mode, tolerance 1e-10) from one
Gaussian source, timed by the library's own events (gpu_seconds), for launch
lists of a complete solve; --delta, --eps and --kappa set the reliable-update
threshold, the links and the hopping parameter.

--op hmc: --iters trajectories (10 leapfrog steps, beta 5.5, two Wilson
flavours at --kappa, solves to 1e-10 in --mode; each trajectory is
accepted and the next one continues from its links), wall time per
trajectory.

--op multishift: --iters multi-shift solves of Mhat^dag Mhat + sigma for the
eight shifts 1e-4 ... 0.3 to 1e-10 (double-word) from one Gaussian even-site
right-hand side, timed by the library's events."""
from __future__ import annotations

import argparse
import json

import torch

from . import jqcd, synth

HOP_BYTES = {"dw": (1536, 192), "f64": (1536, 192), "f32": (576, 96), "f16n": (488, 52)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 48])
    ap.add_argument("--prec", default="dw", choices=sorted(HOP_BYTES))
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--axpy", action="store_true")
    ap.add_argument("--dagger", action="store_true")
    ap.add_argument("--op", default="wilson", choices=["wilson", "staggered", "force", "cg", "hmc", "multishift"])
    ap.add_argument("--mode", default="mixed_f16", choices=sorted(jqcd.MODES))
    ap.add_argument("--delta", type=float, default=0.0, help="reliable-update threshold (0: library default)")
    ap.add_argument("--eps", type=float, default=0.3, help="link generator exp(i eps H)")
    ap.add_argument("--kappa", type=float, default=0.12, help="hopping parameter of --op cg")
    a = ap.parse_args()
    dims = tuple(a.dims)
    prec = jqcd.PRECS[a.prec]
    ctx = jqcd.Context(0)
    g = ctx.gauge_upload(dims, synth.gauge(dims, "expi", eps=a.eps, seed=1))
    stream = torch.cuda.Stream()
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    if a.op == "hmc":
        import numpy as np
        rng = np.random.default_rng(62)
        normals = rng.normal(size=(4,) + tuple(reversed(dims)) + (8,))
        xi = synth.gaussian_spinor(dims, seed=63)
        mode = jqcd.MODES[a.mode]
        for _ in range(a.warmup):
            g.hmc_trajectory(normals, xi, 0.0, 5.5, kappa=a.kappa, n_md=2, tol=1e-10, mode=mode)
        secs, iters = [], 0
        for _ in range(a.iters):
            info, _ = g.hmc_trajectory(normals, xi, 0.0, 5.5, kappa=a.kappa, n_md=10, tol=1e-10, mode=mode)
            secs.append(info["seconds"])
            iters = info["cg_iters"]
        print(json.dumps({"op": "hmc", "dims": dims, "mode": a.mode, "cg_iters": iters,
                          "s_per_trajectory": round(sum(secs) / len(secs), 4)}))
        g.free()
        ctx.close()
        return
    if a.op == "multishift":
        shifts = [1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3]
        with torch.cuda.stream(stream):
            rhs, _ = g.pack(synth.gaussian_spinor(dims, seed=2), jqcd.PREC_DW, stream=stream)
            xs = [g.empty(jqcd.PREC_DW) for _ in shifts]
        for _ in range(a.warmup):
            g.cg_multishift_dev(rhs, xs, a.kappa, shifts, tol=1e-10, stream=stream)
        secs = []
        for _ in range(a.iters):
            infos, _ = g.cg_multishift_dev(rhs, xs, a.kappa, shifts, tol=1e-10, stream=stream)
            secs.append(infos[0]["gpu_seconds"])
        print(json.dumps({"op": "multishift", "dims": dims, "shifts": shifts, "kappa": a.kappa,
                          "iters": [i["iters"] for i in infos],
                          "ms_per_solve": round(1e3 * sum(secs) / len(secs), 3),
                          "max_true_rel_resid": max(i["true_rel_resid"] for i in infos)}))
        g.free()
        ctx.close()
        return
    if a.op == "cg":
        import numpy as np
        b = synth.gaussian_spinor(dims, seed=2)
        x = np.empty_like(b)
        for _ in range(a.warmup):
            g.cg_solve(b, a.kappa, tol=1e-10, mode=jqcd.MODES[a.mode], delta=a.delta, out=x)
        secs, iters = [], 0
        for _ in range(a.iters):
            _, info, _ = g.cg_solve(b, a.kappa, tol=1e-10, mode=jqcd.MODES[a.mode], delta=a.delta, out=x)
            secs.append(info["gpu_seconds"])
            iters = info["iters"]
        print(json.dumps({"op": "cg", "dims": dims, "mode": a.mode, "delta": a.delta, "eps": a.eps,
                          "kappa": a.kappa, "iters": iters, "reliable_updates": info["reliable_updates"],
                          "ms_per_solve": round(1e3 * sum(secs) / len(secs), 3),
                          "true_rel_resid": info["true_rel_resid"]}))
        g.free()
        ctx.close()
        return
    if a.op == "wilson":
        with torch.cuda.stream(stream):
            pe, po = g.pack(synth.gaussian_spinor(dims, seed=2), prec, stream=stream)
            out = g.empty(prec)
        x = pe if a.axpy else None
        launch = lambda: g.dslash_eo(prec, 0, int(a.dagger), po, x, out, 1.0, -0.12, stream=stream)  # noqa: E731
        per_site = HOP_BYTES[a.prec][0] + (HOP_BYTES[a.prec][1] if a.axpy else 0)
        n_sites = vh
    elif a.op == "staggered":
        with torch.cuda.stream(stream):
            pe, po = g.stag_pack(synth.gaussian_colour(dims, seed=2), stream=stream)
            out = g.stag_empty()
        x = pe if a.axpy else None
        launch = lambda: g.stag_dslash_eo(0, int(a.dagger), po, x, out, 1.0, -0.5, stream=stream)  # noqa: E731
        per_site, n_sites = 1248 + (48 if a.axpy else 0), vh
    else:
        with torch.cuda.stream(stream):
            xe, xo = g.pack(synth.gaussian_spinor(dims, seed=2), 0, stream=stream)
            ye, yo = g.pack(synth.gaussian_spinor(dims, seed=3), 0, stream=stream)
            out = torch.empty(g.linkfield_bytes(), dtype=torch.uint8, device=xe.device)
        launch = lambda: g.fermi_force_dev(0.12, xe, xo, ye, yo, out, stream=stream)  # noqa: E731
        per_site, n_sites = 1536, 2 * vh
    for _ in range(a.warmup):
        launch()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.iters):
        launch()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / a.iters
    vh = n_sites
    print(json.dumps({"op": a.op, "dims": dims, "prec": a.prec, "axpy": a.axpy, "dagger": a.dagger,
                      "us_per_launch": round(ms * 1e3, 2), "bytes_per_launch": vh * per_site,
                      "gbs": round(vh * per_site / (ms * 1e-3) / 1e9, 1)}))
    g.free()
    ctx.close()


if __name__ == "__main__":
    main()
