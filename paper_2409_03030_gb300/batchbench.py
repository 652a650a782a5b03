"""Time one batched solve of the point-source/Gaussian workload:
python -m paper_2409_03030_gb300.batchbench.

12 point sources (4 spins x 3 colours at the origin) on 24^3x48 and 12
Gaussian sources on 16^4, links exp(i 0.3 H), kappa 0.12, tolerance 1e-10,
mixed precision (FP16 inner by default), all through one
jqcd_cg_solve_batch call with pinned host buffers.  Prints one JSON line per
repetition."""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import jqcd, synth


def pinned(a):
    t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
    t.numpy()[...] = a
    return t.numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mode", default="mixed_f16", choices=["mixed_f16", "mixed_f32"])
    ap.add_argument("--verbose", action="store_true", help="phase times of each batch on stderr")
    a = ap.parse_args()
    ctx = jqcd.Context(0)
    dA, dB = (24, 24, 24, 48), (16, 16, 16, 16)
    gA = ctx.gauge_upload(dA, synth.gauge(dA, "expi", eps=0.3, seed=31))
    gB = ctx.gauge_upload(dB, synth.gauge(dB, "expi", eps=0.3, seed=32))
    bs = [pinned(synth.point_source(dA, s, c)) for s in range(4) for c in range(3)]
    bs += [pinned(synth.gaussian_spinor(dB, seed=100 + i)) for i in range(12)]
    gauges = [gA] * 12 + [gB] * 12
    outs = [pinned(b * 0) for b in bs]
    for rep in range(a.reps):
        t0 = time.perf_counter()
        xs, infos, st = ctx.cg_solve_batch(gauges, bs, [0.12] * 24, [1e-10] * 24,
                                           mode=jqcd.MODES[a.mode], verbose=2 if a.verbose else 0,
                                           out=outs)
        dt = time.perf_counter() - t0
        print(json.dumps({"rep": rep, "seconds": round(dt, 4), "status": st,
                          "iters": [infos[0]["iters"], infos[12]["iters"]],
                          "max_true_rel_resid": max(i["true_rel_resid"] for i in infos)}),
              flush=True)
    gA.free()
    gB.free()
    ctx.close()


if __name__ == "__main__":
    main()
