"""Batched mixed-precision CG (jqcd_cg_solve_batch) against single solves and
the FP64 oracle: uneven lattices, different kappa and tolerances in one batch,
and the 24-solve point-source/Gaussian workload at full size."""
import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth
from test_gpu_parity import only_parity, rel, system_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd
    ctx = jqcd.Context(0)
    yield jqcd, ctx
    ctx.close()


def host_buffer(a, pinned):
    """a itself (pageable) or a copy in page-locked memory, which the engine
    moves on its copy stream."""
    if not pinned:
        return a
    import torch
    t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
    t.numpy()[...] = a
    return t.numpy()


@pytest.mark.parametrize("mode,host", [("mixed_f16", "pageable"), ("mixed_f32", "pageable"),
                                       ("mixed_f16", "pinned"), ("mixed_f16", "mixed")])
def test_batch_mixed_lattices(jq, mode, host):
    jqcd, ctx = jq
    d1, d2, d3 = (8, 8, 8, 8), (6, 6, 6, 10), (4, 4, 4, 4)
    U1 = synth.gauge(d1, "expi", eps=0.3, seed=1)
    U2 = synth.gauge(d2, "expi", eps=0.3, seed=2)
    U3 = synth.gauge(d3, "haar", seed=3)
    g1, g2, g3 = ctx.gauge_upload(d1, U1), ctx.gauge_upload(d2, U2), ctx.gauge_upload(d3, U3)
    solves = []  # (gauge, U, dims, b, kappa, tol)
    for s in range(4):
        solves.append((g1, U1, d1, synth.point_source(d1, s, s % 3), 0.12, 1e-10))
    for s in range(3):
        solves.append((g2, U2, d2, synth.gaussian_spinor(d2, seed=20 + s), 0.11 + 0.005 * s,
                       [1e-8, 1e-10, 1e-12][s]))
    solves.append((g3, U3, d3, synth.gaussian_spinor(d3, seed=30), 0.10, 1e-12))
    solves.append((g3, U3, d3, np.zeros(synth.spinor_shape(d3), complex), 0.10, 1e-10))
    # pinned: sources and solutions through the copy stream; mixed: alternate
    pin = [host == "pinned" or (host == "mixed" and i % 2 == 0) for i in range(len(solves))]
    bs = [host_buffer(s[3], p) for s, p in zip(solves, pin)]
    outs = [host_buffer(np.full_like(s[3], np.nan), p) for s, p in zip(solves, pin)]
    xs, infos, st = ctx.cg_solve_batch([s[0] for s in solves], bs,
                                       [s[4] for s in solves], [s[5] for s in solves],
                                       mode=jqcd.MODES[mode], out=outs)
    assert st == 0
    for (g, U, dims, b, k, tol), x, info in zip(solves, xs, infos):
        assert info["status"] == 0
        if not np.any(b):
            assert not np.any(x) and info["iters"] == 0
            continue
        res = system_residual(dims, U, b, x, k, True)
        assert res <= tol * (1 + 1e-6), (dims, k, tol, res)
        assert abs(info["true_rel_resid"] - res) <= 1e-2 * tol + 1e-14
        full = rel(oracle.dirac(dims, U, x, k), b)
        assert abs(info["full_rel_resid"] - full) <= 1e-3 * full + 1e-13
        # the same solve alone
        xa, ia, sa = g.cg_solve(b, k, tol=tol, eo=True, mode=jqcd.MODES[mode])
        assert rel(x, xa) <= 1e3 * tol
    for g in (g1, g2, g3):
        g.free()


def test_batch_config3_full(jq):
    """12 point sources on 24^3x48 and 12 Gaussian sources on 16^4,
    exp(i 0.3 H) links, kappa 0.12, tol 1e-10, one batch."""
    jqcd, ctx = jq
    dA, dB = (24, 24, 24, 48), (16, 16, 16, 16)
    UA = synth.gauge(dA, "expi", eps=0.3, seed=31)
    UB = synth.gauge(dB, "expi", eps=0.3, seed=32)
    gA, gB = ctx.gauge_upload(dA, UA), ctx.gauge_upload(dB, UB)
    bsA = [synth.point_source(dA, s, c) for s in range(4) for c in range(3)]
    bsB = [synth.gaussian_spinor(dB, seed=100 + i) for i in range(12)]
    gauges = [gA] * 12 + [gB] * 12
    xs, infos, st = ctx.cg_solve_batch(gauges, bsA + bsB, [0.12] * 24, [1e-10] * 24,
                                       mode=jqcd.CG_MIXED_F16)
    assert st == 0
    for i in (0, 5, 11):
        assert system_residual(dA, UA, bsA[i], xs[i], 0.12, True) <= 1e-10 * (1 + 1e-6)
    for i in (12, 17, 23):
        assert system_residual(dB, UB, bsB[i - 12], xs[i], 0.12, True) <= 1e-10 * (1 + 1e-6)
    assert all(inf["status"] == 0 and inf["true_rel_resid"] <= 1e-10 for inf in infos)
    gA.free()
    gB.free()
