"""Multi-shift CG on the GPU (jqcd_cg_multishift / _dev) against the oracle's
shifted textbook CG: every shift's solution, its true residual recomputed by
the oracle, edge cases, and the property checks at 24^3x48."""
import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth
from test_gpu_parity import rel

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


def shifted_residual(dims, U, rhs, x, kappa, sigma):
    r = rhs - oracle.normal_apply(dims, U, x, kappa, eo=True) - sigma * x
    return np.linalg.norm(r) / np.linalg.norm(rhs)


@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 4), "haar"), ((6, 4, 2, 8), "expi"),
                                       ((8, 8, 8, 8), "expi")])
def test_multishift_vs_oracle(jq, dims, kind):
    jqcd, ctx = jq
    U = synth.gauge(dims, kind, eps=0.3, seed=101)
    rhs = oracle.zero_parity(dims, synth.gaussian_spinor(dims, seed=102), 1)
    shifts = [0.0, 1e-3, 0.02, 0.3, 2.5]
    g = ctx.gauge_upload(dims, U)
    tol = 1e-12
    xs, infos, st = g.cg_multishift(rhs, 0.12, shifts, tol=tol)
    assert st == 0
    odd = np.broadcast_to(oracle.parity_mask(dims)[None, ..., None], rhs.shape)
    for sigma, x, info in zip(shifts, xs, infos):
        assert info["status"] == 0 and info["iters"] > 0
        assert not np.any(x[odd])
        res = shifted_residual(dims, U, rhs, x, 0.12, sigma)
        assert res <= tol * (1 + 1e-6), (sigma, res)
        assert abs(info["true_rel_resid"] - res) <= 1e-2 * tol + 1e-15
        xo, _, _, ok = oracle.cg_shift(dims, U, rhs, 0.12, sigma, eo=True, tol=1e-13, maxiter=20000)
        assert ok and rel(x, xo) <= 1e-9
    # larger shifts converge no later than smaller ones
    its = [i["iters"] for i in infos]
    assert its == sorted(its, reverse=True)
    g.free()


def test_multishift_edge_cases(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=103)
    g = ctx.gauge_upload(dims, U)
    zero = np.zeros(synth.spinor_shape(dims), complex)
    xs, infos, st = g.cg_multishift(zero, 0.12, [0.0, 0.5])
    assert st == 0 and all(not np.any(x) for x in xs) and all(i["iters"] == 0 for i in infos)
    rhs = oracle.zero_parity(dims, synth.gaussian_spinor(dims, seed=104), 1)
    for bad in ([-0.1], [float("nan")], [0.1] * 33, []):
        _, _, st = g.cg_multishift(rhs, 0.12, bad, check=False)
        assert st == jqcd.EINVAL, bad
    # a single shift of zero is the plain CG on Mhat^dag Mhat
    xs, infos, st = g.cg_multishift(rhs, 0.12, [0.0], tol=1e-12)
    xo, *_ = oracle.cg(dims, U, rhs, 0.12, eo=True, tol=1e-13)
    assert st == 0 and rel(xs[0], xo) <= 1e-9
    # maxiter too small: ENOCONV, infos filled
    xs, infos, st = g.cg_multishift(rhs, 0.12, [0.0, 0.1], tol=1e-12, maxiter=3, check=False)
    assert st == jqcd.ENOCONV and infos[0]["iters"] == 3
    g.free()


def test_multishift_full_size(jq):
    """24^3x48, eight RHMC-like shifts, tol 1e-10 through the device entry:
    every reported true residual meets tol, and one shift's residual is
    recomputed by the oracle."""
    jqcd, ctx = jq
    import torch
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, "expi", eps=0.3, seed=105)
    b = synth.gaussian_spinor(dims, seed=106)
    g = ctx.gauge_upload(dims, U)
    shifts = [1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3]
    be, bo = g.pack(b, jqcd.PREC_DW)
    xe = [g.empty(jqcd.PREC_DW) for _ in shifts]
    infos, st = g.cg_multishift_dev(be, xe, 0.12, shifts, tol=1e-10)
    assert st == 0
    assert all(i["true_rel_resid"] <= 1e-10 * (1 + 1e-6) for i in infos)
    zero = g.empty(jqcd.PREC_DW)
    zero.zero_()
    x3 = g.unpack(xe[3], zero, jqcd.PREC_DW)
    rhs = oracle.zero_parity(dims, b, 1)
    res = shifted_residual(dims, U, rhs, x3, 0.12, shifts[3])
    assert res <= 1e-10 * (1 + 1e-6) and abs(res - infos[3]["true_rel_resid"]) <= 1e-12
    g.free()
