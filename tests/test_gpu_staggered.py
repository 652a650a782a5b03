"""Staggered operator and solver on the GPU against the FP64 oracle: hop per
parity (adjoint, axpy, fused norm), whole-lattice D and D^dag, the even-odd
solve (true residuals recomputed by the oracle), edge cases, and a 24^3x48
solve checked through one oracle apply."""
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


def only_parity(dims, f, parity):
    odd = oracle.parity_mask(dims)[..., None]
    return np.where(odd == bool(parity), f, 0)


LATTICES = [((4, 4, 4, 4), True), ((6, 4, 2, 8), True), ((2, 2, 2, 2), True), ((4, 6, 2, 4), False),
            ((8, 8, 8, 16), True)]


@pytest.mark.parametrize("dims,tanti", LATTICES)
@pytest.mark.parametrize("dagger", [0, 1])
def test_staggered_hop_vs_oracle(jq, dims, tanti, dagger):
    jqcd, ctx = jq
    import torch
    U = synth.gauge(dims, "haar", seed=131)
    psi = synth.gaussian_colour(dims, seed=132)
    xf = synth.gaussian_colour(dims, seed=133)
    g = ctx.gauge_upload(dims, U, t_antiperiodic=tanti)
    ie, io = g.stag_pack(psi)
    xe, xo = g.stag_pack(xf)
    for p in (0, 1):
        src, xp = (io, xe) if p == 0 else (ie, xo)
        out = g.stag_empty()
        n2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.stag_dslash_eo(p, dagger, src, xp, out, a=0.3, b=-0.7, norm2=n2)
        zero = g.stag_empty()
        zero.zero_()
        got = g.stag_unpack(out, zero) if p == 0 else g.stag_unpack(zero, out)
        hop = oracle.stag_hop(dims, U, psi, dagger=bool(dagger), out_parity=p, t_antiperiodic=tanti)
        want = 0.3 * only_parity(dims, xf, p) - 0.7 * hop
        assert rel(got, want) <= 1e-12
        assert abs(n2.item() - np.vdot(want, want).real) <= 1e-12 * np.vdot(want, want).real
    g.free()


@pytest.mark.parametrize("dagger", [0, 1])
def test_staggered_apply_vs_oracle(jq, dagger):
    jqcd, ctx = jq
    dims = (6, 4, 4, 8)
    U = synth.gauge(dims, "expi", eps=0.3, seed=134)
    psi = synth.gaussian_colour(dims, seed=135)
    g = ctx.gauge_upload(dims, U)
    ie, io = g.stag_pack(psi)
    oe, oo = g.stag_empty(), g.stag_empty()
    g.stag_apply(0.05, dagger, ie, io, oe, oo)
    assert rel(g.stag_unpack(oe, oo), oracle.stag_dirac(dims, U, psi, 0.05, dagger=bool(dagger))) <= 1e-12
    g.free()


@pytest.mark.parametrize("dims,mass,tol", [((4, 4, 4, 4), 0.1, 1e-12), ((8, 8, 8, 8), 0.05, 1e-10),
                                           ((6, 4, 2, 8), 0.2, 1e-12)])
def test_staggered_solve_vs_oracle(jq, dims, mass, tol):
    jqcd, ctx = jq
    U = synth.gauge(dims, "expi", eps=0.3, seed=136)
    b = synth.gaussian_colour(dims, seed=137)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.stag_solve(b, mass, tol=tol)
    assert st == 0 and info["iters"] > 0
    assert info["true_rel_resid"] <= tol
    # even-odd system residual recomputed by the oracle
    be, bo = only_parity(dims, b, 0), only_parity(dims, b, 1)
    rhs = mass * be - oracle.stag_hop(dims, U, bo, out_parity=0)
    xe = only_parity(dims, x, 0)
    Ax = mass ** 2 * xe - oracle.stag_hop(dims, U, oracle.stag_hop(dims, U, xe, out_parity=1), out_parity=0)
    res = np.linalg.norm(rhs - Ax) / np.linalg.norm(rhs)
    assert res <= tol * (1 + 1e-6) and abs(res - info["true_rel_resid"]) <= 1e-2 * tol + 1e-15
    full = rel(oracle.stag_dirac(dims, U, x, mass), b)
    assert abs(full - info["full_rel_resid"]) <= 1e-3 * full + 1e-13
    xo, *_ = oracle.stag_solve(dims, U, b, mass, tol=1e-13)
    assert rel(x, xo) <= 1e3 * tol
    g.free()


def test_staggered_edge_cases(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    g = ctx.gauge_upload(dims, synth.gauge(dims, "haar", seed=138))
    zero = np.zeros(g.colour_shape(), complex)
    x, info, st = g.stag_solve(zero, 0.1)
    assert st == 0 and not np.any(x) and info["iters"] == 0
    b = synth.gaussian_colour(dims, seed=139)
    for bad in (0.0, -0.1, float("nan")):
        _, _, st = g.stag_solve(b, bad, check=False)
        assert st == jqcd.EINVAL
    _, info, st = g.stag_solve(b, 0.01, tol=1e-14, maxiter=5, check=False)
    assert st == jqcd.ENOCONV and info["iters"] >= 5
    g.free()


def test_staggered_full_size(jq):
    """24^3x48 through the device entry: the residual of the returned x is
    recomputed by one oracle apply."""
    jqcd, ctx = jq
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, "expi", eps=0.3, seed=140)
    b = synth.gaussian_colour(dims, seed=141)
    g = ctx.gauge_upload(dims, U)
    be, bo = g.stag_pack(b)
    xe, xo = g.stag_empty(), g.stag_empty()
    info, st = g.stag_solve_dev(be, bo, xe, xo, 0.05, tol=1e-10)
    assert st == 0
    x = g.stag_unpack(xe, xo)
    full = rel(oracle.stag_dirac(dims, U, x, 0.05), b)
    assert abs(full - info["full_rel_resid"]) <= 1e-3 * full + 1e-13
    # |b - Dx| = |r_e| / m and |rhs_e| <= (m + 4) |b| (||D_hop|| <= 4): full <= tol (m + 4) / m
    assert full <= 1e-10 * (0.05 + 4) / 0.05
    g.free()
