"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative 2-norm over the whole output field):
  double-word and native FP64 applies: 1e-12;  FP32: 1e-5;
  FP16 + per-site norm: 2e-3 (reported precision of the inner solver only).
Solves: the oracle recomputes the CG system's residual from the GPU solution
and it must be <= tol * (1 + 1e-6).
"""
import numpy as np
import pytest

import oracle
from conditioning import free_cond_eo
from paper_2409_03030_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 3: 1e-12, 1: 1e-5, 2: 2e-3}  # by precision code


@pytest.fixture(scope="module")
def jq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd
    ctx = jqcd.Context(0)
    yield jqcd, ctx
    ctx.close()


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def odd_mask(dims):
    return oracle.parity_mask(dims)[None, :, :, :, :, None]


def only_parity(dims, psi, parity):
    m = odd_mask(dims)
    return np.where(m if parity == 1 else ~m, psi, 0)


LATTICES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (6, 6, 6, 10), (8, 8, 8, 16)]
PRECS = [0, 3, 1, 2]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (6, 4, 2, 8)])
def test_pack_roundtrip(jq, dims, prec):
    jqcd, ctx = jq
    g = ctx.gauge_upload(dims, synth.gauge(dims, "unit"))
    psi = synth.gaussian_spinor(dims, seed=3)
    ev, od = g.pack(psi, prec)
    back = g.unpack(ev, od, prec)
    bound = {0: 1e-14, 3: 0.0, 1: 1e-7, 2: 1e-3}[prec]
    assert rel(back, psi) <= bound
    g.free()


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [0, 1])
def test_hop_vs_oracle(jq, dims, prec, dagger):
    jqcd, ctx = jq
    import torch
    U = synth.gauge(dims, "expi", eps=0.3, seed=11)
    g = ctx.gauge_upload(dims, U, t_antiperiodic=True)
    psi = synth.gaussian_spinor(dims, seed=12)
    xs = synth.gaussian_spinor(dims, seed=13)
    pe, po = g.pack(psi, prec)
    xe, xo = g.pack(xs, prec)
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for p in (0, 1):
        want_h = oracle.hop(dims, U, psi, dagger=bool(dagger), out_parity=p)
        inp = po if p == 0 else pe
        xin = xe if p == 0 else xo
        out = g.empty(prec)
        # plain hop with fused norm
        g.dslash_eo(prec, p, dagger, inp, None, out, 0.0, 1.0, norm2=norm)
        ev = out if p == 0 else g.empty(prec).zero_()
        od = out if p == 1 else g.empty(prec).zero_()
        got = only_parity(dims, g.unpack(ev, od, prec), p)
        assert rel(got, want_h) <= TOL[prec], (p, rel(got, want_h))
        n_want = np.linalg.norm(got) ** 2
        assert abs(norm.item() - n_want) <= max(TOL[prec], 1e-12) * 10 * n_want
        # fused axpy: out = a x + b H in
        a, b = 0.7, -0.12
        g.dslash_eo(prec, p, dagger, inp, xin, out, a, b)
        got = only_parity(dims, g.unpack(ev, od, prec), p)
        want = a * only_parity(dims, xs, p) + b * want_h
        assert rel(got, want) <= TOL[prec], (p, rel(got, want))
    g.free()


@pytest.mark.parametrize("mode", ["dw", "mixed_f16"])
def test_solve_bitwise_repeatable(jq, mode):
    """Reductions are fixed-order (per-block partials, then one single-block
    pass that issues all of a thread's loads before adding them in order), so
    the same solve run twice gives bit-identical solutions, iteration counts
    and residuals.  16^3x64: 1024 hop-block partials, four per thread in the
    single-block pass."""
    jqcd, ctx = jq
    dims = (16, 16, 16, 64)
    U = synth.gauge(dims, "expi", eps=0.3, seed=81)
    b = synth.gaussian_spinor(dims, seed=82)
    g = ctx.gauge_upload(dims, U)
    x1, i1, s1 = g.cg_solve(b, 0.12, tol=1e-10, mode=jqcd.MODES[mode])
    x2, i2, s2 = g.cg_solve(b, 0.12, tol=1e-10, mode=jqcd.MODES[mode])
    assert s1 == 0 and s2 == 0
    assert i1["iters"] == i2["iters"] and i1["reliable_updates"] == i2["reliable_updates"]
    assert i1["true_rel_resid"] == i2["true_rel_resid"] and i1["true_rel_resid"] <= 1e-10
    assert np.array_equal(x1, x2)
    g.free()


@pytest.mark.parametrize("case", ["nonunitary", "scaled_up", "scaled_down", "mixed_scales", "zero_block"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_hop_dw_magnitudes(jq, case, dagger):
    """Double-word hop at inputs that stress its offset-grid SU(3) sums, whose
    grid step is set per site and hop from max|link| and the half-spinor's
    magnitude: link components far above 1 (general complex matrices), spinors
    scaled by 2^60 and 2^-60, neighbours 2^80 apart in one launch (time slices
    0-3 at 2^40, 4-7 at 2^-40), and an all-zero region, whose outputs must be
    exact zeros.  Sites whose 8 neighbours share one scale are compared
    against the oracle per scale class, at the double-word gate."""
    jqcd, ctx = jq
    dims = (4, 4, 4, 8)
    U = synth.gauge(dims, "expi", eps=0.3, seed=31)
    psi = synth.gaussian_spinor(dims, seed=32)
    if case == "nonunitary":
        rng = np.random.default_rng(33)
        U = 3.0 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    elif case == "scaled_up":
        psi = psi * 2.0 ** 60
    elif case == "scaled_down":
        psi = psi * 2.0 ** -60
    elif case in ("mixed_scales", "zero_block"):
        t = np.arange(dims[3])[None, :, None, None, None, None]
        low = 0.0 if case == "zero_block" else 2.0 ** -40
        psi = psi * np.where(t < 4, 2.0 ** 40, low)
    g = ctx.gauge_upload(dims, U, t_antiperiodic=True)
    pe, po = g.pack(psi, 0)
    for p in (0, 1):
        want = oracle.hop(dims, U, psi, dagger=bool(dagger), out_parity=p)
        out = g.empty(0)
        g.dslash_eo(0, p, dagger, po if p == 0 else pe, None, out, 0.0, 1.0)
        ev = out if p == 0 else g.empty(0).zero_()
        od = out if p == 1 else g.empty(0).zero_()
        got = only_parity(dims, g.unpack(ev, od, 0), p)
        if case in ("mixed_scales", "zero_block"):
            for ts in ((1, 2), (5, 6)):  # output slices whose neighbours share one scale
                sl = (slice(None), slice(ts[0], ts[1] + 1))
                if case == "zero_block" and ts == (5, 6):
                    assert np.all(got[sl] == 0)
                    continue
                assert rel(got[sl], want[sl]) <= TOL[0], (p, ts, rel(got[sl], want[sl]))
            # slices on a scale boundary: error against the large scale
            assert np.linalg.norm((got - want).ravel()) <= TOL[0] * np.linalg.norm(want.ravel())
        else:
            assert rel(got, want) <= TOL[0], (p, rel(got, want))
    g.free()


@pytest.mark.parametrize("dims", [(10, 10, 10, 134), (10, 10, 10, 66)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_hop_dw_one_thread_per_site_ragged(jq, dagger, dims):
    """Double-word hop above the two-threads-per-site size, one thread per
    site with a ragged last block, with the fused axpy and norm, against the
    oracle: 10^3x134 (67,000 sites per parity) runs the kernel of large
    lattices, 10^3x66 (33,000, between the split limit and two blocks per SM
    on 152 SMs) the same kernel compiled for two blocks per SM.  Every smaller
    lattice of these tests runs the two-threads-per-site kernels."""
    jqcd, ctx = jq
    import torch
    assert np.prod(dims) // 2 > 29184 and (np.prod(dims) // 2) % 128 != 0
    U = synth.gauge(dims, "expi", eps=0.3, seed=41)
    g = ctx.gauge_upload(dims, U, t_antiperiodic=True)
    psi = synth.gaussian_spinor(dims, seed=42)
    xs = synth.gaussian_spinor(dims, seed=43)
    pe, po = g.pack(psi, 0)
    xe, xo = g.pack(xs, 0)
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for p in (0, 1):
        want = 0.7 * only_parity(dims, xs, p) - 0.12 * oracle.hop(dims, U, psi, dagger=bool(dagger),
                                                                   out_parity=p)
        out = g.empty(0)
        g.dslash_eo(0, p, dagger, po if p == 0 else pe, xe if p == 0 else xo, out, 0.7, -0.12,
                    norm2=norm)
        ev = out if p == 0 else g.empty(0).zero_()
        od = out if p == 1 else g.empty(0).zero_()
        got = only_parity(dims, g.unpack(ev, od, 0), p)
        assert rel(got, want) <= TOL[0], (p, rel(got, want))
        n_want = np.linalg.norm(got) ** 2
        assert abs(norm.item() - n_want) <= 1e-11 * n_want
    g.free()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 6, 10)])
@pytest.mark.parametrize("prec", PRECS)
def test_mdagm_vs_oracle(jq, dims, prec):
    jqcd, ctx = jq
    import torch
    U = synth.gauge(dims, "expi", eps=0.3, seed=21)
    g = ctx.gauge_upload(dims, U)
    v = only_parity(dims, synth.gaussian_spinor(dims, seed=22), 0)
    ve, vo = g.pack(v, prec)
    out = g.empty(prec)
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    k = 0.12
    g.mdagm(prec, k, ve, out, norm2=norm)
    got = only_parity(dims, g.unpack(out, vo, prec), 0)
    want = oracle.normal_apply(dims, U, v, k, eo=True)
    assert rel(got, want) <= TOL[prec]
    mv = oracle.schur(dims, U, v, k)
    assert abs(norm.item() - np.linalg.norm(mv) ** 2) <= max(TOL[prec], 1e-12) * 10 * np.linalg.norm(mv) ** 2
    g.free()


@pytest.mark.parametrize("prec", [0, 3, 1])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dirac_apply_vs_oracle(jq, prec, dagger):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=1)
    g = ctx.gauge_upload(dims, U)
    psi = synth.gaussian_spinor(dims, seed=1)
    ie, io = g.pack(psi, prec)
    oe, oo = g.empty(prec), g.empty(prec)
    g.dirac_apply(prec, 0.10, dagger, ie, io, oe, oo)
    got = g.unpack(oe, oo, prec)
    want = oracle.dirac(dims, U, psi, 0.10, dagger=bool(dagger))
    assert rel(got, want) <= TOL[prec]
    g.free()


def system_residual(dims, U, b, x, kappa, eo):
    """||rhs - A x|| / ||rhs|| of the CG system, recomputed by the oracle."""
    if eo:
        bhat = only_parity(dims, b, 0) + kappa * oracle.hop(dims, U, only_parity(dims, b, 1),
                                                            out_parity=0)
        rhs = oracle.schur(dims, U, bhat, kappa, dagger=True)
        r = rhs - oracle.normal_apply(dims, U, only_parity(dims, x, 0), kappa, eo=True)
    else:
        rhs = oracle.dirac(dims, U, b, kappa, dagger=True)
        r = rhs - oracle.normal_apply(dims, U, x, kappa, eo=False)
    return np.linalg.norm(r) / np.linalg.norm(rhs)


@pytest.mark.parametrize("eo", [False, True])
def test_cg_config0_4x4(jq, eo):
    """4^4, Haar links, kappa 0.10, antiperiodic time, Gaussian source, tol 1e-12."""
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=1)
    b = synth.gaussian_spinor(dims, seed=1)
    g = ctx.gauge_upload(dims, U)
    tol = 1e-12
    x, info, st = g.cg_solve(b, 0.10, tol=tol, eo=eo, mode=jqcd.CG_DW)
    assert st == 0 and info["iters"] > 0
    res = system_residual(dims, U, b, x, 0.10, eo)
    assert res <= tol * (1 + 1e-6), res
    assert abs(info["true_rel_resid"] - res) <= 1e-2 * tol + 1e-14
    full = rel(oracle.dirac(dims, U, x, 0.10), b)
    assert abs(info["full_rel_resid"] - full) <= 1e-13
    xo, *_ = oracle.solve(dims, U, b, 0.10, eo=eo, tol=1e-13)
    assert rel(x, xo) < 1e-10
    g.free()


def test_cg_config1_16x4(jq):
    """16^4, exp(i 0.3 H) links, kappa 0.12, even-odd, Gaussian source, tol 1e-10."""
    jqcd, ctx = jq
    dims = (16, 16, 16, 16)
    U = synth.gauge(dims, "expi", eps=0.3, seed=2)
    b = synth.gaussian_spinor(dims, seed=3)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-10, eo=True, mode=jqcd.CG_DW)
    assert st == 0
    res = system_residual(dims, U, b, x, 0.12, True)
    assert res <= 1e-10 * (1 + 1e-6), res
    g.free()


def test_cg_zero_source_and_limits(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=5)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(np.zeros(synth.spinor_shape(dims), complex), 0.1, tol=1e-10)
    assert st == 0 and info["iters"] == 0 and not np.any(x)
    b = synth.gaussian_spinor(dims, seed=6)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-14, maxiter=3, check=False)
    assert st == jqcd.ENOCONV and info["iters"] >= 3
    g.free()


def test_errors(jq):
    jqcd, ctx = jq
    with pytest.raises(jqcd.JqcdError) as e:
        ctx.gauge_upload((3, 4, 4, 4), np.zeros((4, 4, 4, 4, 3, 3, 3), complex))
    assert e.value.status == jqcd.EINVAL
    g = ctx.gauge_upload((2, 2, 2, 2), synth.gauge((2, 2, 2, 2), "unit"))
    g.free()
    with pytest.raises(jqcd.JqcdError) as e:
        g2 = jqcd.Gauge(ctx, 999999, (2, 2, 2, 2), True)
        g2.cg_solve(np.zeros(synth.spinor_shape((2, 2, 2, 2)), complex), 0.1)
    assert e.value.status == jqcd.ENOTFOUND


def test_hop_full_size_sampled(jq):
    """24^3x48 (the bench lattice): double-word hop at sampled output sites
    against the oracle's per-site hop."""
    jqcd, ctx = jq
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, "expi", eps=0.3, seed=7)
    psi = synth.gaussian_spinor(dims, seed=8)
    g = ctx.gauge_upload(dims, U)
    pe, po = g.pack(psi, 0)
    out_e, out_o = g.empty(0), g.empty(0)
    g.dslash_eo(0, 0, 0, po, None, out_e)
    g.dslash_eo(0, 1, 0, pe, None, out_o)
    got = g.unpack(out_e, out_o, 0).reshape(4, -1, 3)
    rng = np.random.default_rng(9)
    V = int(np.prod(dims))
    sites = np.unique(np.concatenate([rng.integers(0, V, 2000), [0, 1, V - 1, V - 2, V // 2]]))
    want = oracle.hop_sites(dims, U, psi, sites)
    got_s = np.transpose(got[:, sites, :], (1, 0, 2))
    assert rel(got_s, want) <= 1e-12
    g.free()


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16"])
def test_mixed_cg_16x4(jq, mode):
    """Mixed-precision CG (FP32 or FP16+norm inner, double-word reliable
    updates) reaches the requested true residual of the even-odd system, and
    agrees with the FP64 oracle's solution and with the double-word solve
    within the conditioning bound cond * (both residuals)."""
    jqcd, ctx = jq
    dims = (16, 16, 16, 16)
    U = synth.gauge(dims, "expi", eps=0.3, seed=2)
    b = synth.gaussian_spinor(dims, seed=3)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-10, eo=True, mode=jqcd.MODES[mode])
    assert st == 0 and info["reliable_updates"] >= 1
    res = system_residual(dims, U, b, x, 0.12, True)
    assert res <= 1e-10 * (1 + 1e-6), res
    assert abs(info["true_rel_resid"] - res) <= 1e-2 * 1e-10 + 1e-14
    xo, _, res_o, _, conv = oracle.solve(dims, U, b, 0.12, eo=True, tol=1e-13)
    assert conv
    bound = free_cond_eo(dims, 0.12) * (res + res_o)
    err = rel(only_parity(dims, x, 0), only_parity(dims, xo, 0))
    assert err <= bound, (err, bound)
    xd, info_d, st_d = g.cg_solve(b, 0.12, tol=1e-10, eo=True, mode=jqcd.CG_DW)
    assert rel(x, xd) < 1e-7
    g.free()


@pytest.mark.parametrize("eo", [False, True])
def test_cg_f64_config0_4x4(jq, eo):
    """Plain FP64 CG (JQCD_CG_F64: native FP64 hops, vectors and reductions):
    4^4 Haar links, kappa 0.10, tol 1e-12, whole-lattice D^dag D and even-odd.
    FP64 on both sides: the library's own true residual agrees with the
    oracle's recomputation to 1e-3 of tol, and x with the oracle's solution."""
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=1)
    b = synth.gaussian_spinor(dims, seed=1)
    g = ctx.gauge_upload(dims, U)
    tol = 1e-12
    x, info, st = g.cg_solve(b, 0.10, tol=tol, eo=eo, mode=jqcd.CG_F64)
    assert st == 0 and info["iters"] > 0 and info["reliable_updates"] == 0
    res = system_residual(dims, U, b, x, 0.10, eo)
    assert res <= tol * (1 + 1e-6), res
    assert abs(info["true_rel_resid"] - res) <= 1e-3 * tol
    full = rel(oracle.dirac(dims, U, x, 0.10), b)
    assert abs(info["full_rel_resid"] - full) <= 1e-14
    xo, *_ = oracle.solve(dims, U, b, 0.10, eo=eo, tol=1e-13)
    assert rel(x, xo) < 1e-10
    xd, _, _ = g.cg_solve(b, 0.10, tol=tol, eo=eo, mode=jqcd.CG_DW)
    assert rel(x, xd) < 1e-10
    g.free()


def test_cg_f64_config1_16x4(jq):
    """16^4, exp(i 0.3 H) links, kappa 0.12, even-odd, tol 1e-10 in plain FP64:
    the oracle's residual, the oracle's solution within cond * residuals, and
    the device-buffer entry (double-word b widened to FP64, x rounded back)
    giving the same solution to the double-word rounding of b and x."""
    jqcd, ctx = jq
    dims = (16, 16, 16, 16)
    U = synth.gauge(dims, "expi", eps=0.3, seed=2)
    b = synth.gaussian_spinor(dims, seed=3)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-10, eo=True, mode=jqcd.CG_F64)
    assert st == 0
    res = system_residual(dims, U, b, x, 0.12, True)
    assert res <= 1e-10 * (1 + 1e-6), res
    assert abs(info["true_rel_resid"] - res) <= 1e-3 * 1e-10
    xo, _, res_o, _, conv = oracle.solve(dims, U, b, 0.12, eo=True, tol=1e-13)
    err = rel(only_parity(dims, x, 0), only_parity(dims, xo, 0))
    assert err <= free_cond_eo(dims, 0.12) * (res + res_o), err
    be, bo = g.pack(b, jqcd.PREC_DW)
    xe, xo_dev = g.empty(jqcd.PREC_DW), g.empty(jqcd.PREC_DW)
    info_d, st_d = g.cg_solve_dev(be, bo, xe, xo_dev, 0.12, tol=1e-10, eo=True, mode=jqcd.CG_F64)
    assert st_d == 0
    xdev = g.unpack(xe, xo_dev, jqcd.PREC_DW)
    assert rel(xdev, x) <= 1e-9
    g.free()


def test_cg_f64_zero_source_and_limits(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=5)
    g = ctx.gauge_upload(dims, U)
    for eo in (True, False):
        x, info, st = g.cg_solve(np.zeros(synth.spinor_shape(dims), complex), 0.1, tol=1e-10,
                                 eo=eo, mode=jqcd.CG_F64)
        assert st == 0 and info["iters"] == 0 and not np.any(x)
    b = synth.gaussian_spinor(dims, seed=6)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-15, maxiter=3, mode=jqcd.CG_F64, check=False)
    assert st == jqcd.ENOCONV and info["iters"] >= 3
    # restart from the returned iterate (use_x0) reaches the tolerance
    x2, info2, st2 = g.cg_solve(b, 0.12, tol=1e-12, mode=jqcd.CG_F64, x0=x)
    assert st2 == 0 and system_residual(dims, U, b, x2, 0.12, True) <= 1e-12 * (1 + 1e-6)
    g.free()


@pytest.mark.parametrize("mode", ["dw", "mixed_f16", "mixed_f32", "f64"])
def test_tight_tol_24x48_oracle_residual(jq, mode):
    """tol 1e-12 on the 24^3x48 lattice (exp(i 0.3 H), kappa 0.12): the CG
    system's residual recomputed in FP64 by the oracle from the returned x
    meets the tolerance, in every solver mode."""
    jqcd, ctx = jq
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, "expi", eps=0.3, seed=1)
    b = synth.gaussian_spinor(dims, seed=2)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-12, eo=True, mode=jqcd.MODES[mode])
    assert st == 0
    res = system_residual(dims, U, b, x, 0.12, True)
    assert res <= 1e-12 * (1 + 1e-6), (res, info["true_rel_resid"])
    g.free()


def test_mixed_cg_config2_32x64(jq):
    """32^3x64, exp(i 0.4 H) links, kappa 0.122: FP16+norm mixed CG and plain
    FP64 CG to 1e-10.  Full size: the oracle recomputes the CG system's
    residual from each GPU solution, and solves the system itself to 1e-12;
    each GPU solution agrees with the oracle's within cond * residuals, and
    the two GPU solutions with each other."""
    jqcd, ctx = jq
    dims = (32, 32, 32, 64)
    U = synth.gauge(dims, "expi", eps=0.4, seed=4)
    b = synth.gaussian_spinor(dims, seed=5)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.122, tol=1e-10, eo=True, mode=jqcd.CG_MIXED_F16)
    assert st == 0
    res = system_residual(dims, U, b, x, 0.122, True)
    assert res <= 1e-10 * (1 + 1e-6), res
    x64, info64, st64 = g.cg_solve(b, 0.122, tol=1e-10, eo=True, mode=jqcd.CG_F64)
    assert st64 == 0
    res64 = system_residual(dims, U, b, x64, 0.122, True)
    assert res64 <= 1e-10 * (1 + 1e-6), res64
    xo, _, res_o, _, conv = oracle.solve(dims, U, b, 0.122, eo=True, tol=1e-12)
    assert conv
    cond = free_cond_eo(dims, 0.122)
    xe, x64e, xoe = (only_parity(dims, v, 0) for v in (x, x64, xo))
    assert rel(xe, xoe) <= cond * (res + res_o), (rel(xe, xoe), cond)
    assert rel(x64e, xoe) <= cond * (res64 + res_o), (rel(x64e, xoe), cond)
    assert rel(xe, x64e) <= cond * (res + res64)
    g.free()


def test_mixed_rejects_whole_lattice(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    g = ctx.gauge_upload(dims, synth.gauge(dims, "haar", seed=1))
    x, info, st = g.cg_solve(synth.gaussian_spinor(dims, seed=1), 0.1, eo=False,
                             mode=jqcd.CG_MIXED_F32, check=False)
    assert st == jqcd.EINVAL
    g.free()


@pytest.mark.parametrize("mode", ["dw", "mixed_f16"])
def test_cg_solve_pinned_host_buffers(jq, mode):
    """jqcd_cg_solve with page-locked b, x0 and x (the pack and unpack kernels
    read and write host memory directly) returns exactly what it returns for
    pageable buffers, with and without a start vector, on a ragged lattice."""
    jqcd, ctx = jq
    import torch
    dims = (6, 6, 6, 10)
    U = synth.gauge(dims, "expi", eps=0.3, seed=61)
    b = synth.gaussian_spinor(dims, seed=62)
    x0 = 0.5 * synth.gaussian_spinor(dims, seed=63)
    g = ctx.gauge_upload(dims, U)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    m = jqcd.MODES[mode]
    for start in (None, x0):
        x_ref, info_ref, _ = g.cg_solve(b, 0.12, tol=1e-10, mode=m, x0=start)
        out = pinned(np.full_like(b, np.nan))
        if start is not None:
            out[...] = start
        x_pin, info_pin, _ = g.cg_solve(pinned(b), 0.12, tol=1e-10, mode=m,
                                        x0=None if start is None else out, out=out)
        assert np.array_equal(x_pin, x_ref)
        assert info_pin["iters"] == info_ref["iters"]
        assert system_residual(dims, U, b, x_pin, 0.12, True) <= 1e-10 * (1 + 1e-6)
    g.free()


@pytest.mark.parametrize("mode", ["mixed_f16", "mixed_f32", "dw"])
def test_point_source_solve(jq, mode):
    """Point source (spin 2, colour 1 at the origin): the solution's support
    spreads one site per hop and its edge reaches denormal magnitudes."""
    jqcd, ctx = jq
    dims = (8, 8, 8, 16)
    U = synth.gauge(dims, "expi", eps=0.3, seed=9)
    b = synth.point_source(dims, 2, 1)
    g = ctx.gauge_upload(dims, U)
    x, info, st = g.cg_solve(b, 0.12, tol=1e-10, eo=True, mode=jqcd.MODES[mode])
    assert st == 0
    assert system_residual(dims, U, b, x, 0.12, True) <= 1e-10 * (1 + 1e-6)
    g.free()
