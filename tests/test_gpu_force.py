"""Fermion action and force on the GPU (jqcd_fermi_action / _force / _force_xy /
_force_dev) against the FP64 oracle: the per-link kernel on given X, Y to
1e-12; the whole pipeline (two even-odd solves, Re <eta, X>, the kernel)
within the solves' tolerance; the heatbath identity; sampled links of the
kernel at 24^3x48 in the launch configuration the benchmark times."""
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


@pytest.mark.parametrize("dims,tanti", [((4, 4, 4, 4), True), ((6, 4, 2, 8), True),
                                        ((2, 2, 2, 2), True), ((4, 2, 6, 4), False)])
def test_force_kernel_vs_oracle(jq, dims, tanti):
    jqcd, ctx = jq
    U = synth.gauge(dims, "haar", seed=61)
    X = synth.gaussian_spinor(dims, seed=62)
    Y = synth.gaussian_spinor(dims, seed=63)
    g = ctx.gauge_upload(dims, U, t_antiperiodic=tanti)
    got = g.fermi_force_xy(X, Y, 0.12)
    want = oracle.fermi_force_xy(dims, U, X, Y, 0.12, t_antiperiodic=tanti)
    assert rel(got, want) <= 1e-12
    g.free()


@pytest.mark.parametrize("mode,tol,gate", [("dw", 1e-12, 1e-9), ("mixed_f16", 1e-10, 1e-7),
                                           ("mixed_f32", 1e-10, 1e-7)])
def test_action_and_force_vs_oracle(jq, mode, tol, gate):
    jqcd, ctx = jq
    dims = (4, 4, 4, 8)
    U = synth.gauge(dims, "expi", eps=0.3, seed=64)
    eta = synth.gaussian_spinor(dims, seed=65)
    g = ctx.gauge_upload(dims, U)
    S, G, info, st = g.fermi_force(eta, 0.12, tol=tol, mode=jqcd.MODES[mode])
    assert st == 0 and info["iters"] > 0 and info["true_rel_resid"] <= tol
    S_o, G_o = oracle.fermi_force(dims, U, eta, 0.12, tol=1e-13)
    assert abs(S - S_o) <= gate * S_o, (S, S_o)
    assert rel(G, G_o) <= gate
    S2, info2, st2 = g.fermi_action(eta, 0.12, tol=tol, mode=jqcd.MODES[mode])
    assert st2 == 0 and abs(S2 - S) <= 1e-12 * S
    g.free()


def test_heatbath_identity_gpu(jq):
    """eta = D^dag xi (jqcd_dirac_apply, dagger) gives S = |xi|^2."""
    jqcd, ctx = jq
    dims = (8, 8, 8, 8)
    U = synth.gauge(dims, "expi", eps=0.3, seed=66)
    xi = synth.gaussian_spinor(dims, seed=67)
    g = ctx.gauge_upload(dims, U)
    ie, io = g.pack(xi, jqcd.PREC_DW)
    oe, oo = g.empty(jqcd.PREC_DW), g.empty(jqcd.PREC_DW)
    g.dirac_apply(jqcd.PREC_DW, 0.12, 1, ie, io, oe, oo)
    eta = g.unpack(oe, oo, jqcd.PREC_DW)
    S, info, st = g.fermi_action(eta, 0.12, tol=1e-12)
    assert st == 0
    assert abs(S - np.vdot(xi, xi).real) <= 1e-10 * S
    g.free()


def decode_linkfield(buf, dims):
    """[parity][mu][3a+b][cb] chunks (re.h, im.h, re.l, im.l) -> links [mu,t,z,y,x,b,a]."""
    nx, ny, nz, nt = dims
    vh = nx * ny * nz * nt // 2
    f = buf.cpu().numpy().view(np.float32).reshape(2, 4, 9, vh, 4).astype(np.float64)
    val = (f[..., 0] + f[..., 2]) + 1j * (f[..., 1] + f[..., 3])       # [p, mu, k, cb]
    cb = np.arange(vh)
    r = cb // (nx // 2)
    y, z, t = r % ny, (r // ny) % nz, r // (ny * nz)
    out = np.empty((4, nt, nz, ny, nx, 3, 3), dtype=complex)
    for p in range(2):
        x = 2 * (cb % (nx // 2)) + ((y + z + t + p) & 1)
        for k in range(9):
            a, b = divmod(k, 3)
            out[:, t, z, y, x, b, a] = val[p, :, k, :]
    return out


def test_force_full_size_sampled(jq):
    """24^3x48: the device entry (as timed by the benchmark) on X, Y resident in
    HBM, 2048 sampled links against the oracle, plus the host entry's field."""
    jqcd, ctx = jq
    import torch
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, "expi", eps=0.3, seed=68)
    X = synth.gaussian_spinor(dims, seed=69)
    Y = synth.gaussian_spinor(dims, seed=70)
    g = ctx.gauge_upload(dims, U)
    xe, xo = g.pack(X, jqcd.PREC_DW)
    ye, yo = g.pack(Y, jqcd.PREC_DW)
    out = torch.empty(g.linkfield_bytes(), dtype=torch.uint8, device="cuda")
    g.fermi_force_dev(0.12, xe, xo, ye, yo, out)
    torch.cuda.synchronize()
    G = g.fermi_force_xy(X, Y, 0.12)  # same kernel, host-layout result
    V = int(np.prod(dims))
    rng = np.random.default_rng(71)
    links = np.concatenate([rng.integers(0, 4 * V, 2000),
                            3 * V + (dims[3] - 1) * V // dims[3] + np.arange(48)])  # t = NT-1 links
    want = oracle.fermi_force_links(dims, U, X, Y, 0.12, links)
    got = G.reshape(4 * V, 3, 3)[links]
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-12 * scale
    # the device entry's double-word link field, decoded here, is the same field
    assert np.array_equal(decode_linkfield(out, dims), G)
    g.free()
