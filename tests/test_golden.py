"""The paper's worked example (section "Definition of Dirac operators": 4^4
cold start, kappa = 0.141139, eps_CG = 1.0e-8) as stored golden values.

CPU: the stored values equal the free-field closed form in momentum space
(independent of the oracle) and the oracle still reproduces them.
GPU: the CUDA path reproduces them (apply and solve) through the C ABI."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_example_4x4x4x4.json")))
DIMS = tuple(GOLD["dims"])
KAPPA = GOLD["kappa"]
SAMPLES = [tuple(s) for s in GOLD["samples"]]
G = np.array([  # DeGrand-Rossi, mu = x, y, z, t
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=complex)


def source():
    return synth.gaussian_spinor(DIMS, seed=GOLD["source_seed"])


def stored(key):
    return np.array([complex(*v) for v in GOLD[key]])


def free_field(psi, inverse=False):
    """D psi (or D^-1 psi) for unit links and antiperiodic time, by the
    momentum-space symbol D(p) = (1 - 2 kappa sum cos p) + 2i kappa sum gamma sin p."""
    nx, ny, nz, nt = DIMS
    t = np.arange(nt)[:, None, None, None]
    twist = np.exp(-1j * np.pi * t / nt)  # antiperiodic -> periodic
    f = np.fft.fftn(psi * twist[None, ..., None], axes=(1, 2, 3, 4))
    kt, kz, ky, kx = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx),
                                 indexing="ij")
    p = np.stack([2 * np.pi * kx / nx, 2 * np.pi * ky / ny, 2 * np.pi * kz / nz,
                  (2 * np.pi * kt + np.pi) / nt])  # [mu, t, z, y, x]
    sym = ((1 - 2 * KAPPA * np.cos(p).sum(0))[..., None, None] * np.eye(4)
           + 2j * KAPPA * np.einsum("mtzyx,mab->tzyxab", np.sin(p), G))
    if inverse:
        sym = np.linalg.inv(sym)
    g = np.einsum("tzyxab,btzyxc->atzyxc", sym, f)
    return np.fft.ifftn(g, axes=(1, 2, 3, 4)) / twist[None, ..., None]


def test_golden_is_the_free_field_closed_form():
    x = source()
    assert abs(np.linalg.norm(x) - GOLD["norm_x"]) <= 1e-13 * GOLD["norm_x"]
    dx = free_field(x)
    assert abs(np.linalg.norm(dx) - GOLD["norm_Dx"]) <= 1e-13 * GOLD["norm_Dx"]
    want = np.array([dx[s] for s in SAMPLES])
    assert np.max(np.abs(stored("Dx") - want)) <= 1e-13 * GOLD["norm_Dx"]
    y = free_field(x, inverse=True)
    assert abs(np.linalg.norm(y) - GOLD["norm_y"]) <= 1e-11 * GOLD["norm_y"]
    want = np.array([y[s] for s in SAMPLES])
    assert np.max(np.abs(stored("y") - want)) <= 1e-11 * GOLD["norm_y"]


def test_oracle_reproduces_golden():
    U = synth.gauge(DIMS, "unit")
    x = source()
    dx = oracle.dirac(DIMS, U, x, KAPPA)
    assert np.max(np.abs(np.array([dx[s] for s in SAMPLES]) - stored("Dx"))) <= 1e-14 * GOLD["norm_Dx"]
    y, iters, sys_rel, full_rel, ok = oracle.solve(DIMS, U, x, KAPPA, eo=False, tol=GOLD["cg_tol"],
                                                   maxiter=100000)
    assert ok and sys_rel <= GOLD["cg_tol"]
    assert np.max(np.abs(np.array([y[s] for s in SAMPLES]) - stored("y"))) <= 1e-13 * GOLD["norm_y"]


@pytest.fixture(scope="module")
def jq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd
    ctx = jqcd.Context(0)
    yield jqcd, ctx
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-12), (1, 1e-5)])
def test_gpu_apply_matches_golden(jq, prec, tol):
    jqcd, ctx = jq
    g = ctx.gauge_upload(DIMS, synth.gauge(DIMS, "unit"))
    ie, io = g.pack(source(), prec)
    oe, oo = g.empty(prec), g.empty(prec)
    g.dirac_apply(prec, KAPPA, 0, ie, io, oe, oo)
    got = g.unpack(oe, oo, prec)
    assert abs(np.linalg.norm(got) - GOLD["norm_Dx"]) <= tol * GOLD["norm_Dx"]
    assert np.max(np.abs(np.array([got[s] for s in SAMPLES]) - stored("Dx"))) <= tol * GOLD["norm_Dx"]
    g.free()


@pytest.mark.gpu
@pytest.mark.parametrize("eo,mode", [(False, "dw"), (True, "dw"), (True, "mixed_f16")])
def test_gpu_solve_matches_golden(jq, eo, mode):
    """solve_DinvX! of the example at the paper's eps_CG = 1e-8."""
    jqcd, ctx = jq
    g = ctx.gauge_upload(DIMS, synth.gauge(DIMS, "unit"))
    y, info, st = g.cg_solve(source(), KAPPA, tol=1e-8, eo=eo, mode=jqcd.MODES[mode])
    assert st == 0 and info["true_rel_resid"] <= 1e-8
    # error of the solution <= cond(D^dag D)-ish * tol; the free 4^4 operator is well conditioned
    err = np.max(np.abs(np.array([y[s] for s in SAMPLES]) - stored("y"))) / GOLD["norm_y"]
    assert err <= 1e-6, err
    assert np.linalg.norm(y - free_field(source(), inverse=True)) <= 1e-6 * GOLD["norm_y"]
    g.free()
