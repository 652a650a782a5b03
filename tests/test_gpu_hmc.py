"""HMC on the GPU (jqcd_hmc_trajectory, jqcd_gauge_plaquette,
jqcd_gauge_download) against the oracle's trajectory of the paper's MD step:
the field and H after a trajectory, pure gauge and with two-flavour Wilson
fermions, the Metropolis decision with the link restore on rejection, and the
integrator's second-order energy error."""
import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth
from test_gpu_parity import rel

pytestmark = pytest.mark.gpu
BETA = 5.5


@pytest.fixture(scope="module")
def jq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd
    ctx = jqcd.Context(0)
    yield jqcd, ctx
    ctx.close()


def normals_for(dims, seed):
    return np.random.default_rng(seed).normal(size=(4,) + tuple(reversed(dims)) + (8,))


def test_plaquette_and_download(jq):
    jqcd, ctx = jq
    dims = (4, 6, 2, 8)
    g = ctx.gauge_upload(dims, synth.gauge(dims, "unit"))
    assert g.plaquette() == 1.0
    g.free()
    U = synth.gauge(dims, "haar", seed=171)
    g = ctx.gauge_upload(dims, U)
    assert abs(g.plaquette() - oracle.plaquette_sum(dims, U) / (18 * np.prod(dims))) < 1e-14
    assert np.array_equal(g.download(), U)
    g.free()


@pytest.mark.parametrize("fermions,dims", [(False, (4, 4, 4, 4)), (True, (4, 4, 4, 4)),
                                            (False, (8, 8, 8, 8))])
def test_trajectory_vs_oracle(jq, fermions, dims):
    """The trajectory against the oracle's; 8^4 without fermions covers the
    double-word staple force and the link exponential on a larger lattice."""
    jqcd, ctx = jq
    U = synth.gauge(dims, "expi", eps=0.5, seed=172)
    normals = normals_for(dims, 173)
    xi = synth.gaussian_spinor(dims, seed=174) if fermions else None
    g = ctx.gauge_upload(dims, U)
    info, st = g.hmc_trajectory(normals, xi, 0.0, BETA, kappa=0.12, n_md=4, tol=1e-12)
    assert st == 0 and info["accepted"] == 1
    U1, P1, H0, H1 = oracle.hmc_trajectory(dims, U, normals, xi, BETA, 0.12, n_md=4, tol=1e-13)
    gate = 1e-8 if fermions else 1e-11
    assert rel(g.download(), U1) <= gate
    assert abs(info["H_old"] - H0) <= 1e-10 * abs(H0)
    assert abs(info["H_new"] - H1) <= gate * abs(H1)
    assert abs(info["dH"] - (H1 - H0)) <= gate * abs(H1)
    assert abs(info["plaquette"] - oracle.plaquette_sum(dims, U1) / (18 * np.prod(dims))) <= 1e-12
    if fermions:
        assert info["cg_iters"] > 0
    g.free()


def test_metropolis_and_restore(jq):
    jqcd, ctx = jq
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "expi", eps=0.5, seed=175)
    g = ctx.gauge_upload(dims, U)
    # a coarse trajectory: |dH| well away from 0; u = 1 accepts only when dH <= 0
    info, st = g.hmc_trajectory(normals_for(dims, 176), None, 1.0, BETA, n_md=1, tau=1.5)
    assert st == 0 and info["accepted"] == (info["dH"] <= 0.0)
    if not info["accepted"]:
        assert np.array_equal(g.download(), U)
        assert abs(g.plaquette() - oracle.plaquette_sum(dims, U) / (18 * 256)) < 1e-14
    # u = 0 always accepts
    before = g.download()
    info, st = g.hmc_trajectory(normals_for(dims, 177), None, 0.0, BETA, n_md=2)
    assert st == 0 and info["accepted"] == 1 and not np.array_equal(g.download(), before)
    g.free()


@pytest.mark.parametrize("fermions", [False, True])
def test_second_order_energy_error(jq, fermions):
    jqcd, ctx = jq
    dims = (8, 8, 8, 8)
    U = synth.gauge(dims, "expi", eps=0.3, seed=178)
    normals = normals_for(dims, 179)
    xi = synth.gaussian_spinor(dims, seed=180) if fermions else None
    dH = []
    for n in (8, 16):
        g = ctx.gauge_upload(dims, U)
        info, st = g.hmc_trajectory(normals, xi, 0.0, BETA, kappa=0.12, n_md=n, tol=1e-12,
                                    mode=jqcd.CG_DW)
        assert st == 0
        dH.append(abs(info["dH"]))
        g.free()
    assert 2.8 < dH[0] / dH[1] < 5.5, dH
