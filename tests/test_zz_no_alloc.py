"""jqcd_dslash_eo_noalloc: the allocation-free hop matches jqcd_dslash_eo.

The allocation-free entry point serves callers that cannot let the library
allocate device memory during a call (fixed HBM budgets, or streams that must
not be stalled by the device-wide synchronisation of cudaMalloc/cudaFree).
Its norm scratch is a fixed array inside the library that every call reuses,
so this test makes two calls in a row, with different operands, and compares
each with the allocating entry point through the C ABI, in every precision;
then a call without a norm, and a lattice above the fixed limit, which must
be refused before anything is launched.  The file name sorts last so that a
run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2409_03030_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3, 3: 1e-12}  # by precision: DW, FP32, FP16+norm, FP64


@pytest.fixture(scope="module")
def jq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd
    return jqcd, torch


def _whole(g, prec, buf, out_parity):
    zero = g.empty(prec).zero_()
    return g.unpack(buf if out_parity == 0 else zero, buf if out_parity == 1 else zero, prec)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_dslash_eo_twice(jq, prec):
    jqcd, torch = jq
    dims = (6, 6, 6, 10)  # 1080 sites per parity: several blocks and a ragged tail
    with jqcd.Context(0) as ctx:
        g = ctx.gauge_upload(dims, synth.gauge(dims, "expi", eps=0.3, seed=3))
        calls = [  # (out_parity, dagger, a, b, source seed)
            (0, 0, 0.7, -0.12, 10),
            (1, 1, 1.0, 0.5, 11),
        ]
        for out_parity, dagger, a, b, seed in calls:
            pe, po = g.pack(synth.gaussian_spinor(dims, seed=seed), prec)
            xe, xo = g.pack(synth.gaussian_spinor(dims, seed=seed + 100), prec)
            inp = po if out_parity == 0 else pe
            x = xe if out_parity == 0 else xo
            want, got = g.empty(prec), g.empty(prec)
            n_want = torch.zeros(1, dtype=torch.float64, device="cuda")
            n_got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            g.dslash_eo(prec, out_parity, dagger, inp, x, want, a, b, norm2=n_want)
            g.dslash_eo_noalloc(prec, out_parity, dagger, inp, x, got, a, b, norm2=n_got)
            torch.cuda.synchronize()
            w = _whole(g, prec, want, out_parity)
            r = _whole(g, prec, got, out_parity)
            err = np.linalg.norm(r - w) / np.linalg.norm(w)
            assert err <= TOL[prec], err
            assert abs(n_got.item() - n_want.item()) <= TOL[prec] * n_want.item()
        g.free()


@pytest.mark.parametrize("prec", [0, 3])
def test_noalloc_without_norm(jq, prec):
    """norm2 = NULL: no scratch is touched; the plain hop (no axpy) matches."""
    jqcd, torch = jq
    dims = (4, 4, 4, 8)
    with jqcd.Context(0) as ctx:
        g = ctx.gauge_upload(dims, synth.gauge(dims, "expi", eps=0.3, seed=5))
        pe, po = g.pack(synth.gaussian_spinor(dims, seed=6), prec)
        want, got = g.empty(prec), g.empty(prec)
        g.dslash_eo(prec, 1, 0, pe, None, want)
        g.dslash_eo_noalloc(prec, 1, 0, pe, None, got)
        torch.cuda.synchronize()
        w, r = _whole(g, prec, want, 1), _whole(g, prec, got, 1)
        assert np.linalg.norm(r - w) <= TOL[prec] * np.linalg.norm(w)
        g.free()


def test_noalloc_rejects_lattice_above_limit(jq):
    """A lattice with more sites per parity than the fixed scratch covers is
    refused with JQCD_EINVAL before any launch (the small buffers passed here
    are never read)."""
    jqcd, torch = jq
    dims = (32, 32, 32, 130)  # 2,129,920 sites per parity > 2,097,152
    assert np.prod(dims) // 2 > jqcd.NOALLOC_MAX_SITES_PER_PARITY
    with jqcd.Context(0) as ctx:
        g = ctx.gauge_upload(dims, synth.gauge(dims, "unit"))
        a = torch.zeros(256, dtype=torch.uint8, device="cuda")
        b = torch.zeros(256, dtype=torch.uint8, device="cuda")
        n = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(jqcd.JqcdError) as e:
            g.dslash_eo_noalloc(0, 0, 0, a, None, b, norm2=n)
        assert e.value.status == jqcd.EINVAL
        assert "limit" in str(e.value)
        g.free()
