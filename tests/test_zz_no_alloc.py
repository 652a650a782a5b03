"""jqcd_dslash_eo_noalloc: the allocation-free hop matches jqcd_dslash_eo.

The allocation-free entry point serves callers that cannot let the library
allocate device memory during a call (fixed HBM budgets, or streams that must
not be stalled by the device-wide synchronisation of cudaMalloc/cudaFree).
Its norm scratch is a fixed array inside the library that every call reuses,
so this test makes two calls in a row, with different operands, and compares
each with the allocating entry point through the C ABI.  The file name sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2409_03030_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_dslash_eo_twice(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03030_gb300 import jqcd

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
            zero = g.empty(prec).zero_()
            w = g.unpack(want if out_parity == 0 else zero, want if out_parity == 1 else zero, prec)
            r = g.unpack(got if out_parity == 0 else zero, got if out_parity == 1 else zero, prec)
            err = np.linalg.norm(r - w) / np.linalg.norm(w)
            assert err <= TOL[prec], err
            assert abs(n_got.item() - n_want.item()) <= TOL[prec] * n_want.item()
        g.free()
