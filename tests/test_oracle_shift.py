"""Pins of the oracle's shifted CG, (A + sigma) x = rhs, the definition of what
a multi-shift solve (RHMC; paper's feature list) returns for each shift:
dense LU of A + sigma assembled column by column from the oracle's normal
operator on small lattices, and sigma = 0 reducing to the plain CG."""
import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth


def dense_normal(dims, U, kappa, eo):
    shape = synth.spinor_shape(dims)
    n = int(np.prod(shape))
    mask = np.ones(shape, bool)
    if eo:
        mask = ~np.broadcast_to(oracle.parity_mask(dims)[None, ..., None], shape)
    idx = np.flatnonzero(mask.ravel())
    M = np.empty((len(idx), len(idx)), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for j, k in enumerate(idx):
        e[k] = 1.0
        M[:, j] = oracle.normal_apply(dims, U, e.reshape(shape), kappa, eo=eo).ravel()[idx]
        e[k] = 0.0
    return M, idx


@pytest.mark.parametrize("eo", [True, False])
def test_shifted_cg_against_dense(eo):
    dims = (2, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=91)
    b = synth.gaussian_spinor(dims, seed=92)
    rhs = oracle.zero_parity(dims, b, 1) if eo else b
    M, idx = dense_normal(dims, U, 0.12, eo)
    for sigma in (0.0, 0.003, 0.1, 1.7):
        x, iters, true_rel, ok = oracle.cg_shift(dims, U, rhs, 0.12, sigma, eo=eo, tol=1e-13,
                                                 maxiter=5000)
        assert ok and true_rel <= 1e-13
        want = np.linalg.solve(M + sigma * np.eye(len(idx)), rhs.ravel()[idx])
        got = x.ravel()
        assert np.linalg.norm(got[idx] - want) <= 1e-11 * np.linalg.norm(want)
        if eo:  # odd sites stay zero
            assert not np.any(np.delete(got, idx))


def test_zero_shift_is_plain_cg():
    dims = (4, 4, 2, 4)
    U = synth.gauge(dims, "expi", eps=0.3, seed=93)
    rhs = oracle.zero_parity(dims, synth.gaussian_spinor(dims, seed=94), 1)
    x0, *_ = oracle.cg(dims, U, rhs, 0.12, eo=True, tol=1e-12)
    x1, *_ = oracle.cg_shift(dims, U, rhs, 0.12, 0.0, eo=True, tol=1e-12)
    assert np.array_equal(x0, x1)
