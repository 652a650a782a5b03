"""The closed-form free-field condition number (tests/conditioning.py) against
the oracle's Mhat^dag Mhat assembled as a dense matrix on small lattices:
every eigenvalue of the dense matrix is one of the closed form's squared
singular values, and the extremes agree."""
import numpy as np
import pytest

import oracle
from conditioning import free_cond_eo, free_singular_values
from paper_2409_03030_gb300 import synth


def dense_normal_eo(dims, kappa, t_antiperiodic):
    U = synth.gauge(dims, "unit")
    odd = oracle.parity_mask(dims)
    shape = synth.spinor_shape(dims)
    cols = []
    idx = [i for i in np.ndindex(shape) if not odd[i[1:5]]]
    for i in idx:
        v = np.zeros(shape, complex)
        v[i] = 1.0
        w = oracle.normal_apply(dims, U, v, kappa, eo=True, t_antiperiodic=t_antiperiodic)
        cols.append(np.array([w[j] for j in idx]))
    return np.array(cols).T


@pytest.mark.parametrize("dims,anti", [((2, 2, 2, 4), True), ((4, 2, 2, 2), False),
                                       ((2, 4, 2, 4), True)])
def test_free_cond_matches_dense(dims, anti):
    kappa = 0.12
    A = dense_normal_eo(dims, kappa, anti)
    assert np.allclose(A, A.conj().T, atol=1e-14)
    ev = np.linalg.eigvalsh(A)
    sv2 = np.sort(free_singular_values(dims, kappa, anti) ** 2)
    # every dense eigenvalue appears among the closed form's values
    assert np.all(np.min(np.abs(ev[:, None] - sv2[None, :]), axis=1) <= 1e-12 * sv2.max())
    assert abs(ev.max() - sv2.max()) <= 1e-12 * sv2.max()
    assert abs(ev.min() - sv2.min()) <= 1e-12 * sv2.max()
    assert abs(ev.max() / ev.min() - free_cond_eo(dims, kappa, anti)) <= 1e-9 * ev.max() / ev.min()
