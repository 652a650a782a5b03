"""Seeded input generators: determinism, SU(3) properties, distributions."""
import numpy as np
import pytest

from paper_2409_03030_gb300 import synth


def unitarity_err(M):
    I = np.eye(3)
    return np.abs(np.einsum("...ka,...kb->...ab", M.conj(), M) - I).max()


def test_haar_links_are_su3():
    U = synth.link_matrices(synth.gauge((4, 4, 4, 4), "haar", seed=1))
    assert unitarity_err(U) < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # Haar: E[U_ab] = 0 and E|U_ab|^2 = 1/3
    assert np.abs(U.mean(axis=(0, 1, 2, 3, 4))).max() < 0.05
    assert np.abs((np.abs(U) ** 2).mean() - 1 / 3) < 0.01


@pytest.mark.parametrize("eps", [0.3, 0.4])
def test_expi_links(eps):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    U = synth.link_matrices(synth.gauge((4, 2, 2, 4), "expi", eps=eps, seed=2))
    assert unitarity_err(U) < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # U = exp(i eps H): recover H = -i log(U)/eps, which must be Hermitian and
    # traceless, and exp(i eps H) must give U back.
    flat = U.reshape(-1, 3, 3)
    for M in flat[:50]:
        H = -1j * scipy_linalg.logm(M) / eps
        assert np.abs(H - H.conj().T).max() < 1e-10
        assert abs(np.trace(H)) < 1e-10
        assert np.abs(scipy_linalg.expm(1j * eps * H) - M).max() < 1e-12


def test_unit_links():
    U = synth.link_matrices(synth.gauge((2, 2, 2, 2), "unit"))
    assert np.array_equal(U, np.broadcast_to(np.eye(3), U.shape))


def test_deterministic_and_seeded():
    a = synth.gaussian_spinor((4, 4, 4, 4), seed=9)
    b = synth.gaussian_spinor((4, 4, 4, 4), seed=9)
    c = synth.gaussian_spinor((4, 4, 4, 4), seed=10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    g1 = synth.gauge((4, 4, 2, 2), "expi", 0.3, seed=3)
    g2 = synth.gauge((4, 4, 2, 2), "expi", 0.3, seed=3)
    assert np.array_equal(g1, g2)


def test_gaussian_variance():
    z = synth.gaussian_spinor((8, 8, 8, 8), seed=4).ravel()
    assert abs(z.real.var() - 0.5) < 0.01 and abs(z.imag.var() - 0.5) < 0.01
    assert abs(z.real.mean()) < 0.01 and abs(np.mean(z.real * z.imag)) < 0.01


def test_uniforms_in_range():
    u = synth.uniforms(200000, seed=5)
    assert u.min() > 0 and u.max() <= 1 and abs(u.mean() - 0.5) < 0.005


def test_point_source():
    p = synth.point_source((4, 4, 4, 6), spin=2, colour=1)
    assert p.sum() == 1 and p[2, 0, 0, 0, 0, 1] == 1
