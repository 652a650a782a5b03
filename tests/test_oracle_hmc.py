"""Pins of the oracle's HMC pieces (paper: section "Hybrid Monte Carlo":
plaquette gauge action with beta, momenta in su(3), leapfrog MD step,
Metropolis on H = K + S_g + S_f) against facts fixed by the mathematics:
cold-start action, the gauge force as the derivative of the action (central
differences), gauge invariance and covariance, the kinetic energy of the
momentum refresh, the exponential's group properties, and the leapfrog's
reversibility and second-order energy error."""
import numpy as np
import pytest

import oracle
import test_oracle_force as fpins
import test_oracle_pins as pins
from paper_2409_03030_gb300 import synth

BETA = 5.5


def test_cold_start_action():
    dims = (4, 2, 6, 4)
    U = synth.gauge(dims, "unit")
    V = int(np.prod(dims))
    assert oracle.plaquette_sum(dims, U) == 18.0 * V
    assert oracle.gauge_action(dims, U, BETA) == -BETA / 3 * 18 * V


def test_gauge_force_is_the_derivative():
    dims = (2, 4, 2, 2)
    U = synth.gauge(dims, "haar", seed=151)
    G = oracle.gauge_force(dims, U, BETA)
    rng = np.random.default_rng(152)
    eps = 1e-5
    for mu, site in [(0, (1, 0, 2, 1)), (1, (0, 1, 3, 0)), (2, (1, 1, 0, 1)), (3, (0, 0, 1, 1))]:
        w = fpins.su3_generator(rng)
        Um = fpins.link_matrix(U, mu, *site)
        Sp = oracle.gauge_action(dims, fpins.with_link(U, mu, site, fpins.expm_ah(eps * w) @ Um), BETA)
        Sm = oracle.gauge_action(dims, fpins.with_link(U, mu, site, fpins.expm_ah(-eps * w) @ Um), BETA)
        fd = (Sp - Sm) / (2 * eps)
        want = np.trace(fpins.link_matrix(G, mu, *site) @ w).real
        assert abs(fd - want) <= 1e-7 * max(1.0, abs(want)), (mu, site, fd, want)


def test_gauge_invariance_and_covariance():
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=153)
    Om = synth.gauge_transform(dims, seed=154)
    psi = synth.gaussian_spinor(dims, seed=155)
    Up, _ = pins._transform(dims, U, psi, Om)
    assert abs(oracle.plaquette_sum(dims, Up) - oracle.plaquette_sum(dims, U)) < 1e-11
    G, Gp = oracle.gauge_force(dims, U, BETA), oracle.gauge_force(dims, Up, BETA)
    Omm = np.swapaxes(Om, -1, -2)
    want = np.einsum("tzyxab,mtzyxbc,tzyxdc->mtzyxad", Omm, np.swapaxes(G, -1, -2), Omm.conj())
    assert pins.rel(np.swapaxes(Gp, -1, -2), want) < 1e-12


def test_momenta_and_exponential():
    dims = (2, 2, 2, 4)
    rng = np.random.default_rng(156)
    normals = rng.normal(size=(4,) + tuple(reversed(dims)) + (8,))
    P = oracle.momenta(normals)
    assert abs(oracle.kinetic(P) - 0.5 * np.sum(normals ** 2)) < 1e-12 * np.sum(normals ** 2)
    M = np.swapaxes(P, -1, -2)
    assert np.allclose(M, -np.conj(np.swapaxes(M, -1, -2))) and np.allclose(np.einsum("...ii", M), 0)
    U = synth.gauge(dims, "haar", seed=157)
    U1 = oracle.exp_update(U, P, 0.3)
    Um = np.swapaxes(U1, -1, -2)
    assert np.allclose(Um @ np.conj(np.swapaxes(Um, -1, -2)), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(Um), 1, atol=1e-14)
    assert pins.rel(oracle.exp_update(U1, P, -0.3), U) < 1e-14
    # against the power series on one link
    m = 0.3 * M[1, 0, 1, 0, 1]
    series, term = np.eye(3, dtype=complex), np.eye(3, dtype=complex)
    for k in range(1, 30):
        term = term @ m / k
        series = series + term
    assert np.abs(np.swapaxes(oracle.exp_update(synth.gauge(dims, "unit"), P, 0.3), -1, -2)[1, 0, 1, 0, 1]
                  - series).max() < 1e-14
    # the traceless anti-Hermitian projection keeps only su(3): Re Tr[TA(G) w] = Re Tr[G w]
    G = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    w = fpins.su3_generator(rng)
    TA = np.swapaxes(oracle.traceless_antihermitian(np.swapaxes(G, -1, -2)), -1, -2)
    assert abs(np.trace(TA @ w).real - np.trace(G @ w).real) < 1e-13


@pytest.mark.parametrize("with_fermions", [False, True])
def test_leapfrog_reversible_and_second_order(with_fermions):
    dims = (2, 2, 2, 4)
    U = synth.gauge(dims, "expi", eps=0.5, seed=158)
    rng = np.random.default_rng(159)
    normals = rng.normal(size=(4,) + tuple(reversed(dims)) + (8,))
    xi = synth.gaussian_spinor(dims, seed=160) if with_fermions else None
    kappa, tol = 0.12, 1e-14
    U1, P1, H0, H1 = oracle.hmc_trajectory(dims, U, normals, xi, BETA, kappa, n_md=8, tol=tol)
    # reversibility: from (U1, -P1) back to (U, -P0)
    eta = None if xi is None else oracle.dirac(dims, U, xi, kappa, dagger=True)
    U2, P2 = U1, -P1
    dt = 1.0 / 8
    for _ in range(8):
        U2 = oracle.exp_update(U2, P2, dt / 2)
        P2 = P2 + dt * 0.5 * oracle.traceless_antihermitian(oracle.hmc_forces(dims, U2, eta, BETA, kappa, tol))
        U2 = oracle.exp_update(U2, P2, dt / 2)
    assert pins.rel(U2, U) < 1e-11
    assert pins.rel(-P2, oracle.momenta(normals)) < 1e-10
    # energy error of a second-order integrator: halving dt divides dH by ~4
    dH = []
    for n in (8, 16):
        _, _, Ha, Hb = oracle.hmc_trajectory(dims, U, normals, xi, BETA, kappa, n_md=n, tol=tol)
        dH.append(abs(Hb - Ha))
    assert 2.8 < dH[0] / dH[1] < 5.5, dH
