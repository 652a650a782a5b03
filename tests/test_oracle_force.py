"""Pins of the oracle's fermion action and force (paper: evaluate_FermiAction,
calc_UdSfdU) against facts fixed by the mathematics:

* the force is the derivative of the action: for U_mu(x) -> exp(eps w) U_mu(x),
  w in su(3), dS/deps = Re Tr[(U dS/dU) w], checked by central differences of
  S computed by a dense solve (no CG), on links inside the lattice and across
  the antiperiodic boundary;
* heatbath identity: eta = D^dag xi gives S = |xi|^2;
* gauge covariance: U dS/dU at x transforms as Omega(x) (.) Omega(x)^dag.
"""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
from paper_2409_03030_gb300 import synth

KAPPA = 0.12


def dense_action(dims, U, eta, kappa, tanti=True):
    """S = eta^dag (D^dag D)^-1 eta = |D^-dag eta|^2 by dense LU, with D assembled
    column by column (D e_k).  Returns (S, D)."""
    shape = synth.spinor_shape(dims)
    n = int(np.prod(shape))
    D = np.empty((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for k in range(n):
        e[k] = 1.0
        D[:, k] = oracle.dirac(dims, U, e.reshape(shape), kappa, t_antiperiodic=tanti).ravel()
        e[k] = 0.0
    z = np.linalg.solve(D.conj().T, eta.ravel())
    return float(np.vdot(z, z).real), D


def su3_generator(rng):
    a = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    w = (a - a.conj().T) / 2
    return w - np.trace(w) / 3 * np.eye(3)


def expm_ah(w):
    """exp(w) for anti-Hermitian w via the Hermitian eigendecomposition of i w."""
    lam, v = np.linalg.eigh(1j * w)
    return (v * np.exp(-1j * lam)) @ v.conj().T


def link_matrix(U, mu, t, z, y, x):
    return U[mu, t, z, y, x].T  # stored [.., b, a]


def with_link(U, mu, site, Mnew):
    Up = U.copy()
    Up[(mu,) + site] = Mnew.T
    return Up


@pytest.mark.parametrize("tanti", [True, False])
def test_force_is_the_derivative_of_the_action(tanti):
    dims = (2, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=41)
    eta = synth.gaussian_spinor(dims, seed=42)
    S0, D = dense_action(dims, U, eta, KAPPA, tanti)
    X = np.linalg.solve(D.conj().T @ D, eta.ravel()).reshape(eta.shape)
    Y = (D @ X.ravel()).reshape(eta.shape)
    G = oracle.fermi_force_xy(dims, U, X, Y, KAPPA, t_antiperiodic=tanti)
    rng = np.random.default_rng(43)
    eps = 1e-5
    # (mu, (t, z, y, x)): one link per direction, two of them across the time boundary
    for mu, site in [(3, (3, 1, 0, 1)), (3, (3, 0, 1, 0)), (0, (1, 0, 1, 1)), (1, (2, 1, 1, 0)),
                     (2, (0, 1, 0, 1)), (3, (1, 0, 0, 0))]:
        w = su3_generator(rng)
        Um = link_matrix(U, mu, *site)
        Sp, _ = dense_action(dims, with_link(U, mu, site, expm_ah(eps * w) @ Um), eta, KAPPA, tanti)
        Sm, _ = dense_action(dims, with_link(U, mu, site, expm_ah(-eps * w) @ Um), eta, KAPPA, tanti)
        fd = (Sp - Sm) / (2 * eps)
        want = np.trace(link_matrix(G, mu, *site) @ w).real
        assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (mu, site, fd, want)


def test_cg_force_matches_dense_force():
    dims = (2, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=44)
    eta = synth.gaussian_spinor(dims, seed=45)
    S_dense, D = dense_action(dims, U, eta, KAPPA)
    X = np.linalg.solve(D.conj().T @ D, eta.ravel()).reshape(eta.shape)
    G_dense = oracle.fermi_force_xy(dims, U, X, oracle.dirac(dims, U, X, KAPPA), KAPPA)
    S, G = oracle.fermi_force(dims, U, eta, KAPPA, tol=1e-13)
    assert abs(S - S_dense) <= 1e-11 * S_dense
    assert pins.rel(G, G_dense) <= 1e-10


def test_heatbath_identity():
    """eta = D^dag xi (paper: sample_pseudofermions) gives S = |xi|^2 (Sfold = dot(xi, xi))."""
    dims = (4, 4, 2, 6)
    U = synth.gauge(dims, "expi", eps=0.3, seed=46)
    xi = synth.gaussian_spinor(dims, seed=47)
    eta = oracle.dirac(dims, U, xi, KAPPA, dagger=True)
    S, _ = oracle.fermi_action(dims, U, eta, KAPPA, tol=1e-13)
    assert abs(S - np.vdot(xi, xi).real) <= 1e-10 * S


def test_force_gauge_covariance():
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=48)
    eta = synth.gaussian_spinor(dims, seed=49)
    Om = synth.gauge_transform(dims, seed=50)
    Up, etap = pins._transform(dims, U, eta, Om)
    S, G = oracle.fermi_force(dims, U, eta, KAPPA, tol=1e-13)
    Sp, Gp = oracle.fermi_force(dims, Up, etap, KAPPA, tol=1e-13)
    assert abs(S - Sp) <= 1e-10 * S
    Omm = np.swapaxes(Om, -1, -2)  # [t,z,y,x, a, b]
    Gm = np.swapaxes(G, -1, -2)    # [mu, t,z,y,x, a, b]
    want = np.einsum("tzyxab,mtzyxbc,tzyxdc->mtzyxad", Omm, Gm, Omm.conj())
    assert pins.rel(np.swapaxes(Gp, -1, -2), want) <= 1e-10
