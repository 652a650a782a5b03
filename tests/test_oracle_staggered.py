"""Pins of the oracle's staggered operator (paper: Dirac_operator "staggered"
with a mass) against facts fixed by the mathematics:

* a dense matrix of D_hop assembled here from the definition with its own
  index code (shift matrices, phases eta_mu, links), on lattices with
  distinct extents and both boundary conditions;
* anti-Hermiticity of D_hop and anticommutation with eps(x) = (-1)^(sum x);
* free field: D_hop^2 on an (anti)periodic plane wave is -sum_mu sin^2 p_mu;
* gauge covariance under Haar Omega(x);
* the CG solve of D x = b against dense LU.
"""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
from paper_2409_03030_gb300 import synth


def coords(dims):
    nx, ny, nz, nt = dims
    return np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


def dense_hop(dims, U, tanti):
    """D_hop as a (3V x 3V) matrix, rows/cols ordered like [t, z, y, x, colour]."""
    nx, ny, nz, nt = dims
    ext = {0: nx, 1: ny, 2: nz, 3: nt}
    V = nx * ny * nz * nt
    Um = synth.link_matrices(U)  # [mu, t, z, y, x, a, b]
    M = np.zeros((3 * V, 3 * V), dtype=complex)

    def idx(t, z, y, x):
        return ((t * nz + z) * ny + y) * nx + x

    for t in range(nt):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    c = [x, y, z, t]
                    s = idx(t, z, y, x)
                    for mu in range(4):
                        eta = (-1) ** (sum(c[:mu]) % 2)
                        f = list(c); f[mu] = (c[mu] + 1) % ext[mu]
                        b = list(c); b[mu] = (c[mu] - 1) % ext[mu]
                        sf = -1.0 if (mu == 3 and tanti and c[mu] == ext[mu] - 1) else 1.0
                        sb = -1.0 if (mu == 3 and tanti and c[mu] == 0) else 1.0
                        jf = idx(f[3], f[2], f[1], f[0])
                        jb = idx(b[3], b[2], b[1], b[0])
                        M[3 * s:3 * s + 3, 3 * jf:3 * jf + 3] += 0.5 * eta * sf * Um[mu, t, z, y, x]
                        M[3 * s:3 * s + 3, 3 * jb:3 * jb + 3] -= 0.5 * eta * sb * \
                            Um[mu, b[3], b[2], b[1], b[0]].conj().T
    return M


@pytest.mark.parametrize("dims,tanti", [((2, 2, 2, 4), True), ((4, 2, 2, 2), True), ((2, 4, 2, 2), False)])
def test_staggered_dense_brute_force(dims, tanti):
    U = synth.gauge(dims, "haar", seed=111)
    M = dense_hop(dims, U, tanti)
    psi = synth.gaussian_colour(dims, seed=112)
    got = oracle.stag_hop(dims, U, psi, t_antiperiodic=tanti).ravel()
    assert pins.rel(got, M @ psi.ravel()) < 1e-14
    got = oracle.stag_dirac(dims, U, psi, 0.07, t_antiperiodic=tanti).ravel()
    assert pins.rel(got, 0.07 * psi.ravel() + M @ psi.ravel()) < 1e-14
    got = oracle.stag_dirac(dims, U, psi, 0.07, dagger=True, t_antiperiodic=tanti).ravel()
    assert pins.rel(got, 0.07 * psi.ravel() + M.conj().T @ psi.ravel()) < 1e-14


def test_staggered_antihermitian_and_eps():
    dims = (4, 6, 2, 8)
    U = synth.gauge(dims, "haar", seed=113)
    phi, psi = synth.gaussian_colour(dims, seed=114), synth.gaussian_colour(dims, seed=115)
    lhs = np.vdot(phi, oracle.stag_hop(dims, U, psi))
    rhs = -np.vdot(oracle.stag_hop(dims, U, phi), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    t, z, y, x = coords(dims)
    eps = ((-1.0) ** ((x + y + z + t) % 2))[..., None]
    assert pins.rel(eps * oracle.stag_hop(dims, U, eps * psi), -oracle.stag_hop(dims, U, psi)) < 1e-14
    # even-odd structure: D_hop maps each parity to the other
    odd = oracle.parity_mask(dims)[..., None]
    out = oracle.stag_hop(dims, U, np.where(odd, psi, 0), out_parity=1)
    assert not np.any(out)


@pytest.mark.parametrize("tanti", [True, False])
def test_staggered_free_field(tanti):
    dims = (4, 6, 8, 10)
    U = synth.gauge(dims, "unit")
    nx, ny, nz, nt = dims
    t, z, y, x = coords(dims)
    rng = np.random.default_rng(116)
    for n in [(1, 2, 3, 4), (0, 5, 1, 9), (3, 0, 7, 2)]:
        p = np.array([2 * np.pi * n[0] / nx, 2 * np.pi * n[1] / ny, 2 * np.pi * n[2] / nz,
                      (2 * np.pi * n[3] + (np.pi if tanti else 0.0)) / nt])
        u = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None] * u
        h2 = oracle.stag_hop(dims, U, oracle.stag_hop(dims, U, psi, t_antiperiodic=tanti), t_antiperiodic=tanti)
        assert pins.rel(h2, -np.sum(np.sin(p) ** 2) * psi) < 1e-13


def test_staggered_gauge_covariance():
    dims = (4, 6, 2, 8)
    U = synth.gauge(dims, "haar", seed=117)
    psi = synth.gaussian_colour(dims, seed=118)
    Om = synth.gauge_transform(dims, seed=119)
    Up, _ = pins._transform(dims, U, np.broadcast_to(psi[None], (4,) + psi.shape).copy(), Om)
    Omm = np.swapaxes(Om, -1, -2)
    rot = lambda f: np.einsum("tzyxab,tzyxb->tzyxa", Omm, f)  # noqa: E731
    lhs = oracle.stag_dirac(dims, Up, rot(psi), 0.05)
    rhs = rot(oracle.stag_dirac(dims, U, psi, 0.05))
    assert pins.rel(lhs, rhs) < 1e-13


def test_staggered_solve_against_dense():
    dims = (2, 2, 2, 4)
    U = synth.gauge(dims, "haar", seed=120)
    b = synth.gaussian_colour(dims, seed=121)
    m = 0.1
    D = m * np.eye(3 * 32) + dense_hop(dims, U, True)
    x, iters, sys_rel, full_rel, ok = oracle.stag_solve(dims, U, b, m, tol=1e-13)
    assert ok and sys_rel <= 1e-13
    assert pins.rel(x.ravel(), np.linalg.solve(D, b.ravel())) <= 1e-10
