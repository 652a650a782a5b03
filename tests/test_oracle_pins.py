"""Pins of the FP64 CPU oracle against facts fixed by the mathematics.

None of these compare the oracle with itself: each check is a closed form
(free-field plane waves and their inverse), a symmetry (gauge covariance,
adjointness, gamma5-hermiticity), or a brute-force construction that shares no
index code with the oracle (dense matrices assembled here from shift and link
block matrices, the Schur complement by dense block algebra, and dense LU).
Lattices have distinct extents so a swapped axis cannot pass.
"""
import numpy as np
import pytest

import oracle
from paper_2409_03030_gb300 import synth

# DeGrand-Rossi chiral basis, mu = x, y, z, t.  This is the library's spin
# convention; the oracle must use exactly these matrices.
I4 = np.eye(4, dtype=complex)
G = np.array([
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=complex)
G5 = G[0] @ G[1] @ G[2] @ G[3]


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def test_gamma_basis():
    assert np.array_equal(oracle.gamma(), G)
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2 * (m == n) * I4)
    assert np.allclose(G5, np.diag([1, 1, -1, -1]))
    for m in range(4):  # (1 +/- gamma_mu)/2 are rank-2 projectors
        assert np.linalg.matrix_rank(I4 - G[m]) == 2


def coords(dims):
    nx, ny, nz, nt = dims
    return np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx),
                       indexing="ij")  # t, z, y, x arrays of shape (nt,nz,ny,nx)


def plane_wave(dims, n, u, tanti):
    """psi(x) = exp(i p.x) u with p_mu = 2 pi n_mu / L_mu, p_t shifted by pi/NT
    when time is antiperiodic."""
    nx, ny, nz, nt = dims
    t, z, y, x = coords(dims)
    p = np.array([2 * np.pi * n[0] / nx, 2 * np.pi * n[1] / ny, 2 * np.pi * n[2] / nz,
                  (2 * np.pi * n[3] + (np.pi if tanti else 0.0)) / nt])
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return np.einsum("tzyx,ac->atzyxc", ph, u), p


def symbol(p, kappa, dagger=False):
    s = -1.0 if dagger else 1.0
    return (1 - 2 * kappa * np.cos(p).sum()) * I4 + s * 2j * kappa * np.einsum(
        "m,mab->ab", np.sin(p), G)


@pytest.mark.parametrize("tanti", [True, False])
@pytest.mark.parametrize("dagger", [False, True])
def test_free_field_closed_form(tanti, dagger):
    dims = (4, 6, 8, 10)
    U = synth.gauge(dims, "unit")
    rng = np.random.default_rng(5)
    for n in [(1, 2, 3, 4), (3, 1, 5, 7), (0, 0, 0, 0), (2, 5, 1, 9)]:
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi, p = plane_wave(dims, n, u, tanti)
        out = oracle.dirac(dims, U, psi, 0.13, dagger=dagger, t_antiperiodic=tanti)
        want = np.einsum("ab,btzyxc->atzyxc", symbol(p, 0.13, dagger), psi)
        assert rel(out, want) < 1e-13


def test_constant_field_periodic():
    dims = (4, 4, 6, 4)
    U = synth.gauge(dims, "unit")
    u = np.arange(12).reshape(4, 3) + 1j
    psi = np.broadcast_to(u[:, None, None, None, None, :], synth.spinor_shape(dims)).copy()
    out = oracle.dirac(dims, U, psi, 0.11, t_antiperiodic=False)
    assert rel(out, (1 - 8 * 0.11) * psi) < 1e-14


def test_kappa_zero_is_identity():
    dims = (4, 2, 2, 6)
    U = synth.gauge(dims, "haar", seed=3)
    psi = synth.gaussian_spinor(dims, seed=4)
    assert np.array_equal(oracle.dirac(dims, U, psi, 0.0), psi)


def _transform(dims, U, psi, Om):
    """U'_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag, psi'(x) = Om(x) psi(x)."""
    Um = synth.link_matrices(U)               # [mu, t,z,y,x, a, b]
    Omm = np.swapaxes(Om, -1, -2)             # [t,z,y,x, a, b]
    axis = {0: 3, 1: 2, 2: 1, 3: 0}           # mu -> axis of [t,z,y,x]
    Up = np.empty_like(Um)
    for mu in range(4):
        Om_fwd = np.roll(Omm, -1, axis=axis[mu])
        Up[mu] = Omm @ Um[mu] @ np.conj(np.swapaxes(Om_fwd, -1, -2))
    Up = np.ascontiguousarray(np.swapaxes(Up, -1, -2))
    psip = np.ascontiguousarray(np.einsum("tzyxab,stzyxb->stzyxa", Omm, psi))
    return Up, psip


@pytest.mark.parametrize("tanti", [True, False])
def test_gauge_covariance(tanti):
    dims = (4, 6, 2, 8)
    U = synth.gauge(dims, "haar", seed=11)
    psi = synth.gaussian_spinor(dims, seed=12)
    Om = synth.gauge_transform(dims, seed=13)
    Up, psip = _transform(dims, U, psi, Om)
    for dag in (False, True):
        lhs = oracle.dirac(dims, Up, psip, 0.12, dagger=dag, t_antiperiodic=tanti)
        _, rhs = _transform(dims, U, oracle.dirac(dims, U, psi, 0.12, dagger=dag,
                                                  t_antiperiodic=tanti), Om)
        assert rel(lhs, rhs) < 1e-13


def test_adjoint_and_gamma5_hermiticity():
    dims = (6, 4, 4, 8)
    U = synth.gauge(dims, "haar", seed=21)
    phi = synth.gaussian_spinor(dims, seed=22)
    psi = synth.gaussian_spinor(dims, seed=23)
    k = 0.1
    lhs = np.vdot(phi, oracle.dirac(dims, U, psi, k))
    rhs = np.vdot(oracle.dirac(dims, U, phi, k, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g5 = np.array([1, 1, -1, -1])[:, None, None, None, None, None]
    assert rel(g5 * oracle.dirac(dims, U, g5 * psi, k), oracle.dirac(dims, U, psi, k, True)) < 1e-14
    # Schur complement: <phi_e, Mhat psi_e> = <Mhat^dag phi_e, psi_e>
    pe = oracle.zero_parity(dims, psi, 1)
    fe = oracle.zero_parity(dims, phi, 1)
    l2 = np.vdot(fe, oracle.schur(dims, U, pe, k))
    r2 = np.vdot(oracle.schur(dims, U, fe, k, dagger=True), pe)
    assert abs(l2 - r2) < 1e-12 * abs(l2)
    # <v, Mhat^dag Mhat v> = ||Mhat v||^2, real and positive
    q = np.vdot(pe, oracle.normal_apply(dims, U, pe, k, eo=True))
    assert abs(q.imag) < 1e-12 * q.real and q.real > 0
    assert abs(q.real - np.linalg.norm(oracle.schur(dims, U, pe, k)) ** 2) < 1e-12 * q.real


def dense_dirac(dims, U, kappa, tanti):
    """D as a dense matrix in canonical index order ic + 3*(site + V*alpha),
    built as 1 - kappa sum_mu [(1-g_mu) x F_mu + (1+g_mu) x F_mu^dag] where F_mu
    is the forward hop U_mu(x) psi(x+mu) (times the boundary sign) on colour x
    site space, and the backward hop is its adjoint."""
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    Um = synth.link_matrices(U).reshape(4, V, 3, 3)
    ext = [nx, ny, nz, nt]
    D = np.eye(12 * V, dtype=complex)
    for mu in range(4):
        F = np.zeros((3 * V, 3 * V), dtype=complex)
        for s in range(V):
            c = [s % nx, (s // nx) % ny, (s // (nx * ny)) % nz, s // (nx * ny * nz)]
            c2 = list(c)
            c2[mu] = (c[mu] + 1) % ext[mu]
            sign = -1.0 if (tanti and mu == 3 and c[3] == nt - 1) else 1.0
            s2 = c2[0] + nx * (c2[1] + ny * (c2[2] + nz * c2[3]))
            F[3 * s:3 * s + 3, 3 * s2:3 * s2 + 3] += sign * Um[mu, s]
        D -= kappa * (np.kron(I4 - G[mu], F) + np.kron(I4 + G[mu], F.conj().T))
    return D


def parity_of_index(dims):
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    par = np.zeros(12 * V, dtype=int)
    for a in range(4):
        for s in range(V):
            c = [s % nx, (s // nx) % ny, (s // (nx * ny)) % nz, s // (nx * ny * nz)]
            par[3 * (s + V * a):3 * (s + V * a) + 3] = sum(c) % 2
    return par


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (4, 2, 2, 2)])
@pytest.mark.parametrize("tanti", [True, False])
def test_dense_brute_force(dims, tanti):
    U = synth.gauge(dims, "haar", seed=31)
    k = 0.1
    D = dense_dirac(dims, U, k, tanti)
    n = D.shape[0]
    shape = synth.spinor_shape(dims)
    cols = np.empty((n, n), dtype=complex)
    cols_dag = np.empty((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols[:, j] = oracle.dirac(dims, U, e.reshape(shape), k, t_antiperiodic=tanti).ravel()
        cols_dag[:, j] = oracle.dirac(dims, U, e.reshape(shape), k, dagger=True,
                                      t_antiperiodic=tanti).ravel()
    assert np.abs(cols - D).max() < 1e-14
    assert np.abs(cols_dag - D.conj().T).max() < 1e-14

    # Schur complement D_ee - D_eo D_oo^-1 D_oe against the oracle's Mhat.
    par = parity_of_index(dims)
    e_idx, o_idx = np.where(par == 0)[0], np.where(par == 1)[0]
    S = D[np.ix_(e_idx, e_idx)] - D[np.ix_(e_idx, o_idx)] @ np.linalg.solve(
        D[np.ix_(o_idx, o_idx)], D[np.ix_(o_idx, e_idx)])
    M = np.empty((len(e_idx), len(e_idx)), dtype=complex)
    Md = np.empty_like(M)
    for jj, j in enumerate(e_idx):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        full = oracle.schur(dims, U, e.reshape(shape), k, t_antiperiodic=tanti).ravel()
        assert np.abs(full[o_idx]).max() == 0.0
        M[:, jj] = full[e_idx]
        Md[:, jj] = oracle.schur(dims, U, e.reshape(shape), k, dagger=True,
                                 t_antiperiodic=tanti).ravel()[e_idx]
    assert np.abs(M - S).max() < 1e-13
    assert np.abs(Md - S.conj().T).max() < 1e-13

    # Solves against dense LU: error bounded by cond(A) * tol of the CG system.
    b = synth.gaussian_spinor(dims, seed=32)
    x_lu = np.linalg.solve(D, b.ravel())
    tol = 1e-12
    for eo in (False, True):
        x, it, sys_rel, full_rel, ok = oracle.solve(dims, U, b, k, eo=eo, tol=tol,
                                                    t_antiperiodic=tanti)
        assert ok and sys_rel <= tol * (1 + 1e-6)
        A = (S.conj().T @ S) if eo else (D.conj().T @ D)
        bound = np.linalg.cond(A) * tol * 4
        assert rel(x.ravel(), x_lu) < bound, (eo, rel(x.ravel(), x_lu), bound)
        assert full_rel < bound


def test_cg_free_field_inverse():
    dims = (4, 6, 4, 8)
    U = synth.gauge(dims, "unit")
    k = 0.12
    rng = np.random.default_rng(41)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    b, p = plane_wave(dims, (1, 2, 3, 1), u, True)
    want = np.einsum("ab,btzyxc->atzyxc", np.linalg.inv(symbol(p, k)), b)
    for eo in (False, True):
        x, it, sys_rel, full_rel, ok = oracle.solve(dims, U, b, k, eo=eo, tol=1e-12)
        assert ok and rel(x, want) < 1e-10


@pytest.mark.parametrize("eo", [False, True])
def test_cg_config0(eo):
    """4^4, Haar links, kappa = 0.10, antiperiodic time, Gaussian source, tol 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=1)
    b = synth.gaussian_spinor(dims, seed=1)
    x, it, sys_rel, full_rel, ok = oracle.solve(dims, U, b, 0.10, eo=eo, tol=1e-12)
    assert ok and sys_rel <= 1e-12 * (1 + 1e-6) and full_rel < 1e-10
    assert rel(oracle.dirac(dims, U, x, 0.10), b) == pytest.approx(full_rel, rel=1e-6)


def test_cg_maxiter_reports_nonconvergence():
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, "haar", seed=1)
    b = synth.gaussian_spinor(dims, seed=2)
    rhs = oracle.zero_parity(dims, b, 1)
    x, it, tr, ok = oracle.cg(dims, U, rhs, 0.12, eo=True, tol=1e-14, maxiter=3)
    assert not ok and it == 3 and tr > 1e-14


def test_hop_sites_matches_full_hop():
    dims = (4, 6, 4, 6)
    U = synth.gauge(dims, "expi", eps=0.3, seed=51)
    psi = synth.gaussian_spinor(dims, seed=52)
    full = oracle.hop(dims, U, psi, dagger=True)
    sites = np.array([0, 5, 17, 100, 575])
    part = oracle.hop_sites(dims, U, psi, sites, dagger=True)
    flat = full.reshape(4, -1, 3)
    for i, s in enumerate(sites):
        assert np.array_equal(part[i], flat[:, s, :])


def test_eo_hop_parity_restriction():
    dims = (4, 4, 6, 4)
    U = synth.gauge(dims, "expi", eps=0.3, seed=61)
    psi = synth.gaussian_spinor(dims, seed=62)
    full = oracle.hop(dims, U, psi)
    odd = oracle.parity_mask(dims)[None, :, :, :, :, None]
    # H_eo reads only odd inputs: the even-output hop of the odd part equals
    # the even part of the full hop.
    h_eo = oracle.hop(dims, U, oracle.zero_parity(dims, psi, 0), out_parity=0)
    assert np.array_equal(h_eo, np.where(odd, 0, full))
