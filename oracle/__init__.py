"""jqcd oracle: plain FP64 CPU Wilson-Dirac operator, Schur complement and CG.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_2409_03030_gb300``) and never
imports it.  The arithmetic lives in ``jqcd_oracle.c`` (compiled with gcc);
this module only marshals numpy arrays.

All arrays are complex128 in the canonical host layouts of the generators in
``paper_2409_03030_gb300.synth``: spinors ``[alpha, t, z, y, x, colour]`` and
links ``[mu, t, z, y, x, b, a]`` (element (a, b) of U_mu).  ``dims`` is
``(NX, NY, NZ, NT)``.  Even-odd routines take whole-lattice arrays whose
other-parity sites are ignored on input and zero on output.

Parity pins (tests marked ``not gpu``): free-field closed form, gauge
covariance, adjointness and gamma5-hermiticity, a dense matrix assembled
independently on 2^4 and 2^3x4 lattices (including the Schur complement), and
CG against dense LU and the free-field inverse.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jqcd_oracle.c")
_LIB = os.path.join(_HERE, "libjqcd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over sites in the hop if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    lib.jo_gamma.argtypes = [dp]
    lib.jo_hop.argtypes = [ip, c_int, dp, dp, dp, c_int, c_int]
    lib.jo_dirac.argtypes = [ip, c_int, c_double, dp, dp, dp, c_int]
    lib.jo_hop_sites.argtypes = [ip, c_int, dp, dp, c_int, i64p, ctypes.c_int64, dp]
    lib.jo_schur.argtypes = [ip, c_int, c_double, dp, dp, dp, c_int]
    lib.jo_normal_apply.argtypes = [ip, c_int, c_double, dp, c_int, dp, dp]
    lib.jo_cg.argtypes = [ip, c_int, c_double, dp, c_int, dp, dp, c_double, c_int,
                          ip, dp]
    lib.jo_solve.argtypes = [ip, c_int, c_double, dp, c_int, dp, dp, c_double, c_int,
                             ip, dp, dp]
    lib.jo_zero_parity.argtypes = [ip, dp, c_int]
    lib.jo_cg_shift.argtypes = [ip, c_int, c_double, dp, c_int, c_double, dp, dp, c_double, c_int,
                                ip, dp]
    lib.jo_cg_shift.restype = c_int
    lib.jo_stag_hop.argtypes = [ip, c_int, dp, dp, dp, c_int, c_int]
    lib.jo_stag_dirac.argtypes = [ip, c_int, c_double, dp, dp, dp, c_int]
    lib.jo_stag_solve.argtypes = [ip, c_int, c_double, dp, dp, dp, c_double, c_int, ip, dp, dp]
    for name in ("jo_stag_hop", "jo_stag_dirac", "jo_stag_solve"):
        getattr(lib, name).restype = c_int
    lib.jo_plaquette_sum.argtypes = [ip, dp]
    lib.jo_plaquette_sum.restype = c_double
    lib.jo_gauge_force.argtypes = [ip, c_double, dp, dp]
    lib.jo_gauge_force.restype = c_int
    lib.jo_set_threads.argtypes = [c_int]
    lib.jo_fermi_force.argtypes = [ip, c_int, c_double, dp, dp, dp, dp]
    lib.jo_fermi_force.restype = c_int
    lib.jo_fermi_force_links.argtypes = [ip, c_int, c_double, dp, dp, dp, i64p, ctypes.c_int64, dp]
    lib.jo_fermi_force_links.restype = c_int
    lib.jo_set_threads.restype = c_int
    for name in ("jo_hop", "jo_dirac", "jo_hop_sites", "jo_schur", "jo_normal_apply",
                 "jo_cg", "jo_solve", "jo_zero_parity"):
        getattr(lib, name).restype = c_int
    lib.jo_gamma.restype = None
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _dims(dims):
    d = tuple(int(v) for v in dims)
    if len(d) != 4 or min(d) < 1:
        raise ValueError(f"bad dims {dims}")
    return d, (ctypes.c_int * 4)(*d)


def _p(a):
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError("oracle arrays must be C-contiguous complex128")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"{what} failed with status {rc}")
    return rc


def _spinor(dims):
    nx, ny, nz, nt = dims
    return np.zeros((4, nt, nz, ny, nx, 3), dtype=np.complex128)


def gamma() -> np.ndarray:
    """The oracle's gamma matrices, shape (4, 4, 4), [mu, alpha, beta]."""
    out = np.zeros((4, 4, 4), dtype=np.complex128)
    _load().jo_gamma(_p(out))
    return out


def hop(dims, U, psi, dagger=False, out_parity=-1, t_antiperiodic=True):
    """H psi (or the adjoint hop), at sites of `out_parity` (-1: all)."""
    d, cd = _dims(dims)
    out = _spinor(d)
    _check(_load().jo_hop(cd, int(t_antiperiodic), _p(U), _p(psi), _p(out), int(dagger),
                          int(out_parity)), "jo_hop")
    return out


def dirac(dims, U, psi, kappa, dagger=False, t_antiperiodic=True):
    """D psi = psi - kappa H psi (paper: mul!(y, D, x)); dagger: D'."""
    d, cd = _dims(dims)
    out = _spinor(d)
    _check(_load().jo_dirac(cd, int(t_antiperiodic), float(kappa), _p(U), _p(psi), _p(out),
                            int(dagger)), "jo_dirac")
    return out


def hop_sites(dims, U, psi, sites, dagger=False, t_antiperiodic=True):
    """(H psi) at the given lexicographic site indices; shape (n, 4, 3)."""
    d, cd = _dims(dims)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.zeros((len(s), 4, 3), dtype=np.complex128)
    _check(_load().jo_hop_sites(cd, int(t_antiperiodic), _p(U), _p(psi), int(dagger),
                                s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(s),
                                _p(out)), "jo_hop_sites")
    return out


def schur(dims, U, psi_e, kappa, dagger=False, t_antiperiodic=True):
    """Mhat psi_e = psi_e - kappa^2 H_eo H_oe psi_e on even sites (dagger: Mhat^dag)."""
    d, cd = _dims(dims)
    out = _spinor(d)
    _check(_load().jo_schur(cd, int(t_antiperiodic), float(kappa), _p(U), _p(psi_e), _p(out),
                            int(dagger)), "jo_schur")
    return out


def normal_apply(dims, U, psi, kappa, eo=True, t_antiperiodic=True):
    """Mhat^dag Mhat psi (eo) or D^dag D psi (not eo); paper: DdagD_operator."""
    d, cd = _dims(dims)
    out = _spinor(d)
    _check(_load().jo_normal_apply(cd, int(t_antiperiodic), float(kappa), _p(U), int(bool(eo)),
                                   _p(psi), _p(out)), "jo_normal_apply")
    return out


def cg(dims, U, rhs, kappa, eo=True, tol=1e-10, maxiter=10000, x0=None, t_antiperiodic=True):
    """Textbook CG on the normal equations A x = rhs.  Returns (x, iters, true_rel, converged)."""
    d, cd = _dims(dims)
    x = _spinor(d) if x0 is None else np.array(x0, dtype=np.complex128, order="C")
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    rc = _check(_load().jo_cg(cd, int(t_antiperiodic), float(kappa), _p(U), int(bool(eo)),
                              _p(rhs), _p(x), float(tol), int(maxiter), ctypes.byref(it),
                              ctypes.byref(tr)), "jo_cg")
    return x, it.value, tr.value, rc == 0


def cg_shift(dims, U, rhs, kappa, shift, eo=True, tol=1e-10, maxiter=10000, t_antiperiodic=True):
    """Textbook CG on (A + shift) x = rhs, A = Mhat^dag Mhat (eo, even sites) or
    D^dag D: what a multi-shift solve returns for that shift.
    Returns (x, iters, true_rel, converged)."""
    d, cd = _dims(dims)
    x = _spinor(d)
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    rc = _check(_load().jo_cg_shift(cd, int(t_antiperiodic), float(kappa), _p(U), int(bool(eo)),
                                    float(shift), _p(rhs), _p(x), float(tol), int(maxiter),
                                    ctypes.byref(it), ctypes.byref(tr)), "jo_cg_shift")
    return x, it.value, tr.value, rc == 0


def solve(dims, U, b, kappa, eo=True, tol=1e-10, maxiter=10000, t_antiperiodic=True):
    """Solve D x = b (paper: solve_DinvX!).  Returns
    (x, iters, system_true_rel, full_rel, converged)."""
    d, cd = _dims(dims)
    x = _spinor(d)
    it = ctypes.c_int(0)
    sr = ctypes.c_double(0)
    fr = ctypes.c_double(0)
    rc = _check(_load().jo_solve(cd, int(t_antiperiodic), float(kappa), _p(U), int(bool(eo)),
                                 _p(b), _p(x), float(tol), int(maxiter), ctypes.byref(it),
                                 ctypes.byref(sr), ctypes.byref(fr)), "jo_solve")
    return x, it.value, sr.value, fr.value, rc == 0


def zero_parity(dims, psi, parity):
    """Copy of psi with the sites of `parity` set to zero."""
    d, cd = _dims(dims)
    out = np.array(psi, dtype=np.complex128, order="C")
    _check(_load().jo_zero_parity(cd, _p(out), int(parity)), "jo_zero_parity")
    return out


def fermi_force_xy(dims, U, X, Y, kappa, t_antiperiodic=True):
    """U_mu(x) dS/dU_mu(x) for all links from X = (D^dag D)^-1 eta and Y = D X
    (convention dS = Re Tr[(dS/dU) dU]); canonical link layout like U."""
    d, cd = _dims(dims)
    out = np.zeros_like(U)
    _check(_load().jo_fermi_force(cd, int(t_antiperiodic), float(kappa), _p(U), _p(X), _p(Y),
                                  _p(out)), "jo_fermi_force")
    return out


def fermi_force_links(dims, U, X, Y, kappa, links, t_antiperiodic=True):
    """U dS/dU of the given links (site + V*mu, lexicographic site); shape (n, 3, 3)
    as [k, b, a] like the link arrays."""
    d, cd = _dims(dims)
    ls = np.ascontiguousarray(np.asarray(links, dtype=np.int64))
    out = np.zeros((len(ls), 3, 3), dtype=np.complex128)
    _check(_load().jo_fermi_force_links(cd, int(t_antiperiodic), float(kappa), _p(U), _p(X), _p(Y),
                                        ls.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(ls),
                                        _p(out)), "jo_fermi_force_links")
    return out


def fermi_action(dims, U, eta, kappa, tol=1e-12, t_antiperiodic=True):
    """S = eta^dag (D^dag D)^-1 eta (paper: evaluate_FermiAction) by textbook CG
    on D^dag D.  Returns (S, X) with X = (D^dag D)^-1 eta."""
    X, iters, rel_res, ok = cg(dims, U, eta, kappa, eo=False, tol=tol, maxiter=100000,
                               t_antiperiodic=t_antiperiodic)
    if not ok:
        raise RuntimeError("oracle CG did not converge")
    return float(np.vdot(eta, X).real), X


def fermi_force(dims, U, eta, kappa, tol=1e-12, t_antiperiodic=True):
    """(S, U dS/dU) of S = eta^dag (D^dag D)^-1 eta (paper: calc_UdSfdU)."""
    S, X = fermi_action(dims, U, eta, kappa, tol, t_antiperiodic)
    Y = dirac(dims, U, X, kappa, t_antiperiodic=t_antiperiodic)
    return S, fermi_force_xy(dims, U, X, Y, kappa, t_antiperiodic)


# ---- staggered fermions: one colour vector per site, shape [t, z, y, x, colour] ----
def _colour(dims):
    nx, ny, nz, nt = dims
    return np.zeros((nt, nz, ny, nx, 3), dtype=np.complex128)


def stag_hop(dims, U, psi, dagger=False, out_parity=-1, t_antiperiodic=True):
    """D_hop psi = (1/2) sum_mu eta_mu [U psi(x+mu) - U^dag psi(x-mu)] (dagger: -D_hop psi)."""
    d, cd = _dims(dims)
    out = _colour(d)
    _check(_load().jo_stag_hop(cd, int(t_antiperiodic), _p(U), _p(psi), _p(out), int(dagger),
                               int(out_parity)), "jo_stag_hop")
    return out


def stag_dirac(dims, U, psi, mass, dagger=False, t_antiperiodic=True):
    """Staggered D psi = m psi + D_hop psi (dagger: m psi - D_hop psi)."""
    d, cd = _dims(dims)
    out = _colour(d)
    _check(_load().jo_stag_dirac(cd, int(t_antiperiodic), float(mass), _p(U), _p(psi), _p(out),
                                 int(dagger)), "jo_stag_dirac")
    return out


def stag_solve(dims, U, b, mass, tol=1e-12, maxiter=100000, t_antiperiodic=True):
    """Solve staggered D x = b by textbook CG on D^dag D.
    Returns (x, iters, system_true_rel, full_rel, converged)."""
    d, cd = _dims(dims)
    x = _colour(d)
    it, sr, fr = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_double(0)
    rc = _check(_load().jo_stag_solve(cd, int(t_antiperiodic), float(mass), _p(U), _p(b), _p(x), float(tol),
                                      int(maxiter), ctypes.byref(it), ctypes.byref(sr), ctypes.byref(fr)),
                "jo_stag_solve")
    return x, it.value, sr.value, fr.value, rc == 0


# ---- pure-gauge part of the HMC (plaquette action, its force) -------------------
def plaquette_sum(dims, U):
    """sum over x and mu < nu of Re Tr P_munu(x)."""
    d, cd = _dims(dims)
    return float(_load().jo_plaquette_sum(cd, _p(U)))


def gauge_action(dims, U, beta):
    """S_g = -(beta/3) sum Re Tr P (the paper's plaquette gauge action, Sg = -evaluate/NC)."""
    return -beta / 3.0 * plaquette_sum(dims, U)


def gauge_force(dims, U, beta):
    """U dS_g/dU for every link (convention dS = Re Tr[(dS/dU) dU])."""
    d, cd = _dims(dims)
    out = np.zeros_like(U)
    _check(_load().jo_gauge_force(cd, float(beta), _p(U), _p(out)), "jo_gauge_force")
    return out


# Gell-Mann generators T^a = lambda^a / 2 (Tr T^a T^b = delta_ab / 2)
def gell_mann():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l / 2


def _mats(F):
    """link-layout array [mu, t, z, y, x, b, a] -> matrices [..., a, b]."""
    return np.swapaxes(F, -1, -2)


def _links(M):
    return np.ascontiguousarray(np.swapaxes(M, -1, -2))


def momenta(normals):
    """P = i sum_a p^a T^a per link from normals of shape [mu, t, z, y, x, 8]
    (the momentum refresh of the MD step); link layout like U."""
    return _links(1j * np.einsum("...a,aij->...ij", normals, gell_mann()))


def kinetic(P):
    """K = sum over links of -Tr(P^2) = (1/2) sum (p^a)^2."""
    M = _mats(P)
    return float(-np.einsum("...ij,...ji->...", M, M).sum().real)


def traceless_antihermitian(G):
    """TA(G) = (G - G^dag)/2 - Tr(G - G^dag)/6, per link (link layout in and out)."""
    M = _mats(G)
    A = (M - np.conj(np.swapaxes(M, -1, -2))) / 2
    tr = np.einsum("...ii->...", A) / 3
    return _links(A - tr[..., None, None] * np.eye(3))


def exp_update(U, P, eps):
    """U <- exp(eps P) U per link (exp through the Hermitian eigendecomposition of -i P)."""
    H = -1j * _mats(P)
    lam, v = np.linalg.eigh(H)
    E = np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * lam), v.conj())
    return _links(E @ _mats(U))


def hmc_forces(dims, U, eta, beta, kappa, tol, t_antiperiodic=True):
    """U dS/dU of S_g + S_f (S_f = eta^dag (D^dag D)^-1 eta; no fermions when eta is None)."""
    G = gauge_force(dims, U, beta)
    if eta is not None:
        _, Gf = fermi_force(dims, U, eta, kappa, tol=tol, t_antiperiodic=t_antiperiodic)
        G = G + Gf
    return G


def hmc_trajectory(dims, U, normals, xi, beta, kappa, n_md, tau=1.0, tol=1e-12, P0=None,
                   t_antiperiodic=True):
    """One HMC trajectory as the paper's MDstep!: momenta from normals (or P0),
    pseudofermion eta = D^dag xi (no fermions when xi is None), S_f,old = |xi|^2,
    n_md leapfrog steps U(dt/2) P(dt) U(dt/2) of dt = tau / n_md with
    dP/dt = (1/2) TA(U dS/dU), and H = K + S_g + S_f before and after.
    Returns (U_new, P_new, H_old, H_new)."""
    P = momenta(normals) if P0 is None else P0.copy()
    eta = None if xi is None else dirac(dims, U, xi, kappa, dagger=True, t_antiperiodic=t_antiperiodic)
    S_f = 0.0 if xi is None else float(np.vdot(xi, xi).real)
    H_old = kinetic(P) + gauge_action(dims, U, beta) + S_f
    dt = tau / n_md
    for _ in range(n_md):
        U = exp_update(U, P, dt / 2)
        G = hmc_forces(dims, U, eta, beta, kappa, tol, t_antiperiodic)
        P = P + dt * 0.5 * traceless_antihermitian(G)
        U = exp_update(U, P, dt / 2)
    S_f = 0.0 if eta is None else fermi_action(dims, U, eta, kappa, tol=tol, t_antiperiodic=t_antiperiodic)[0]
    H_new = kinetic(P) + gauge_action(dims, U, beta) + S_f
    return U, P, H_old, H_new


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's site loop (n <= 0: unchanged); returns the count in force."""
    return int(_load().jo_set_threads(int(n)))


def parity_mask(dims) -> np.ndarray:
    """Boolean array [t, z, y, x]: True on odd sites."""
    nx, ny, nz, nt = dims
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    return ((x + y + z + t) % 2) == 1
