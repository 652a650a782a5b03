"""Seeded synthetic inputs: SU(3) gauge fields and fermion sources.

These generators draw the inputs that both the CUDA library and the CPU
oracle consume (random numbers the method itself would draw are inputs here).
They contain none of the Wilson-Dirac or solver arithmetic.  Arrays are
complex128 numpy arrays in the canonical host layouts:

* spinor ``psi[alpha, it, iz, iy, ix, ic]`` -- the column-major order of
  JuliaQCD's ``x[ic,ix,iy,iz,it,ialpha]`` (paper, "Definition of pseudo-fermion
  fields"), i.e. complex offset ``ic + 3*(site + V*alpha)``;
* links ``U[mu, it, iz, iy, ix, b, a]`` = element (a, b) of U_mu(x), the
  column-major order of ``U[mu][a,b,ix,iy,iz,it]`` (gauge field shape
  ``(NC,NC,NX,NY,NZ,NT)``, paper, HMC with fermions listing).  Use
  :func:`link_matrices` for a ``[..., a, b]`` view.

``dims`` is always ``(NX, NY, NZ, NT)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libjqcd_synth.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in-tree with gcc (OpenMP if available)."""
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


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.synth_gauge.argtypes = [dp, ip, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]
        lib.synth_gaussian_spinor.argtypes = [dp, ip, ctypes.c_uint64]
        lib.synth_point_source.argtypes = [dp, ip, ctypes.c_int, ctypes.c_int]
        lib.synth_gauge_transform.argtypes = [dp, ip, ctypes.c_uint64]
        lib.synth_uniforms.argtypes = [dp, ctypes.c_uint64, ctypes.c_uint64]
        for f in (lib.synth_gauge, lib.synth_gaussian_spinor, lib.synth_point_source,
                  lib.synth_gauge_transform, lib.synth_uniforms):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dims(dims):
    d = tuple(int(v) for v in dims)
    if len(d) != 4 or min(d) < 1:
        raise ValueError(f"dims must be 4 positive extents (NX,NY,NZ,NT), got {dims}")
    return d, (ctypes.c_int * 4)(*d)


def _dptr(a: np.ndarray):
    return a.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def spinor_shape(dims):
    nx, ny, nz, nt = dims
    return (4, nt, nz, ny, nx, 3)


def gauge_shape(dims):
    nx, ny, nz, nt = dims
    return (4, nt, nz, ny, nx, 3, 3)


def gauge(dims, kind: str = "expi", eps: float = 0.3, seed: int = 1) -> np.ndarray:
    """Gauge links.  kind: 'unit' (cold start), 'haar' (Haar SU(3) by QR of a
    complex Gaussian, det fixed to 1) or 'expi' (U = exp(i*eps*H), H a
    traceless Hermitian Gaussian matrix)."""
    d, cd = _dims(dims)
    k = {"unit": 0, "haar": 1, "expi": 2}[kind]
    out = np.empty(gauge_shape(d), dtype=np.complex128)
    rc = _load().synth_gauge(_dptr(out), cd, k, float(eps), int(seed) & (2**64 - 1))
    if rc != 0:
        raise RuntimeError("synth_gauge failed")
    return out


def gaussian_spinor(dims, seed: int = 1) -> np.ndarray:
    """Gaussian source: each complex component has re, im ~ N(0, 1/2)."""
    d, cd = _dims(dims)
    out = np.empty(spinor_shape(d), dtype=np.complex128)
    if _load().synth_gaussian_spinor(_dptr(out), cd, int(seed) & (2**64 - 1)) != 0:
        raise RuntimeError("synth_gaussian_spinor failed")
    return out


def gaussian_colour(dims, seed: int = 1) -> np.ndarray:
    """Gaussian staggered field (one colour vector per site, [t, z, y, x, colour]):
    spin component 0 of gaussian_spinor(dims, seed), re, im ~ N(0, 1/2)."""
    return np.ascontiguousarray(gaussian_spinor(dims, seed)[0])


def colour_shape(dims):
    nx, ny, nz, nt = (int(v) for v in dims)
    return (nt, nz, ny, nx, 3)


def point_source(dims, spin: int, colour: int) -> np.ndarray:
    """delta at site (0,0,0,0), spin index `spin`, colour index `colour`."""
    d, cd = _dims(dims)
    out = np.empty(spinor_shape(d), dtype=np.complex128)
    if _load().synth_point_source(_dptr(out), cd, int(spin), int(colour)) != 0:
        raise ValueError("bad spin/colour")
    return out


def gauge_transform(dims, seed: int = 7) -> np.ndarray:
    """Haar-random Omega(x) per site, shape (NT,NZ,NY,NX,3(b),3(a))."""
    d, cd = _dims(dims)
    nx, ny, nz, nt = d
    out = np.empty((nt, nz, ny, nx, 3, 3), dtype=np.complex128)
    if _load().synth_gauge_transform(_dptr(out), cd, int(seed) & (2**64 - 1)) != 0:
        raise RuntimeError("synth_gauge_transform failed")
    return out


def uniforms(n: int, seed: int = 1) -> np.ndarray:
    out = np.empty(int(n), dtype=np.float64)
    _load().synth_uniforms(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n),
                           int(seed) & (2**64 - 1))
    return out


def link_matrices(U: np.ndarray) -> np.ndarray:
    """View of links with the last two axes ordered [a (row), b (column)]."""
    return np.swapaxes(U, -1, -2)
