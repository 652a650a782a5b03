"""Thin ctypes binding of libjqcd.so (the C ABI in include/jqcd.h).

The functions ``jqcd_*`` are the C entry points with their C names.  The
classes below only marshal arguments: numpy arrays for host data, torch
CUDA tensors (raw byte buffers) for device data, torch streams for streams.
Every step of the computation runs in the library's CUDA kernels; there is
no fallback, and importing this module fails loudly when the library has not
been built (``python -m paper_2409_03030_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libjqcd.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBUSY, ETIMEOUT, ENOTFOUND, EBREAKDOWN = 0, -1, -2, -3, -4, -5, -6, -7, -8
PENDING = 1
PREC_DW, PREC_F32, PREC_F16N, PREC_F64 = 0, 1, 2, 3
CG_DW, CG_F64, CG_MIXED_F32, CG_MIXED_F16 = 0, 1, 2, 3
PRECS = {"dw": PREC_DW, "f32": PREC_F32, "f16n": PREC_F16N, "f64": PREC_F64}
MODES = {"dw": CG_DW, "f64": CG_F64, "mixed_f32": CG_MIXED_F32, "mixed_f16": CG_MIXED_F16}
NOALLOC_MAX_SITES_PER_PARITY = 16384 * 128  # JQCD_NOALLOC_MAX_SITES_PER_PARITY


class JqcdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"jqcd status {status}: {message}")
        self.status = status


class jqcd_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("t_antiperiodic", ctypes.c_int32)]


class jqcd_solve_params(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int32),
                ("eo", ctypes.c_int32), ("mode", ctypes.c_int32), ("verbose", ctypes.c_int32),
                ("delta", ctypes.c_double), ("use_x0", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class jqcd_request(ctypes.Structure):
    _fields_ = [("gauge_id", ctypes.c_uint64), ("params", jqcd_solve_params),
                ("b", ctypes.POINTER(ctypes.c_double)), ("x", ctypes.POINTER(ctypes.c_double))]


class jqcd_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("mean_s", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("peak_hbm_bytes", ctypes.c_double), ("peak_active", ctypes.c_int32),
                ("peak_queue", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class jqcd_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("reliable_updates", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("true_rel_resid", ctypes.c_double), ("full_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("gpu_seconds", ctypes.c_double),
                ("hop_bytes", ctypes.c_double), ("hop_count", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class jqcd_hmc_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kappa", ctypes.c_double), ("tau", ctypes.c_double),
                ("tol", ctypes.c_double), ("n_md", ctypes.c_int32), ("fermions", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("maxiter", ctypes.c_int32)]


class jqcd_hmc_info(ctypes.Structure):
    _fields_ = [("H_old", ctypes.c_double), ("H_new", ctypes.c_double), ("dH", ctypes.c_double),
                ("plaquette", ctypes.c_double), ("seconds", ctypes.c_double), ("accepted", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_st = ctypes.c_int32
_u64 = ctypes.c_uint64
_SIGNATURES = {
    "jqcd_abi_version": (ctypes.c_int32, []),
    "jqcd_kernel_launches": (ctypes.c_uint64, []),
    "jqcd_init": (_st, [ctypes.c_int, ctypes.POINTER(_vp)]),
    "jqcd_finalize": (_st, [_vp]),
    "jqcd_last_error": (ctypes.c_char_p, [_vp]),
    "jqcd_gauge_upload": (_st, [_vp, ctypes.POINTER(jqcd_lattice), _dp, ctypes.c_uint32,
                                ctypes.POINTER(_u64)]),
    "jqcd_gauge_free": (_st, [_vp, _u64]),
    "jqcd_spinor_bytes": (_st, [ctypes.POINTER(jqcd_lattice), ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_size_t)]),
    "jqcd_spinor_pack": (_st, [_vp, _u64, _dp, ctypes.c_int32, _vp, _vp, _vp]),
    "jqcd_spinor_unpack": (_st, [_vp, _u64, ctypes.c_int32, _vp, _vp, _dp, _vp]),
    "jqcd_dslash_eo": (_st, [_vp, _u64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                             _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "jqcd_dslash_eo_noalloc": (_st, [_vp, _u64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "jqcd_mdagm": (_st, [_vp, _u64, ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp, _vp]),
    "jqcd_dirac_apply": (_st, [_vp, _u64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _vp,
                               _vp, _vp, _vp, _vp]),
    "jqcd_cg_solve": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), _dp, _dp,
                            ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_cg_solve_batch": (_st, [_vp, ctypes.c_int32, ctypes.POINTER(_u64),
                                  ctypes.POINTER(jqcd_solve_params), ctypes.POINTER(_dp),
                                  ctypes.POINTER(_dp), ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_serve_start": (_st, [_vp, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32]),
    "jqcd_serve_submit": (_st, [_vp, ctypes.POINTER(jqcd_request), ctypes.POINTER(_u64)]),
    "jqcd_serve_poll": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_serve_stop": (_st, [_vp, ctypes.POINTER(jqcd_serve_stats)]),
    "jqcd_cg_solve_dev": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), _vp, _vp, _vp, _vp,
                                ctypes.POINTER(jqcd_solve_info), _vp]),
    "jqcd_fermi_action": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), _dp, _dp,
                                ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_fermi_force": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), _dp, _dp, _dp,
                               ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_fermi_force_xy": (_st, [_vp, _u64, ctypes.c_double, _dp, _dp, _dp]),
    "jqcd_fermi_force_dev": (_st, [_vp, _u64, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp]),
    "jqcd_linkfield_bytes": (_st, [ctypes.POINTER(jqcd_lattice), ctypes.POINTER(ctypes.c_size_t)]),
    "jqcd_staggered_bytes": (_st, [ctypes.POINTER(jqcd_lattice), ctypes.POINTER(ctypes.c_size_t)]),
    "jqcd_staggered_pack": (_st, [_vp, _u64, _dp, _vp, _vp, _vp]),
    "jqcd_staggered_unpack": (_st, [_vp, _u64, _vp, _vp, _dp, _vp]),
    "jqcd_staggered_dslash_eo": (_st, [_vp, _u64, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_double,
                                       ctypes.c_double, _vp, _vp]),
    "jqcd_staggered_apply": (_st, [_vp, _u64, ctypes.c_double, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "jqcd_staggered_solve": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), ctypes.c_double, _dp, _dp,
                                   ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_staggered_solve_dev": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), ctypes.c_double, _vp, _vp,
                                       _vp, _vp, ctypes.POINTER(jqcd_solve_info), _vp]),
    "jqcd_hmc_trajectory": (_st, [_vp, _u64, ctypes.POINTER(jqcd_hmc_params), _dp, _dp, ctypes.c_double,
                                  ctypes.POINTER(jqcd_hmc_info)]),
    "jqcd_gauge_plaquette": (_st, [_vp, _u64, _dp]),
    "jqcd_gauge_download": (_st, [_vp, _u64, _dp]),
    "jqcd_cg_multishift": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), ctypes.c_int32, _dp, _dp,
                                 ctypes.POINTER(_dp), ctypes.POINTER(jqcd_solve_info)]),
    "jqcd_cg_multishift_dev": (_st, [_vp, _u64, ctypes.POINTER(jqcd_solve_params), ctypes.c_int32, _dp,
                                     _vp, ctypes.POINTER(_vp), ctypes.POINTER(jqcd_solve_info), _vp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libjqcd.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2409_03030_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
        globals()[name] = fn
    return lib


_lib = _load()


def exported_symbols():
    return sorted(_SIGNATURES)


def _host_ptr(a: np.ndarray):
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError("host spinors/links must be C-contiguous complex128 arrays")
    return a.ctypes.data_as(_dp)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _dev_ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))


def lattice(dims, t_antiperiodic=True) -> jqcd_lattice:
    return jqcd_lattice((ctypes.c_int32 * 4)(*[int(d) for d in dims]), int(bool(t_antiperiodic)))


def spinor_bytes(dims, prec, t_antiperiodic=True) -> int:
    n = ctypes.c_size_t(0)
    lat = lattice(dims, t_antiperiodic)
    st = jqcd_spinor_bytes(ctypes.byref(lat), int(prec), ctypes.byref(n))
    if st != OK:
        raise JqcdError(st, "jqcd_spinor_bytes: bad lattice or precision")
    return n.value


class Context:
    """One jqcd context on one CUDA device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        st = jqcd_init(int(device), ctypes.byref(h))
        if st != OK:
            raise JqcdError(st, f"jqcd_init({device}) failed")
        self.h = h
        self.device = int(device)

    def close(self):
        if self.h:
            jqcd_finalize(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, st, what=""):
        if st not in (OK, PENDING):
            raise JqcdError(st, f"{what}: {jqcd_last_error(self.h).decode()}")
        return st

    def cg_solve_batch(self, gauges, bs, kappas, tols, mode=CG_MIXED_F16, maxiter=20000,
                       delta=0.0, check=True, verbose=0, out=None):
        """jqcd_cg_solve_batch: solve D_i x_i = b_i for all i together.
        gauges: list of Gauge; bs: host spinors; kappas, tols: per solve.
        Returns (list of x, list of info dicts, status)."""
        n = len(bs)
        bs = [np.ascontiguousarray(b, dtype=np.complex128) for b in bs]
        # written in full by the library; out: caller's C-contiguous complex128 arrays to reuse
        xs = list(out) if out is not None else [np.empty_like(b) for b in bs]
        for x, b in zip(xs, bs):
            if x.shape != b.shape or x.dtype != np.complex128 or not x.flags.c_contiguous:
                raise ValueError("out arrays must match b (C-contiguous complex128)")
        ids = (ctypes.c_uint64 * n)(*[g.id for g in gauges])
        params = (jqcd_solve_params * n)(*[
            Gauge.params(kappas[i], tols[i], maxiter, True, mode, verbose, delta, False)
            for i in range(n)])
        bp = (_dp * n)(*[_host_ptr(b) for b in bs])
        xp = (_dp * n)(*[_host_ptr(x) for x in xs])
        infos = (jqcd_solve_info * n)()
        st = jqcd_cg_solve_batch(self.h, n, ids, params, bp, xp, infos)
        if check:
            self.check(st, "jqcd_cg_solve_batch")
        return xs, [i.as_dict() for i in infos], st

    # ---- serving ------------------------------------------------------------
    def serve_start(self, hbm_budget_bytes, max_slots=32, max_queue=0, mode=CG_MIXED_F16):
        self.check(jqcd_serve_start(self.h, int(hbm_budget_bytes), int(max_slots), int(max_queue),
                                    int(mode)), "jqcd_serve_start")

    def serve_submit(self, gauge, b, x, kappa, tol, maxiter=20000, mode=CG_MIXED_F16, delta=0.0):
        """Queue a solve.  b, x: C-contiguous complex128 host arrays that must
        stay alive (and x untouched) until poll reports completion.  Returns
        (status, ticket); status is OK, EBUSY (queue full) or an error."""
        req = jqcd_request(int(gauge.id), Gauge.params(kappa, tol, maxiter, True, mode, 0, delta),
                           _host_ptr(b), _host_ptr(x))
        t = ctypes.c_uint64(0)
        st = jqcd_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        return st, t.value

    def serve_poll(self, ticket):
        info = jqcd_solve_info()
        st = jqcd_serve_poll(self.h, int(ticket), ctypes.byref(info))
        return st, (info.as_dict() if st != PENDING else None)

    def serve_stop(self):
        stats = jqcd_serve_stats()
        self.check(jqcd_serve_stop(self.h, ctypes.byref(stats)), "jqcd_serve_stop")
        return stats.as_dict()

    # ---- gauge fields -----------------------------------------------------
    def gauge_upload(self, dims, links: np.ndarray, t_antiperiodic=True) -> "Gauge":
        lat = lattice(dims, t_antiperiodic)
        gid = ctypes.c_uint64(0)
        links = np.ascontiguousarray(links, dtype=np.complex128)
        self.check(jqcd_gauge_upload(self.h, ctypes.byref(lat), _host_ptr(links), 0,
                                     ctypes.byref(gid)), "jqcd_gauge_upload")
        return Gauge(self, gid.value, tuple(int(d) for d in dims), bool(t_antiperiodic))


class Gauge:
    """A gauge field resident on the device, with the operators built on it."""

    def __init__(self, ctx: Context, gid: int, dims, t_antiperiodic: bool):
        self.ctx, self.id, self.dims, self.t_antiperiodic = ctx, gid, dims, t_antiperiodic
        self.volume = int(np.prod(dims))

    def free(self):
        if self.id:
            self.ctx.check(jqcd_gauge_free(self.ctx.h, self.id), "jqcd_gauge_free")
            self.id = 0

    def spinor_bytes(self, prec) -> int:
        return spinor_bytes(self.dims, prec, self.t_antiperiodic)

    def empty(self, prec):
        """One parity of a device spinor field (torch uint8 buffer)."""
        import torch
        return torch.empty(self.spinor_bytes(prec), dtype=torch.uint8,
                           device=f"cuda:{self.ctx.device}")

    def pack(self, host: np.ndarray, prec, stream=None):
        host = np.ascontiguousarray(host, dtype=np.complex128)
        ev, od = self.empty(prec), self.empty(prec)
        self.ctx.check(jqcd_spinor_pack(self.ctx.h, self.id, _host_ptr(host), int(prec),
                                        _dev_ptr(ev), _dev_ptr(od), _stream_ptr(stream)),
                       "jqcd_spinor_pack")
        return ev, od

    def unpack(self, even, odd, prec, stream=None) -> np.ndarray:
        nx, ny, nz, nt = self.dims
        out = np.empty((4, nt, nz, ny, nx, 3), dtype=np.complex128)
        self.ctx.check(jqcd_spinor_unpack(self.ctx.h, self.id, int(prec), _dev_ptr(even),
                                          _dev_ptr(odd), _host_ptr(out), _stream_ptr(stream)),
                       "jqcd_spinor_unpack")
        return out

    def dslash_eo(self, prec, out_parity, dagger, inp, x, out, a=0.0, b=1.0, norm2=None,
                  stream=None):
        self.ctx.check(jqcd_dslash_eo(self.ctx.h, self.id, int(prec), int(out_parity), int(dagger),
                                      _dev_ptr(inp), _dev_ptr(x), _dev_ptr(out), float(a),
                                      float(b), _dev_ptr(norm2), _stream_ptr(stream)),
                       "jqcd_dslash_eo")

    def dslash_eo_noalloc(self, prec, out_parity, dagger, inp, x, out, a=0.0, b=1.0, norm2=None,
                          stream=None):
        """jqcd_dslash_eo_noalloc: the hop without any allocation inside the call."""
        self.ctx.check(jqcd_dslash_eo_noalloc(self.ctx.h, self.id, int(prec), int(out_parity),
                                              int(dagger), _dev_ptr(inp), _dev_ptr(x),
                                              _dev_ptr(out), float(a), float(b), _dev_ptr(norm2),
                                              _stream_ptr(stream)),
                       "jqcd_dslash_eo_noalloc")

    def mdagm(self, prec, kappa, inp, out, norm2=None, stream=None):
        self.ctx.check(jqcd_mdagm(self.ctx.h, self.id, int(prec), float(kappa), _dev_ptr(inp),
                                  _dev_ptr(out), _dev_ptr(norm2), _stream_ptr(stream)),
                       "jqcd_mdagm")

    def dirac_apply(self, prec, kappa, dagger, in_even, in_odd, out_even, out_odd, stream=None):
        self.ctx.check(jqcd_dirac_apply(self.ctx.h, self.id, int(prec), float(kappa), int(dagger),
                                        _dev_ptr(in_even), _dev_ptr(in_odd), _dev_ptr(out_even),
                                        _dev_ptr(out_odd), _stream_ptr(stream)),
                       "jqcd_dirac_apply")

    @staticmethod
    def params(kappa, tol=1e-10, maxiter=20000, eo=True, mode=CG_DW, verbose=0, delta=0.0,
               use_x0=False) -> jqcd_solve_params:
        return jqcd_solve_params(float(kappa), float(tol), int(maxiter), int(bool(eo)), int(mode),
                                 int(verbose), float(delta), int(bool(use_x0)), 0)

    def cg_solve(self, b: np.ndarray, kappa, tol=1e-10, maxiter=20000, eo=True, mode=CG_DW,
                 verbose=0, delta=0.0, x0=None, check=True, out=None):
        """Solve D x = b from host arrays; returns (x, info dict, status).  out: a
        C-contiguous complex128 array to write x into (reused, no allocation)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if out is not None:
            if out.shape != b.shape or out.dtype != np.complex128 or not out.flags.c_contiguous:
                raise ValueError("out must match b (C-contiguous complex128)")
            x = out
            if x0 is not None:
                x[...] = x0
        else:
            x = np.empty_like(b) if x0 is None else np.array(x0, dtype=np.complex128, order="C")
        p = self.params(kappa, tol, maxiter, eo, mode, verbose, delta, x0 is not None)
        info = jqcd_solve_info()
        st = jqcd_cg_solve(self.ctx.h, self.id, ctypes.byref(p), _host_ptr(b), _host_ptr(x),
                           ctypes.byref(info))
        if check:
            self.ctx.check(st, "jqcd_cg_solve")
        return x, info.as_dict(), st

    # ---- hybrid Monte Carlo (paper: MDstep!) -------------------------------------
    def plaquette(self) -> float:
        v = ctypes.c_double(0.0)
        self.ctx.check(jqcd_gauge_plaquette(self.ctx.h, self.id, ctypes.byref(v)), "jqcd_gauge_plaquette")
        return v.value

    def download(self) -> np.ndarray:
        out = np.empty(self.link_shape(), dtype=np.complex128)
        self.ctx.check(jqcd_gauge_download(self.ctx.h, self.id, _host_ptr(out)), "jqcd_gauge_download")
        return out

    def hmc_trajectory(self, normals, xi, u, beta, kappa=0.12, tau=1.0, n_md=10, tol=1e-10, mode=CG_DW,
                       maxiter=20000, check=True):
        """One trajectory on this field; normals: [mu, t, z, y, x, 8] (or flat, link-major),
        xi: host spinor or None (pure gauge); u: Metropolis uniform.  Returns (info, status)."""
        nrm = np.ascontiguousarray(normals, dtype=np.float64)
        p = jqcd_hmc_params(float(beta), float(kappa), float(tau), float(tol), int(n_md), int(xi is not None),
                            int(mode), int(maxiter))
        xp = None
        if xi is not None:
            xi = np.ascontiguousarray(xi, dtype=np.complex128)
            xp = _host_ptr(xi)
        info = jqcd_hmc_info()
        st = jqcd_hmc_trajectory(self.ctx.h, self.id, ctypes.byref(p), nrm.ctypes.data_as(_dp), xp, float(u),
                                 ctypes.byref(info))
        if check:
            self.ctx.check(st, "jqcd_hmc_trajectory")
        return info.as_dict(), st

    # ---- staggered fermions (paper: Dirac_operator "staggered") ----------------------
    def colour_shape(self):
        nx, ny, nz, nt = self.dims
        return (nt, nz, ny, nx, 3)

    def stag_bytes(self) -> int:
        n = ctypes.c_size_t(0)
        lat = lattice(self.dims, self.t_antiperiodic)
        if jqcd_staggered_bytes(ctypes.byref(lat), ctypes.byref(n)) != OK:
            raise ValueError("bad lattice")
        return n.value

    def stag_empty(self):
        import torch
        return torch.empty(self.stag_bytes(), dtype=torch.uint8, device=f"cuda:{self.ctx.device}")

    def stag_pack(self, host, stream=None):
        host = np.ascontiguousarray(host, dtype=np.complex128)
        ev, od = self.stag_empty(), self.stag_empty()
        self.ctx.check(jqcd_staggered_pack(self.ctx.h, self.id, _host_ptr(host), _dev_ptr(ev), _dev_ptr(od),
                                           _stream_ptr(stream)), "jqcd_staggered_pack")
        return ev, od

    def stag_unpack(self, even, odd, stream=None):
        out = np.empty(self.colour_shape(), dtype=np.complex128)
        self.ctx.check(jqcd_staggered_unpack(self.ctx.h, self.id, _dev_ptr(even), _dev_ptr(odd), _host_ptr(out),
                                             _stream_ptr(stream)), "jqcd_staggered_unpack")
        return out

    def stag_dslash_eo(self, out_parity, dagger, inp, x, out, a=0.0, b=1.0, norm2=None, stream=None):
        self.ctx.check(jqcd_staggered_dslash_eo(self.ctx.h, self.id, int(out_parity), int(dagger), _dev_ptr(inp),
                                                _dev_ptr(x), _dev_ptr(out), float(a), float(b), _dev_ptr(norm2),
                                                _stream_ptr(stream)), "jqcd_staggered_dslash_eo")

    def stag_apply(self, mass, dagger, ie, io, oe, oo, stream=None):
        self.ctx.check(jqcd_staggered_apply(self.ctx.h, self.id, float(mass), int(dagger), _dev_ptr(ie), _dev_ptr(io),
                                            _dev_ptr(oe), _dev_ptr(oo), _stream_ptr(stream)), "jqcd_staggered_apply")

    def stag_solve(self, b, mass, tol=1e-10, maxiter=20000, check=True):
        """Solve the staggered D x = b from host arrays; returns (x, info dict, status)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        x = np.empty_like(b)
        p = self.params(0.0, tol, maxiter, True, CG_DW)
        info = jqcd_solve_info()
        st = jqcd_staggered_solve(self.ctx.h, self.id, ctypes.byref(p), float(mass), _host_ptr(b), _host_ptr(x),
                                  ctypes.byref(info))
        if check:
            self.ctx.check(st, "jqcd_staggered_solve")
        return x, info.as_dict(), st

    def stag_solve_dev(self, be, bo, xe, xo, mass, tol=1e-10, maxiter=20000, stream=None, check=True):
        p = self.params(0.0, tol, maxiter, True, CG_DW)
        info = jqcd_solve_info()
        st = jqcd_staggered_solve_dev(self.ctx.h, self.id, ctypes.byref(p), float(mass), _dev_ptr(be), _dev_ptr(bo),
                                      _dev_ptr(xe), _dev_ptr(xo), ctypes.byref(info), _stream_ptr(stream))
        if check:
            self.ctx.check(st, "jqcd_staggered_solve_dev")
        return info.as_dict(), st

    # ---- multi-shift CG (RHMC) ----------------------------------------------------
    def cg_multishift(self, rhs, kappa, shifts, tol=1e-10, maxiter=20000, check=True):
        """Solve (Mhat^dag Mhat + shifts[i]) x_i = rhs (even sites) for all i at
        once; returns (list of x_i, list of info dicts, status)."""
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        n = len(shifts)
        sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
        xs = [np.empty_like(rhs) for _ in range(n)]
        xp = (_dp * n)(*[_host_ptr(x) for x in xs])
        infos = (jqcd_solve_info * n)()
        p = self.params(kappa, tol, maxiter, True, CG_DW)
        st = jqcd_cg_multishift(self.ctx.h, self.id, ctypes.byref(p), n, sh, _host_ptr(rhs), xp, infos)
        if check:
            self.ctx.check(st, "jqcd_cg_multishift")
        return xs, [i.as_dict() for i in infos], st

    def cg_multishift_dev(self, rhs_even, x_evens, kappa, shifts, tol=1e-10, maxiter=20000, stream=None,
                          check=True):
        n = len(shifts)
        sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
        xp = (_vp * n)(*[_dev_ptr(x) for x in x_evens])
        infos = (jqcd_solve_info * n)()
        p = self.params(kappa, tol, maxiter, True, CG_DW)
        st = jqcd_cg_multishift_dev(self.ctx.h, self.id, ctypes.byref(p), n, sh, _dev_ptr(rhs_even), xp, infos,
                                    _stream_ptr(stream))
        if check:
            self.ctx.check(st, "jqcd_cg_multishift_dev")
        return [i.as_dict() for i in infos], st

    # ---- fermion action and force (paper: evaluate_FermiAction, calc_UdSfdU) ----
    def link_shape(self):
        nx, ny, nz, nt = self.dims
        return (4, nt, nz, ny, nx, 3, 3)  # [mu, t, z, y, x, b, a] like the uploaded links

    def fermi_action(self, eta, kappa, tol=1e-10, maxiter=20000, mode=CG_DW, check=True):
        """S = eta^dag (D^dag D)^-1 eta; returns (S, info dict, status)."""
        eta = np.ascontiguousarray(eta, dtype=np.complex128)
        p = self.params(kappa, tol, maxiter, True, mode)
        S = ctypes.c_double(0.0)
        info = jqcd_solve_info()
        st = jqcd_fermi_action(self.ctx.h, self.id, ctypes.byref(p), _host_ptr(eta), ctypes.byref(S),
                               ctypes.byref(info))
        if check:
            self.ctx.check(st, "jqcd_fermi_action")
        return S.value, info.as_dict(), st

    def fermi_force(self, eta, kappa, tol=1e-10, maxiter=20000, mode=CG_DW, check=True):
        """(S, U dS/dU as links [mu,t,z,y,x,b,a], info dict, status)."""
        eta = np.ascontiguousarray(eta, dtype=np.complex128)
        p = self.params(kappa, tol, maxiter, True, mode)
        G = np.empty(self.link_shape(), dtype=np.complex128)
        S = ctypes.c_double(0.0)
        info = jqcd_solve_info()
        st = jqcd_fermi_force(self.ctx.h, self.id, ctypes.byref(p), _host_ptr(eta), _host_ptr(G),
                              ctypes.byref(S), ctypes.byref(info))
        if check:
            self.ctx.check(st, "jqcd_fermi_force")
        return S.value, G, info.as_dict(), st

    def fermi_force_xy(self, X, Y, kappa):
        """U dS/dU from given X = (D^dag D)^-1 eta and Y = D X (host spinors)."""
        X = np.ascontiguousarray(X, dtype=np.complex128)
        Y = np.ascontiguousarray(Y, dtype=np.complex128)
        G = np.empty(self.link_shape(), dtype=np.complex128)
        self.ctx.check(jqcd_fermi_force_xy(self.ctx.h, self.id, float(kappa), _host_ptr(X), _host_ptr(Y),
                                           _host_ptr(G)), "jqcd_fermi_force_xy")
        return G

    def linkfield_bytes(self) -> int:
        n = ctypes.c_size_t(0)
        lat = lattice(self.dims, self.t_antiperiodic)
        if jqcd_linkfield_bytes(ctypes.byref(lat), ctypes.byref(n)) != OK:
            raise ValueError("bad lattice")
        return n.value

    def fermi_force_dev(self, kappa, X_even, X_odd, Y_even, Y_odd, out, stream=None):
        """U dS/dU into a device double-word link field (out: linkfield_bytes())."""
        self.ctx.check(jqcd_fermi_force_dev(self.ctx.h, self.id, float(kappa), _dev_ptr(X_even),
                                            _dev_ptr(X_odd), _dev_ptr(Y_even), _dev_ptr(Y_odd),
                                            _dev_ptr(out), _stream_ptr(stream)), "jqcd_fermi_force_dev")

    def cg_solve_dev(self, b_even, b_odd, x_even, x_odd, kappa, tol=1e-10, maxiter=20000, eo=True,
                     mode=CG_DW, verbose=0, delta=0.0, use_x0=False, stream=None, check=True):
        p = self.params(kappa, tol, maxiter, eo, mode, verbose, delta, use_x0)
        info = jqcd_solve_info()
        st = jqcd_cg_solve_dev(self.ctx.h, self.id, ctypes.byref(p), _dev_ptr(b_even),
                               _dev_ptr(b_odd), _dev_ptr(x_even), _dev_ptr(x_odd),
                               ctypes.byref(info), _stream_ptr(stream))
        if check:
            self.ctx.check(st, "jqcd_cg_solve_dev")
        return info.as_dict(), st
