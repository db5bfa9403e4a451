"""Thin Python binding of the C ABI in ``include/frmg.h`` (ctypes).

Argument marshalling only: every step of the solve runs in ``libfrmg.so``.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays; their data
pointers are passed straight to the library, which stages host memory itself.
There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ENOCONV, FR_EDIVERGED, FR_ETIMEOUT = range(7)
FR_FP64, FR_MIXED = 0, 1

_lock = threading.Lock()
_lib = None


class fr_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_vcycles", ctypes.c_int),
                ("pre", ctypes.c_int), ("post", ctypes.c_int), ("prec", ctypes.c_int),
                ("newton_step_cap", ctypes.c_double), ("inner_cycles", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("allow_negative_density", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("temporal_depth", ctypes.c_int),
                ("tiling", ctypes.c_int), ("defect_precision", ctypes.c_int),
                ("tau_alpha", ctypes.c_double), ("relax", ctypes.c_double),
                ("fmg", ctypes.c_int), ("initial_guess", ctypes.c_int),
                ("smooth_tile", ctypes.c_int)]


FR_HIST = 64


class fr_stats(ctypes.Structure):
    _fields_ = [("vcycles", ctypes.c_int), ("outer", ctypes.c_int),
                ("res0_rms", ctypes.c_double), ("res_rms", ctypes.c_double),
                ("res_max", ctypes.c_double), ("seconds", ctypes.c_double),
                ("nhist", ctypes.c_int), ("hist", ctypes.c_double * FR_HIST),
                ("tau_rms", ctypes.c_double), ("host_copies", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "hist"}
        d["hist"] = list(self.hist[: self.nhist])
        return d


class fr_patch(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int), ("origin", ctypes.c_int * 3), ("n", ctypes.c_int * 3),
                ("density", ctypes.c_void_p), ("u", ctypes.c_void_p)]


EXPORTS = ["fr_opts_default", "fr_status_string", "fr_last_error", "fr_ctx_create",
           "fr_ctx_destroy", "fr_constants", "fr_solve", "fr_solve_levels", "fr_solve_batch",
           "fr_cic_assign", "fr_smooth", "fr_residual", "fr_restrict", "fr_prolong_correct",
           "fr_patch_bc", "fr_vcycles", "fr_launch_count", "fr_profile", "fr_profile_entry", "fr_smooth_f32", "fr_residual_df",
           "fr_residual_norm_noalloc", "fr_autotune", "fr_poisson_solve", "fr_poisson_source",
           "fr_tsc_assign", "fr_particle_forces", "fr_solve_masked", "fr_symmetron_solve",
           "fr_autotune_batch"]


def lib_path():
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfrmg.so; raises if it is not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"{path} is not built; run paper_1110_1379_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "fr_opts_default": (None, [P]),
            "fr_status_string": (ctypes.c_char_p, [I]),
            "fr_last_error": (ctypes.c_char_p, []),
            "fr_ctx_create": (I, [P, I]),
            "fr_ctx_destroy": (None, [P]),
            "fr_constants": (I, [D, I, D, D, D, P]),
            "fr_solve": (I, [P, P, P, D, D, D, D, D, P, P, P, P]),
            "fr_vcycles": (I, [P, P, P, D, D, D, D, P, I, P, P, P]),
            "fr_solve_levels": (I, [P, P, P, D, D, D, D, D, D, P, P, I, P, P, P]),
            "fr_solve_batch": (I, [P, I, P, P, P, P, P, D, D, P, P, P, P]),
            "fr_cic_assign": (I, [P, P, L, P, P, P]),
            "fr_smooth": (I, [P, P, P, P, P, D, D, D, D, D, P, I, D, P]),
            "fr_residual": (I, [P, P, P, P, P, D, D, D, D, D, P, P, P]),
            "fr_restrict": (I, [P, P, P, P, P]),
            "fr_prolong_correct": (I, [P, P, P, P, P, I, P]),
            "fr_patch_bc": (I, [P, P, P, I, P, P, P, P, P]),
            "fr_launch_count": (L, [P]),
            "fr_profile": (I, [P, I]),
            "fr_smooth_f32": (I, [P, P, P, P, P, D, D, D, D, D, P, I, D, I, P]),
            "fr_residual_df": (I, [P, P, P, P, D, D, D, D, D, P, P, P]),
            "fr_residual_norm_noalloc": (I, [P, P, P, D, D, D, D, D, P, P, P]),
            "fr_autotune": (I, [P, P, P, D, D, D, D, D, P, P, P, P]),
            "fr_poisson_solve": (I, [P, P, P, P, D, D, D, D, P, D, D, P, P, P, P, P]),
            "fr_poisson_source": (I, [P, P, P, P, D, D, D, D, P, P]),
            "fr_tsc_assign": (I, [P, P, L, P, P, P]),
            "fr_particle_forces": (I, [P, P, P, P, L, I, P, P]),
            "fr_solve_masked": (I, [P, P, P, P, D, D, D, D, D, D, P, P, P, P]),
            "fr_profile_entry": (I, [P, I, P, I, P, P]),
            "fr_symmetron_solve": (I, [P, P, P, D, D, D, D, D, P, P, P, P]),
            "fr_autotune_batch": (I, [P, I, P, P, P, P, P, D, D, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class FRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_f64(a, name):
    if a is None:
        return
    dt = str(getattr(a, "dtype", ""))
    if "float64" not in dt:
        raise TypeError(f"{name} must be float64, got {dt}")


def _dims(shape):
    """array shape (n2, n1, n0) -> int[3] (n0, n1, n2)."""
    if len(shape) != 3:
        raise ValueError("fields must be 3-D (n2, n1, n0)")
    return (ctypes.c_int * 3)(int(shape[2]), int(shape[1]), int(shape[0]))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def residual_norm_noalloc(u, density, out2, *, box, a, omega_m, fr0, h=None, ub=None,
                          stream=None):
    """Allocation-free residual norm: out2 (device, 2 doubles) <- (rms, max) of
    L(u); asynchronous on the stream.  Returns the status code."""
    h = 1.0 / u.shape[2] if h is None else h
    lib = load()
    return lib.fr_residual_norm_noalloc(_ptr(u), _ptr(density), _dims(u.shape), h, box, a,
                                        omega_m, fr0, _ptr(ub), _ptr(out2), _stream(stream))


def constants(box, n0, a, omega_m, fr0):
    """(alpha, beta, gamma, c~, |fbar~_R|, ubar) as the library derives them."""
    out = (ctypes.c_double * 6)()
    st = load().fr_constants(box, n0, a, omega_m, fr0, out)
    if st != FR_OK:
        raise FRError(st, "fr_constants failed")
    return tuple(out)


class Context:
    """Owns one ``frmg_ctx`` (device workspace, allocator)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self._h = ctypes.c_void_p()
        st = self.lib.fr_ctx_create(ctypes.byref(self._h), device)
        self._raise(st, "fr_ctx_create")

    def close(self):
        if self._h:
            self.lib.fr_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st, what, allow=()):
        if st != FR_OK and st not in allow:
            msg = self.lib.fr_last_error().decode(errors="replace")
            raise FRError(st, f"{what}: {self.lib.fr_status_string(st).decode()}: {msg}")
        return st

    @staticmethod
    def opts(**kw):
        o = fr_opts()
        load().fr_opts_default(ctypes.byref(o))
        for k, v in kw.items():
            if k == "prec" and isinstance(v, str):
                v = {"fp64": FR_FP64, "mixed": FR_MIXED}[v]
            setattr(o, k, v)
        return o

    @property
    def launches(self):
        return int(self.lib.fr_launch_count(self._h))

    def profile(self, enable=True):
        self._raise(self.lib.fr_profile(self._h, int(enable)), "fr_profile")

    def profile_read(self):
        """{kernel family: (launches, total ms)} accumulated since profile(True)."""
        out = {}
        i = 0
        name = ctypes.create_string_buffer(64)
        cnt = ctypes.c_longlong()
        ms = ctypes.c_double()
        while self.lib.fr_profile_entry(self._h, i, name, 64, ctypes.byref(cnt),
                                        ctypes.byref(ms)) == FR_OK:
            out[name.value.decode()] = (int(cnt.value), float(ms.value))
            i += 1
        return out

    def solve(self, density, u, *, box, a, omega_m, fr0, tol=1e-8, stream=None,
              raise_on=(FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ETIMEOUT), **opts):
        _check_f64(density, "density")
        _check_f64(u, "u")
        o = self.opts(tol=tol, **opts)
        s = fr_stats()
        st = self.lib.fr_solve(self._h, _ptr(density), _dims(density.shape), box, a, omega_m,
                               fr0, tol, _ptr(u), ctypes.byref(o), ctypes.byref(s),
                               _stream(stream))
        if st in raise_on:
            self._raise(st, "fr_solve")
        return st, s

    def solve_masked(self, density, mask, u, *, h, box, a, omega_m, fr0, tol=1e-8, stream=None,
                     raise_on=(FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ETIMEOUT), **opts):
        """General mask scheme on one region (box of cells with a mask per cell;
        u: initial/ghost values in, solution out).  Returns (status, stats)."""
        _check_f64(density, "density")
        _check_f64(mask, "mask")
        _check_f64(u, "u")
        o = self.opts(tol=tol, **opts)
        s = fr_stats()
        st = self.lib.fr_solve_masked(self._h, _ptr(density), _ptr(mask), _dims(u.shape), h, box,
                                      a, omega_m, fr0, tol, _ptr(u), ctypes.byref(o),
                                      ctypes.byref(s), _stream(stream))
        if st in raise_on:
            self._raise(st, "fr_solve_masked")
        return st, s

    def symmetron(self, density, chi, *, box, a, a_ssb, lambda0, tol=1e-8, stream=None,
                  raise_on=(FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ETIMEOUT), **opts):
        """Symmetron field chi = phi/phi_0 (in: initial guess unless
        initial_guess=0; out: solution).  Returns (status, stats)."""
        _check_f64(density, "density")
        _check_f64(chi, "chi")
        o = self.opts(tol=tol, **opts)
        s = fr_stats()
        st = self.lib.fr_symmetron_solve(self._h, _ptr(density), _dims(density.shape), box, a,
                                         a_ssb, lambda0, tol, _ptr(chi), ctypes.byref(o),
                                         ctypes.byref(s), _stream(stream))
        if st in raise_on:
            self._raise(st, "fr_symmetron_solve")
        return st, s

    def poisson(self, density, u, phi, *, box, a, omega_m, fr0, tol=1e-8, phib=None, h=None,
                stream=None, raise_on=(FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ETIMEOUT), **opts):
        """Modified Poisson solve for Phi given the f(R) solution u; phi in/out.
        Returns (status, stats, source mean removed)."""
        _check_f64(density, "density")
        _check_f64(u, "u")
        _check_f64(phi, "phi")
        o = self.opts(tol=tol, **opts)
        s = fr_stats()
        mean = ctypes.c_double(0.0)
        st = self.lib.fr_poisson_solve(self._h, _ptr(density), _ptr(u), _dims(phi.shape), box, a,
                                       omega_m, fr0, _ptr(phib), 0.0 if h is None else h, tol,
                                       _ptr(phi), ctypes.byref(o), ctypes.byref(s),
                                       ctypes.byref(mean), _stream(stream))
        if st in raise_on:
            self._raise(st, "fr_poisson_solve")
        return st, s, mean.value

    def poisson_source(self, density, u, out, *, box, a, omega_m, fr0, stream=None):
        """The Poisson source s (FP64) of density and u into out."""
        st = self.lib.fr_poisson_source(self._h, _ptr(density), _ptr(u), _dims(out.shape), box, a,
                                        omega_m, fr0, _ptr(out), _stream(stream))
        self._raise(st, "fr_poisson_source")

    def autotune(self, density, *, box, a, omega_m, fr0, tol=1e-8, stream=None, **base):
        """Fastest (pre, post, temporal_depth) for this problem; returns (opts dict, seconds)."""
        b = self.opts(tol=tol, **base)
        best = fr_opts()
        secs = ctypes.c_double()
        st = self.lib.fr_autotune(self._h, _ptr(density), _dims(density.shape), box, a, omega_m,
                                  fr0, tol, ctypes.byref(b), ctypes.byref(best),
                                  ctypes.byref(secs), _stream(stream))
        self._raise(st, "fr_autotune")
        return {k: getattr(best, k) for k, _ in fr_opts._fields_}, secs.value

    def vcycles(self, density, u, ncycles, *, box, a, omega_m, fr0, stream=None, **opts):
        o = self.opts(**opts)
        s = fr_stats()
        st = self.lib.fr_vcycles(self._h, _ptr(density), _dims(density.shape), box, a, omega_m,
                                 fr0, _ptr(u), ncycles, ctypes.byref(o), ctypes.byref(s),
                                 _stream(stream))
        self._raise(st, "fr_vcycles")
        return s

    def solve_batch(self, densities, us, *, boxes, avals, fr0s, omega_m, tol=1e-8, stream=None,
                    **opts):
        n = len(densities)
        dens = (ctypes.c_void_p * n)(*[_ptr(d).value for d in densities])
        uu = (ctypes.c_void_p * n)(*[_ptr(x).value for x in us])
        dims = ((ctypes.c_int * 3) * n)(*[_dims(d.shape) for d in densities])
        bx = (ctypes.c_double * n)(*boxes)
        av = (ctypes.c_double * n)(*avals)
        fv = (ctypes.c_double * n)(*fr0s)
        o = self.opts(tol=tol, **opts)
        stats = (fr_stats * n)()
        st = self.lib.fr_solve_batch(self._h, n, dens, dims, bx, av, fv, omega_m, tol, uu,
                                     ctypes.byref(o), stats, _stream(stream))
        self._raise(st, "fr_solve_batch", allow=(FR_ENOCONV, FR_EDIVERGED))
        return st, list(stats)

    def autotune_batch(self, densities, *, boxes, avals, fr0s, omega_m, tol=1e-8, stream=None,
                       **base):
        """Fastest batch setting (V-cycle shape, relaxation, tiling, smoother
        tile) for these fields; returns (opts dict, seconds)."""
        n = len(densities)
        dens = (ctypes.c_void_p * n)(*[_ptr(d).value for d in densities])
        dims = ((ctypes.c_int * 3) * n)(*[_dims(d.shape) for d in densities])
        bx = (ctypes.c_double * n)(*boxes)
        av = (ctypes.c_double * n)(*avals)
        fv = (ctypes.c_double * n)(*fr0s)
        b = self.opts(tol=tol, **base)
        best = fr_opts()
        secs = ctypes.c_double()
        st = self.lib.fr_autotune_batch(self._h, n, dens, dims, bx, av, fv, omega_m, tol,
                                        ctypes.byref(b), ctypes.byref(best), ctypes.byref(secs),
                                        _stream(stream))
        self._raise(st, "fr_autotune_batch")
        return {k: getattr(best, k) for k, _ in fr_opts._fields_}, secs.value

    def solve_levels(self, density, u, patches, *, box, a, omega_m, fr0, tol=1e-8,
                     tol_patch=None, stream=None, **opts):
        """patches: list of dicts {parent, origin (x,y,z), density, u}."""
        tol_patch = tol if tol_patch is None else tol_patch
        n = len(patches)
        arr = (fr_patch * max(n, 1))()
        for i, p in enumerate(patches):
            arr[i].parent = p["parent"]
            for d in range(3):
                arr[i].origin[d] = p["origin"][d]
            dims = _dims(p["density"].shape)
            for d in range(3):
                arr[i].n[d] = dims[d]
            arr[i].density = _ptr(p["density"])
            arr[i].u = _ptr(p["u"])
        o = self.opts(tol=tol, **opts)
        stats = (fr_stats * (n + 1))()
        st = self.lib.fr_solve_levels(self._h, _ptr(density), _dims(density.shape), box, a,
                                      omega_m, fr0, tol, tol_patch, _ptr(u), arr, n,
                                      ctypes.byref(o), stats, _stream(stream))
        self._raise(st, "fr_solve_levels", allow=(FR_ENOCONV, FR_EDIVERGED))
        return st, list(stats)

    def tsc(self, pos, out, stream=None):
        """TSC density of particles pos [np, 3] into out [n2, n1, n0]."""
        st = self.lib.fr_tsc_assign(self._h, _ptr(pos), int(pos.shape[0]), _dims(out.shape),
                                    _ptr(out), _stream(stream))
        self._raise(st, "fr_tsc_assign")

    def forces(self, phi, pos, out, scheme="tsc", stream=None):
        """-grad Phi at the particles (same-scheme interpolation) into out [np, 3]."""
        sc = {"cic": 0, "tsc": 1}[scheme]
        st = self.lib.fr_particle_forces(self._h, _ptr(phi), _dims(phi.shape), _ptr(pos),
                                         int(pos.shape[0]), sc, _ptr(out), _stream(stream))
        self._raise(st, "fr_particle_forces")

    def cic(self, pos, out, stream=None):
        st = self.lib.fr_cic_assign(self._h, _ptr(pos), int(pos.shape[0]), _dims(out.shape),
                                    _ptr(out), _stream(stream))
        self._raise(st, "fr_cic_assign")

    def smooth(self, u, density, nsweeps, *, box, a, omega_m, fr0, h=None, f=None, ub=None,
               cap=1.0, stream=None):
        h = 1.0 / u.shape[2] if h is None else h
        st = self.lib.fr_smooth(self._h, _ptr(u), _ptr(density), _ptr(f), _dims(u.shape), h, box,
                                a, omega_m, fr0, _ptr(ub), nsweeps, cap, _stream(stream))
        self._raise(st, "fr_smooth")

    def smooth_f32(self, u, nsweeps, *, box, a, omega_m, fr0, h=None, bg=None, f=None, ub=None,
                   cap=1.0, tiled=True, stream=None):
        h = 1.0 / u.shape[2] if h is None else h
        st = self.lib.fr_smooth_f32(self._h, _ptr(u), _ptr(bg), _ptr(f), _dims(u.shape), h, box,
                                    a, omega_m, fr0, _ptr(ub), nsweeps, cap, int(tiled),
                                    _stream(stream))
        self._raise(st, "fr_smooth_f32")

    def residual(self, u, density, d, *, box, a, omega_m, fr0, h=None, f=None, ub=None,
                 stream=None):
        h = 1.0 / u.shape[2] if h is None else h
        st = self.lib.fr_residual(self._h, _ptr(u), _ptr(density), _ptr(f), _dims(u.shape), h,
                                  box, a, omega_m, fr0, _ptr(ub), _ptr(d), _stream(stream))
        self._raise(st, "fr_residual")

    def residual_df(self, u, density, d, *, box, a, omega_m, fr0, h=None, ub=None, stream=None):
        h = 1.0 / u.shape[2] if h is None else h
        st = self.lib.fr_residual_df(self._h, _ptr(u), _ptr(density), _dims(u.shape), h, box, a,
                                     omega_m, fr0, _ptr(ub), _ptr(d), _stream(stream))
        self._raise(st, "fr_residual_df")

    def restrict(self, fine, coarse, stream=None):
        st = self.lib.fr_restrict(self._h, _ptr(fine), _dims(fine.shape), _ptr(coarse),
                                  _stream(stream))
        self._raise(st, "fr_restrict")

    def prolong_correct(self, uf, uH, uR, dirichlet=False, stream=None):
        st = self.lib.fr_prolong_correct(self._h, _ptr(uf), _dims(uf.shape), _ptr(uH), _ptr(uR),
                                         int(dirichlet), _stream(stream))
        self._raise(st, "fr_prolong_correct")

    def patch_bc(self, uparent, origin, u_init, ub, periodic=True, stream=None):
        org = (ctypes.c_int * 3)(*origin)
        st = self.lib.fr_patch_bc(self._h, _ptr(uparent), _dims(uparent.shape), int(periodic),
                                  org, _dims(u_init.shape), _ptr(u_init), _ptr(ub),
                                  _stream(stream))
        self._raise(st, "fr_patch_bc")
