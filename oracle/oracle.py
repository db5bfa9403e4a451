"""Python access to the plain FP64 CPU oracle (``fr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The GPU library never imports it.

Everything here follows Li, Zhao, Teyssier & Koyama (arXiv:1110.1379):
the operator of Eq. (bc_modified_fR_op), its derivative Eq. (bc_modified_fR_dop),
red-black Newton-Gauss-Seidel, FAS V-cycles (Sec. V.B.2), trilinear
prolongation (Sec. V.A.3), ghost/boundary values of refinement patches
(Sec. V.A.1, V.B.1) and CIC assignment (Sec. VI.C).  Values in and out are the
shifted variable u = ln(f_R / fbar_R); the C code works in the paper's
u~ = ln(-a^2 f_R) internally.

``dense_newton`` is an independent brute force (Sec. V.B.1's Newton step on the
whole grid at once): it solves L(u) = 0 with the full Jacobian and
``numpy.linalg.solve``; it shares only the residual evaluation with the FAS path.

Pins (tests/test_oracle_pins.py; the C functions' pins are listed in
fr_oracle.c): truncation_error by test_truncation_error_vanishes_on_homogeneous_solution
and test_truncation_error_is_second_order; solve_levels by
test_two_level_gaussian_patch and test_three_level_gaussian_patch; dense_newton
by test_dense_newton_matches_fas_periodic / _patch (two independent routes to
the same root).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOCONV = 0, 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.orc_model.argtypes = [D, I, D, D, D, P]
            lib.orc_residual.argtypes = [P, P, P, P, D, D, D, D, D, P, P]
            lib.orc_cell_op.argtypes = [P, P, P, D, D, D, D, D, P, I, I, I, P]
            lib.orc_smooth.argtypes = [P, P, P, P, D, D, D, D, D, P, I, D]
            lib.orc_restrict.argtypes = [P, P, P]
            lib.orc_restrict_faces.argtypes = [P, P, P]
            lib.orc_prolong_correct.argtypes = [P, P, P, P, I]
            lib.orc_num_levels.argtypes = [P]
            lib.orc_solve_grid.argtypes = [P, P, D, D, D, D, D, P, D, I, I, I, D, I, P, P, P, P]
            lib.orc_patch_bc.argtypes = [P, P, I, P, P, P, P]
            lib.orc_cic.argtypes = [P, ctypes.c_long, P, P]
            for name in ("orc_model", "orc_residual", "orc_cell_op", "orc_smooth",
                         "orc_restrict", "orc_restrict_faces", "orc_prolong_correct",
                         "orc_num_levels",
                         "orc_solve_grid", "orc_patch_bc", "orc_cic"):
                getattr(lib, name).restype = I
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(shape):
    """numpy shape (n2, n1, n0) -> C int[3] (n0, n1, n2)."""
    return np.array([shape[2], shape[1], shape[0]], dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st not in (OK, ENOCONV):
        raise ValueError(f"oracle {what} failed with status {st}")


class Model:
    """Model constants as the oracle derives them from the paper's formulas."""

    def __init__(self, box, n0, a, omega_m, fr0):
        out = np.zeros(7)
        _check(_load().orc_model(box, n0, a, omega_m, fr0, _p(out)), "model")
        (self.ctilde, self.xi, self.ubar, self.src, self.bkg, self.dens,
         self.pre) = out.tolist()


def face_sizes(shape):
    """Sizes of the six packed faces (-x,+x,-y,+y,-z,+z) of a (n2,n1,n0) grid."""
    n0, n1, n2 = shape[2], shape[1], shape[0]
    return [n1 * n2, n1 * n2, n0 * n2, n0 * n2, n0 * n1, n0 * n1]


def residual(u, rho, *, box, a, omega_m, fr0, h=None, f=None, ub=None):
    u, rho, f, ub = _f64(u), _f64(rho), _f64(f), _f64(ub)
    h = 1.0 / u.shape[2] if h is None else h
    d = np.empty_like(u)
    _check(_load().orc_residual(_p(u), _p(rho), _p(f), _p(_dims(u.shape)), h, box, a,
                                omega_m, fr0, _p(ub), _p(d)), "residual")
    return d


def cell_op(u, rho, i, j, k, *, box, a, omega_m, fr0, h=None, ub=None):
    """(L, dL/du) at cell (x=i, y=j, z=k)."""
    u, rho, ub = _f64(u), _f64(rho), _f64(ub)
    h = 1.0 / u.shape[2] if h is None else h
    out = np.zeros(2)
    _check(_load().orc_cell_op(_p(u), _p(rho), _p(_dims(u.shape)), h, box, a, omega_m, fr0,
                               _p(ub), i, j, k, _p(out)), "cell_op")
    return float(out[0]), float(out[1])


def smooth(u, rho, nsweeps, *, box, a, omega_m, fr0, h=None, f=None, ub=None, cap=1.0):
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    rho, f, ub = _f64(rho), _f64(f), _f64(ub)
    h = 1.0 / u.shape[2] if h is None else h
    _check(_load().orc_smooth(_p(u), _p(rho), _p(f), _p(_dims(u.shape)), h, box, a, omega_m,
                              fr0, _p(ub), nsweeps, cap), "smooth")
    return u


def restrict(fine):
    fine = _f64(fine)
    out = np.empty((fine.shape[0] // 2, fine.shape[1] // 2, fine.shape[2] // 2))
    _check(_load().orc_restrict(_p(fine), _p(_dims(fine.shape)), _p(out)), "restrict")
    return out


def restrict_faces(ub, shape):
    """Boundary-face values of the grid of half the size of `shape` (n2, n1, n0)
    from the packed faces ub of `shape`: each coarse face value is the mean of
    the 4 fine face values covering it (the reading of Sec. V.B.2 used for the
    coarse levels of a patch)."""
    ub = _f64(ub)
    cs = (shape[0] // 2, shape[1] // 2, shape[2] // 2)
    out = np.empty(sum(face_sizes(cs)))
    _check(_load().orc_restrict_faces(_p(ub), _p(_dims(shape)), _p(out)), "restrict_faces")
    return out


def truncation_error(u, rho, *, box, a, omega_m, fr0, h=None):
    """Truncation-error estimate of Sec. V.B.2 on the coarser grid of a periodic grid:
    tau^h = L^H(R u) - R L^h(u), with L^H at cell size 2h and density R rho."""
    u = _f64(u)
    rho = _f64(rho)
    h = 1.0 / u.shape[2] if h is None else h
    P = dict(box=box, a=a, omega_m=omega_m, fr0=fr0)
    return (residual(restrict(u), restrict(rho), h=2.0 * h, **P)
            - restrict(residual(u, rho, h=h, **P)))


def prolong_correct(uf, uH, uR, dirichlet=False):
    uf = np.array(uf, dtype=np.float64, copy=True, order="C")
    _check(_load().orc_prolong_correct(_p(uf), _p(_dims(uf.shape)), _p(_f64(uH)),
                                       _p(_f64(uR)), int(dirichlet)), "prolong")
    return uf


def num_levels(shape):
    return int(_load().orc_num_levels(_p(_dims(shape))))


class SolveResult:
    def __init__(self, u, cycles, hist, status, res_rms):
        self.u = u
        self.cycles = cycles
        self.hist = hist
        self.status = status
        self.res_rms = res_rms
        self.converged = status == OK


def solve(rho, *, box, a, omega_m, fr0, tol=1e-8, max_cycles=100, pre=2, post=2, cap=1.0,
          u0=None, h=None, ub=None, ncycles=0):
    """FAS V-cycles on one grid until rms(L(u)) <= tol (or exactly ``ncycles``)."""
    rho = _f64(rho)
    u = np.zeros_like(rho) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    h = 1.0 / rho.shape[2] if h is None else h
    nh = max(max_cycles, ncycles) + 1
    hist = np.full(nh, np.nan)
    cyc = ctypes.c_int(0)
    res = np.zeros(1)
    st = _load().orc_solve_grid(_p(rho), _p(_dims(rho.shape)), h, box, a, omega_m, fr0,
                                _p(_f64(ub)), tol, max_cycles, pre, post, cap, ncycles, _p(u),
                                ctypes.cast(ctypes.pointer(cyc), ctypes.c_void_p), _p(hist),
                                _p(res))
    _check(st, "solve")
    return SolveResult(u, cyc.value, hist[: (ncycles or cyc.value) + 1], st, float(res[0]))


def patch_bc(uparent, origin, n, *, parent_periodic=True):
    """(initial patch u, packed u_b) for a patch of n=(n2,n1,n0) fine cells at
    parent cell origin=(ox, oy, oz)."""
    up = _f64(uparent)
    ui = np.empty(tuple(n), dtype=np.float64)
    ub = np.empty(sum(face_sizes(n)), dtype=np.float64)
    org = np.array(origin, dtype=np.int32)
    st = _load().orc_patch_bc(_p(up), _p(_dims(up.shape)), int(parent_periodic), _p(org),
                              _p(_dims(n)), _p(ui), _p(ub))
    _check(st, "patch_bc")
    return ui, ub


def cic(pos, shape):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    rho = np.empty(tuple(shape), dtype=np.float64)
    _check(_load().orc_cic(_p(pos), pos.shape[0], _p(_dims(shape)), _p(rho)), "cic")
    return rho


def solve_levels(rho_domain, patches, *, box, a, omega_m, fr0, tol=1e-8, tol_patch=None,
                 max_cycles=100, pre=2, post=2, cap=1.0):
    """Domain grid then refinement patches, one-way coarse to fine (Sec. V, VI.B).

    ``patches``: list of dicts with keys ``parent`` (-1 = domain, else index of
    an earlier patch), ``origin`` (x, y, z parent cells), ``rho`` (n2, n1, n0).
    Returns (domain result, [patch results]).
    """
    tol_patch = tol if tol_patch is None else tol_patch
    dom = solve(rho_domain, box=box, a=a, omega_m=omega_m, fr0=fr0, tol=tol,
                max_cycles=max_cycles, pre=pre, post=post, cap=cap)
    h0 = 1.0 / rho_domain.shape[2]
    out = []
    hs = []
    for p in patches:
        if p["parent"] < 0:
            up, periodic, hp = dom.u, True, h0
        else:
            up, periodic, hp = out[p["parent"]].u, False, hs[p["parent"]]
        u0, ub = patch_bc(up, p["origin"], p["rho"].shape, parent_periodic=periodic)
        r = solve(p["rho"], box=box, a=a, omega_m=omega_m, fr0=fr0, tol=tol_patch,
                  max_cycles=max_cycles, pre=pre, post=post, cap=cap, u0=u0, h=hp / 2.0,
                  ub=ub)
        r.ub = ub
        r.u0 = u0
        out.append(r)
        hs.append(hp / 2.0)
    return dom, out


def dense_newton(rho, *, box, a, omega_m, fr0, h=None, ub=None, cap=1.0, tol=1e-13,
                 max_iter=200, u0=None, fd_eps=1e-7, step_tol=1e-14):
    """Brute force: Newton on the whole grid with a dense Jacobian.

    The Jacobian is formed column by column from central differences of the
    oracle residual; the Newton step is clamped to |du| <= cap per cell, as in
    the smoother.  Stops when max|L(u)| < tol or, once the rounding floor is
    reached, when the Newton step is below ``step_tol``.  Meant for grids of a
    few hundred cells.
    """
    rho = _f64(rho)
    shp = rho.shape
    n = rho.size
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64).ravel().copy()
    kw = dict(box=box, a=a, omega_m=omega_m, fr0=fr0, h=h, ub=ub)
    for it in range(max_iter):
        L = residual(u.reshape(shp), rho, **kw).ravel()
        if np.max(np.abs(L)) < tol:
            return u.reshape(shp), it
        J = np.empty((n, n))
        for c in range(n):
            up = u.copy()
            um = u.copy()
            up[c] += fd_eps
            um[c] -= fd_eps
            J[:, c] = (residual(up.reshape(shp), rho, **kw).ravel()
                       - residual(um.reshape(shp), rho, **kw).ravel()) / (2 * fd_eps)
        du = np.linalg.solve(J, -L)
        du = np.clip(du, -cap, cap)
        u = u + du
        if np.max(np.abs(du)) < step_tol:
            return u.reshape(shp), it + 1
    raise RuntimeError("dense Newton did not converge")
