"""Plain FP64 CPU oracle of the general mask scheme for refinement boundaries.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and by the CPU-baseline leg
of ``bench.py``).  The GPU library never imports it.

Li, Zhao, Teyssier & Koyama (arXiv:1110.1379), Sec. V (the mask scheme taken
over from RAMSES), Sec. V.A.1 (Eq. phi_b), Sec. V.B.1 (Eqs. u_i-1jk,
bc_modified_fR_op, bc_modified_fR_dop), Sec. V.A.2 and V.B.2 (masked
restriction, coarse masks and boundary values), Sec. V.A.3 (masked
prolongation).  A refinement region is a box grid of cells with a mask value
m in [-1, 1] per cell: cells with m > 0 are active (relaxed), the others are
ghosts whose values are fixed (interpolated from the parent level in an AMR
code).  Every cell of the box's outer layer must be a ghost.

* Ghost relation (Eq. u_i-1jk) across the face between an active cell i and a
  ghost g, with r = m_g / m_i:  u_g = u_b - r u_b + r u_i,  b_g = exp(u_g);
  u_b is fixed for the solve, computed from the initial values by solving the
  same relation for it:  u_b = (m_i u_g - m_g u_i) / (m_i - m_g).
* Operator: the flux form (e^{u_i} + e^{u_j})(u_j - u_i) of Eq. discrete_fR
  times c~^2 / (2 h^2), the ghost face entering with u_g and b_g above; summed
  over the faces this is Eq. bc_modified_fR_op for any number of ghost faces,
  and its derivative in u_i is Eq. bc_modified_fR_dop.
* Multigrid (FAS, Sec. V.B.2): coarse masks are the mean of the 8 children;
  R u^h is the mean of all 8 children (masked children included); R d^h is the
  sum over the active children divided by 8 (a masked fine cell contributes
  nothing); coarse ghosts keep fixed values, the restriction of the initial
  fine values, and their u_b follow from those as on the finest level; the
  prolonged correction reaches active fine cells only and a masked coarse cell
  contributes zero to it.  Levels halve while every size stays even and >= 4,
  the next level keeps its outer layer masked and has an active cell.

Values in and out are the shifted variable u = ln(f_R / fbar_R) of ``oracle.py``;
the arithmetic is in the paper's u~ = u + ubar.  Vectorised over one colour of
the red-black ordering at a time (cells of one colour do not couple).

Pins (tests/test_mask_pins.py; no function here is unpinned): cell_terms and
boundary_values by test_box_mask_is_the_patch_operator,
test_zero_ghost_mask_is_the_unmodified_operator,
test_derivative_matches_finite_differences_for_any_ratio,
test_homogeneous_state_is_exact_for_any_mask and
test_ghost_relation_returns_the_ghost_value; restrict_active and
prolong_masked by test_masked_transfers_by_brute_force; num_levels, the
hierarchy and ngs_sweep by test_level_count_rule_by_hand and
test_hierarchy_masks_cell_sizes_and_sweep_by_hand; vcycle and solve by
test_coarse_ghosts_keep_their_initial_values,
test_multigrid_equals_brute_force_newton and
test_spherical_region_converges_at_second_order.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _orc

# the six faces as (numpy axis, step): -x, +x, -y, +y, -z, +z
FACES = ((2, -1), (2, 1), (1, -1), (1, 1), (0, -1), (0, 1))


def _nb(a, ax, step):
    """Neighbour value across a face (wraps at the box edge; only read for
    active cells, which never touch the edge)."""
    return np.roll(a, -step, axis=ax)


class MLevel:
    """One level of a masked region: u~ everywhere (iterate in active cells,
    fixed ghost values elsewhere), masks, density, right-hand side, and the
    fixed boundary values u_b of every ghost face (NaN elsewhere)."""

    def __init__(self, ut, m, rho, h, model):
        self.u = np.array(ut, dtype=np.float64)
        self.m = np.array(m, dtype=np.float64)
        self.act = self.m > 0
        self.rho = np.array(rho, dtype=np.float64)
        self.f = np.zeros_like(self.u)
        self.h = h
        self.pre = model.ctilde ** 2 / (2.0 * h * h)
        self.ub = boundary_values(self.u, self.m)

    @property
    def shape(self):
        return self.u.shape


def check_region(m):
    m = np.asarray(m)
    edge = np.ones(m.shape, dtype=bool)
    edge[1:-1, 1:-1, 1:-1] = False
    if np.any(m[edge] > 0):
        raise ValueError("the outer layer of a masked region must be masked (m <= 0)")
    if np.any(m > 1) or np.any(m < -1):
        raise ValueError("mask values must lie in [-1, 1]")


def boundary_values(ut, m):
    """u_b of the ghost faces: (m_i u_g - m_g u_i) / (m_i - m_g) (Eq. u_i-1jk
    solved for u_b) on faces from an active cell i to a ghost g; NaN elsewhere."""
    out = []
    act = m > 0
    for ax, st in FACES:
        ug, mg = _nb(ut, ax, st), _nb(m, ax, st)
        ghost = act & (mg <= 0)
        with np.errstate(invalid="ignore", divide="ignore"):
            ub = (m * ug - mg * ut) / (m - mg)
        out.append(np.where(ghost, ub, np.nan))
    return out


def cell_terms(L, model):
    """(L(u), dL/du) of Eq. bc_modified_fR_op / bc_modified_fR_dop at every
    active cell (0 at ghosts).  Density term uses rho~ as in Eq. discrete_fR."""
    ui = L.u
    bi = np.exp(ui)
    flux = np.zeros_like(ui)
    dflux = np.zeros_like(ui)
    for f, (ax, st) in enumerate(FACES):
        uj, mj = _nb(L.u, ax, st), _nb(L.m, ax, st)
        reg = mj > 0
        bj = np.exp(uj)
        t_reg = (bi + bj) * (uj - ui)
        d_reg = bi * (uj - ui) - (bi + bj)
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            r = np.where(L.act, mj / np.where(L.act, L.m, 1.0), 0.0)
            ub = np.nan_to_num(L.ub[f])
            ug = ub - r * ub + r * ui
            bg = np.exp(ug)
            t_gh = (bi + bg) * (ug - ui)
            d_gh = (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0)
        flux += np.where(reg, t_reg, t_gh)
        dflux += np.where(reg, d_reg, d_gh)
    s = np.exp(-ui / 2.0)  # n = 1
    Lv = L.pre * flux - model.dens * (L.rho - 1.0) + model.src * s - model.bkg
    dL = L.pre * dflux - model.src * s / 2.0
    return np.where(L.act, Lv, 0.0), np.where(L.act, dL, 1.0)


def residual_t(L, model):
    """d = L(u) - f on active cells, 0 on ghosts."""
    Lv, _ = cell_terms(L, model)
    return np.where(L.act, Lv - L.f, 0.0)


def ngs_sweep(L, model, cap=1.0, relax=1.0):
    """Red-black Newton-Gauss-Seidel over the active cells (red: i+j+k even)."""
    k, j, i = np.indices(L.shape)
    par = (i + j + k) & 1
    for colour in (0, 1):
        Lv, dL = cell_terms(L, model)
        du = np.clip(-relax * (Lv - L.f) / dL, -cap, cap)
        sel = L.act & (par == colour)
        L.u = np.where(sel, L.u + du, L.u)


def restrict_mean(a):
    n2, n1, n0 = a.shape
    return a.reshape(n2 // 2, 2, n1 // 2, 2, n0 // 2, 2).mean(axis=(1, 3, 5))


def restrict_active(d, act):
    """Sum over the active children divided by 8 (masked children contribute 0)."""
    return restrict_mean(np.where(act, d, 0.0))


def prolong_masked(e, fine_act):
    """Trilinear 27/9/3/1 interpolation of the coarse correction e (zero on
    masked coarse cells and outside the box) onto the active fine cells."""
    n2, n1, n0 = e.shape
    ep = np.pad(e, 1)
    out = np.zeros((2 * n2, 2 * n1, 2 * n0))
    w = (0.25, 0.75)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                acc = np.zeros((n2, n1, n0))
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            # neighbour offsets -1/+1 on the child's side, 0 for the parent
                            oz = (1 if cz else -1) if dz == 0 else 0
                            oy = (1 if cy else -1) if dy == 0 else 0
                            ox = (1 if cx else -1) if dx == 0 else 0
                            wt = w[dz] * w[dy] * w[dx]
                            acc += wt * ep[1 + oz:1 + oz + n2, 1 + oy:1 + oy + n1,
                                           1 + ox:1 + ox + n0]
                out[cz::2, cy::2, cx::2] = acc
    return np.where(fine_act, out, 0.0)


def _masked_outer(m):
    edge = np.ones(m.shape, dtype=bool)
    edge[1:-1, 1:-1, 1:-1] = False
    return not np.any(m[edge] > 0)


def num_levels(m):
    """Levels of the mask hierarchy (reading: halve while sizes stay even and
    >= 4, the next level's outer layer stays masked and it has an active cell)."""
    m = np.asarray(m, dtype=np.float64)
    nl = 1
    while all(s % 2 == 0 and s // 2 >= 4 for s in m.shape):
        mc = restrict_mean(m)
        if not _masked_outer(mc) or not np.any(mc > 0):
            break
        m = mc
        nl += 1
    return nl


class Hierarchy:
    def __init__(self, ut0, m, rho, h, model, nlevels=None):
        self.model = model
        nl = num_levels(m) if nlevels is None else nlevels
        self.lev = [MLevel(ut0, m, rho, h, model)]
        u0, mm, rr, hh = np.asarray(ut0, dtype=np.float64), np.asarray(m, dtype=np.float64), \
            np.asarray(rho, dtype=np.float64), h
        for _ in range(1, nl):
            u0, mm, rr, hh = restrict_mean(u0), restrict_mean(mm), restrict_mean(rr), 2 * hh
            self.lev.append(MLevel(u0, mm, rr, hh, model))


def _rms_active(d, act):
    n = int(act.sum())
    return float(np.sqrt(np.sum(np.where(act, d, 0.0) ** 2) / max(n, 1)))


def _coarsest(H, L, tol, cap, relax):
    r0 = _rms_active(residual_t(L, H.model), L.act)
    thr = max(1e-3 * r0, 0.1 * tol)
    for _ in range(500):
        ngs_sweep(L, H.model, cap, relax)
        if _rms_active(residual_t(L, H.model), L.act) <= thr:
            break


def vcycle(H, l, pre, post, tol, cap=1.0, relax=1.0):
    """One FAS V-cycle from level l (Sec. V.B.2 with the mask rules)."""
    L = H.lev[l]
    if l == len(H.lev) - 1:
        _coarsest(H, L, tol, cap, relax)
        return
    C = H.lev[l + 1]
    for _ in range(pre):
        ngs_sweep(L, H.model, cap, relax)
    d = residual_t(L, H.model)
    uR = np.where(C.act, restrict_mean(L.u), C.u)  # coarse ghosts keep their values
    C.u = uR.copy()
    C.f = np.zeros_like(C.u)
    LH, _ = cell_terms(C, H.model)
    C.f = np.where(C.act, LH - restrict_active(d, L.act), 0.0)
    vcycle(H, l + 1, pre, post, tol, cap, relax)
    e = np.where(C.act, C.u - uR, 0.0)
    L.u = L.u + prolong_masked(e, L.act)
    for _ in range(post):
        ngs_sweep(L, H.model, cap, relax)


class MaskedResult:
    def __init__(self, u, cycles, hist, res_rms, converged):
        self.u, self.cycles, self.hist, self.res_rms = u, cycles, hist, res_rms
        self.converged = converged


def solve(u0, m, rho, *, box, a, omega_m, fr0, h, tol=1e-8, max_cycles=100, pre=2, post=2,
          cap=1.0, ncycles=0, nlevels=None):
    """FAS V-cycles on a masked region until the rms of L(u) over the active
    cells is <= tol (or exactly ``ncycles``).  u0: initial values in active
    cells and the fixed ghost values elsewhere (shifted variable)."""
    check_region(m)
    model = _orc.Model(box, 1, a, omega_m, fr0)
    ut0 = np.asarray(u0, dtype=np.float64) + model.ubar
    H = Hierarchy(ut0, m, rho, h, model, nlevels)
    L0 = H.lev[0]
    res = _rms_active(residual_t(L0, model), L0.act)
    hist = [res]
    cyc = 0
    while (ncycles > 0 and cyc < ncycles) or (ncycles <= 0 and res > tol and cyc < max_cycles):
        vcycle(H, 0, pre, post, tol, cap)
        cyc += 1
        res = _rms_active(residual_t(L0, model), L0.act)
        hist.append(res)
    return MaskedResult(L0.u - model.ubar, cyc, hist, res, res <= tol)


def operator(u, m, rho, *, box, a, omega_m, fr0, h, u_init=None):
    """(L, dL/du) at every active cell of the finest level, with the boundary
    values u_b computed from ``u_init`` (default: u itself)."""
    check_region(m)
    model = _orc.Model(box, 1, a, omega_m, fr0)
    ut = np.asarray(u, dtype=np.float64) + model.ubar
    ut0 = ut if u_init is None else np.asarray(u_init, dtype=np.float64) + model.ubar
    L = MLevel(ut0, m, rho, h, model)
    L.u = ut
    return cell_terms(L, model)


def dense_newton(u0, m, rho, *, box, a, omega_m, fr0, h, tol=1e-13, max_iter=60):
    """Brute-force solve of L(u) = 0 on the active cells of a small masked
    region: Newton's method with the full Jacobian and ``numpy.linalg.solve``;
    shares only the operator evaluation with the multigrid path.  The Jacobian
    is assembled from central differences of the operator, perturbing at once
    all active cells of one class c = (i + 2j + 3k) mod 7 (no two cells of a
    class lie in one 7-point stencil, so each entry is recovered exactly once)."""
    check_region(m)
    model = _orc.Model(box, 1, a, omega_m, fr0)
    ut0 = np.asarray(u0, dtype=np.float64) + model.ubar
    L = MLevel(ut0, m, rho, h, model)
    shape = L.shape
    idx = np.flatnonzero(L.act)
    col = {int(c): n for n, c in enumerate(idx)}
    kk, jj, ii = np.unravel_index(idx, shape)
    cls = (ii + 2 * jj + 3 * kk) % 7
    offs = [(0, 0, 0)] + [(dz, dy, dx) for dz, dy, dx in
                          ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0))]
    eps = 1e-6
    for _ in range(max_iter):
        F = cell_terms(L, model)[0].ravel()[idx]
        if np.sqrt(np.mean(F ** 2)) <= tol:
            break
        J = np.zeros((idx.size, idx.size))
        base = L.u.copy()
        for c in range(7):
            pert = idx[cls == c]
            up = base.copy()
            up.ravel()[pert] += eps
            L.u = up
            Fp = cell_terms(L, model)[0].ravel()[idx]
            um = base.copy()
            um.ravel()[pert] -= eps
            L.u = um
            Fm = cell_terms(L, model)[0].ravel()[idx]
            D = (Fp - Fm) / (2 * eps)
            for row in range(idx.size):
                for dz, dy, dx in offs:
                    z, y, x = kk[row] + dz, jj[row] + dy, ii[row] + dx
                    if (x + 2 * y + 3 * z) % 7 != c:
                        continue
                    q = col.get(int(np.ravel_multi_index((z, y, x), shape)))
                    if q is not None:
                        J[row, q] = D[row]
        L.u = base
        du = np.linalg.solve(J, -F)
        L.u.ravel()[idx] += du
    return L.u - model.ubar
