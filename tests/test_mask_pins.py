"""Pins of the masked-region oracle (general mask scheme, Sec. V, V.A.1, V.B.1,
V.B.2, V.A.3) to things other than itself: the independently written patch and
periodic operators of the C oracle in the two special cases the paper names,
a finite-difference derivative, the homogeneous solution, brute-force Newton
on a small irregular region, and second-order convergence to the closed-form
spherical Gaussian (Sec. VI.B.1's field) on a spherical region."""
import numpy as np
import pytest

import paper_fields as PF
from oracle import masked as M
from oracle import oracle as O

P = dict(box=128.0, a=0.9, omega_m=0.24, fr0=1e-5)


def _box_mask(shape):
    m = -np.ones(shape)
    m[1:-1, 1:-1, 1:-1] = 1.0
    return m


def _faces(u):
    """Packed u_b = (ghost + first interior)/2 of the interior block of u."""
    mid = lambda a, b: 0.5 * (a + b)
    I = (slice(1, -1),) * 3
    fx0 = mid(u[1:-1, 1:-1, 0], u[1:-1, 1:-1, 1])
    fx1 = mid(u[1:-1, 1:-1, -1], u[1:-1, 1:-1, -2])
    fy0 = mid(u[1:-1, 0, 1:-1], u[1:-1, 1, 1:-1])
    fy1 = mid(u[1:-1, -1, 1:-1], u[1:-1, -2, 1:-1])
    fz0 = mid(u[0, 1:-1, 1:-1], u[1, 1:-1, 1:-1])
    fz1 = mid(u[-1, 1:-1, 1:-1], u[-2, 1:-1, 1:-1])
    assert u[I].shape[0] == fx0.shape[0]
    return np.concatenate([f.ravel() for f in (fx0, fx1, fy0, fy1, fz0, fz1)])


def _irregular_mask(shape, seed, frac=0.6):
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1.0, 1.0, shape)
    m = np.where(rng.uniform(size=shape) < frac, np.abs(m) + 0.05, -np.abs(m))
    m = np.clip(m, -1.0, 1.0)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = -1, -1, -1, -1, -1, -1
    return m


def test_box_mask_is_the_patch_operator():
    """Masks +1 inside, -1 on the outer layer: r = -1 on every ghost face and
    u_b = (u_g + u_i)/2, which is the refinement-patch operator (Eq.
    bc_modified_fR_op with r = -1) of the C oracle."""
    shape = (10, 12, 14)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1.0, 0.5, shape)
    rho = np.exp(rng.normal(0, 0.7, shape))
    h = 1.0 / 64
    Lm, dLm = M.operator(u, _box_mask(shape), rho, h=h, **P)
    I = (slice(1, -1),) * 3
    ref = O.residual(u[I], rho[I], h=h, ub=_faces(u), **P)
    assert np.abs(Lm[I] - ref).max() <= 1e-10 * np.abs(ref).max()
    # derivative against the C oracle's cell by cell
    for (k, j, i) in [(0, 0, 0), (3, 4, 5), (7, 9, 11), (0, 5, 11)]:
        _, dref = O.cell_op(u[I], rho[I], i, j, k, h=h, ub=_faces(u), **P)
        assert dLm[1 + k, 1 + j, 1 + i] == pytest.approx(dref, rel=1e-12)


def test_zero_ghost_mask_is_the_unmodified_operator():
    """Ghost masks 0: r = 0 and u_b = u_g, so the equation reduces to the
    regular grid's (the paper's remark after Eq. bc_modified_fR_dop): the C
    oracle's periodic operator on the whole box agrees at every active cell."""
    shape = (8, 10, 12)
    rng = np.random.default_rng(2)
    u = rng.uniform(-1.0, 0.5, shape)
    rho = np.exp(rng.normal(0, 0.7, shape))
    m = np.zeros(shape)
    m[1:-1, 1:-1, 1:-1] = rng.uniform(0.1, 1.0, (6, 8, 10))
    h = 1.0 / 32
    Lm, _ = M.operator(u, m, rho, h=h, **P)
    ref = O.residual(u, rho, h=h, **P)
    I = (slice(1, -1),) * 3
    assert np.abs(Lm[I] - ref[I]).max() <= 1e-10 * np.abs(ref[I]).max()


def test_derivative_matches_finite_differences_for_any_ratio():
    """Eq. bc_modified_fR_dop with general r = m_g/m_i: central differences of
    L_i in u_i (u_b fixed by the initial values)."""
    shape = (8, 8, 8)
    rng = np.random.default_rng(3)
    m = _irregular_mask(shape, 4)
    u0 = rng.uniform(-1.0, 0.5, shape)
    rho = np.exp(rng.normal(0, 0.7, shape))
    h = 1.0 / 32
    _, dL = M.operator(u0, m, rho, h=h, **P)
    act = np.argwhere(m > 0)
    assert len(act) > 20
    eps = 1e-6
    for k, j, i in act[:: max(1, len(act) // 25)]:
        up, um = u0.copy(), u0.copy()
        up[k, j, i] += eps
        um[k, j, i] -= eps
        Lp, _ = M.operator(up, m, rho, h=h, u_init=u0, **P)
        Lmn, _ = M.operator(um, m, rho, h=h, u_init=u0, **P)
        fd = (Lp[k, j, i] - Lmn[k, j, i]) / (2 * eps)
        assert dL[k, j, i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * abs(fd) + 1e-3)


def test_homogeneous_state_is_exact_for_any_mask():
    shape = (10, 10, 10)
    m = _irregular_mask(shape, 5)
    u = np.zeros(shape)
    rho = np.ones(shape)
    Lm, _ = M.operator(u, m, rho, h=1.0 / 40, **P)
    _, beta, gamma = PF.coefficients(P["box"], 40, P["a"], P["omega_m"], P["fr0"])
    assert np.abs(Lm).max() <= 1e-12 * (beta + gamma)


def test_multigrid_equals_brute_force_newton():
    """FAS V-cycles with masked levels reach the solution of dense Newton on the
    active cells of an irregular region (mask values in (-1, 1), several
    ghost ratios)."""
    shape = (16, 16, 16)
    rng = np.random.default_rng(6)
    k, j, i = np.indices(shape)
    r2 = ((i - 7.5) ** 2 + (j - 7.5) ** 2 + (k - 7.5) ** 2) / 25.0
    blob = np.exp(-r2) + 0.3 * rng.uniform(-1, 1, shape)
    m = np.clip(2.0 * blob - 0.4, -1.0, 1.0)
    m[[0, -1]], m[:, [0, -1]], m[:, :, [0, -1]] = -1.0, -1.0, -1.0
    assert (m > 0).sum() > 100 and M.num_levels(m) >= 2
    u0 = 0.2 * np.sin(0.4 * i) * np.cos(0.3 * j) + 0.1 * np.cos(0.5 * k)
    rho = np.exp(rng.normal(0, 0.5, shape))
    h = 1.0 / 64
    res = M.solve(u0, m, rho, h=h, tol=1e-11, **P)
    assert res.converged and res.cycles >= 2
    ref = M.dense_newton(u0, m, rho, h=h, **P)
    act = m > 0
    assert np.abs(res.u[act] - ref[act]).max() < 1e-9
    assert np.abs(res.u[~act] - u0[~act]).max() < 1e-14  # ghost values are never changed


def test_spherical_region_converges_at_second_order():
    """Sec. VI.B.1's spherical Gaussian (3D analogue of Eq. gaussian_dens) on a
    spherical active region whose ghosts hold the closed form: the error at the
    active cells falls about fourfold when h halves."""
    G = dict(amp=0.9, width=0.08, centre=(0.5, 0.5, 0.5))
    errs = []
    for N, nb in ((64, 24), (128, 48)):
        lo = N // 2 - nb // 2
        rho, ue = PF.spherical_gaussian_patch(lo, nb, N, **P, **G)
        x = (np.arange(lo, lo + nb) + 0.5) / N
        z, y, xx = np.meshgrid(x, x, x, indexing="ij")
        rr = np.sqrt((xx - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        m = np.where(rr < 0.15, 1.0, -1.0)
        res = M.solve(ue, m, rho, h=1.0 / N, tol=1e-10, **P)
        assert res.converged
        errs.append(np.abs(res.u - ue)[m > 0].max())
    assert errs[0] / errs[1] > 3.0


def test_masked_transfers_by_brute_force():
    """Masked transfers (Sec. V.A.2, V.A.3) against loops written from their
    definitions: R d = (sum of the active children's d) / 8; the prolonged
    correction at an active fine cell is the 27/9/3/1 / 64 combination of its
    parent and the parent's neighbours on the child's side (a masked coarse
    cell, carrying e = 0, and a cell outside the box contribute 0), and 0 at a
    masked fine cell.  A coarse correction linear in position is reproduced
    exactly at fine cells whose 8 interpolation parents lie in the box."""
    rng = np.random.default_rng(5)
    cs = (3, 4, 5)
    fs = tuple(2 * c for c in cs)
    d = rng.normal(size=fs)
    act = rng.uniform(size=fs) < 0.6
    R = M.restrict_active(d, act)
    for K in range(cs[0]):
        for J in range(cs[1]):
            for I in range(cs[2]):
                s = sum(d[2 * K + z, 2 * J + y, 2 * I + x]
                        for z in (0, 1) for y in (0, 1) for x in (0, 1)
                        if act[2 * K + z, 2 * J + y, 2 * I + x])
                assert R[K, J, I] == pytest.approx(s / 8.0, abs=1e-15)

    e = rng.normal(size=cs)
    e[rng.uniform(size=cs) < 0.3] = 0.0                 # masked coarse cells
    out = M.prolong_masked(e, act)

    def ec(K, J, I):
        inside = 0 <= K < cs[0] and 0 <= J < cs[1] and 0 <= I < cs[2]
        return e[K, J, I] if inside else 0.0

    for k in range(fs[0]):
        for j in range(fs[1]):
            for i in range(fs[2]):
                if not act[k, j, i]:
                    assert out[k, j, i] == 0.0
                    continue
                K, J, I = k // 2, j // 2, i // 2
                sk, sj, si = (1 if k % 2 else -1), (1 if j % 2 else -1), (1 if i % 2 else -1)
                v = 0.0
                for oz, wz in ((0, 3), (sk, 1)):
                    for oy, wy in ((0, 3), (sj, 1)):
                        for ox, wx in ((0, 3), (si, 1)):
                            v += wz * wy * wx * ec(K + oz, J + oy, I + ox)
                assert out[k, j, i] == pytest.approx(v / 64.0, abs=1e-14)

    # exact for a linear correction (coordinates in fine cell widths, cell centres)
    Kc, Jc, Ic = np.indices(cs).astype(float)
    lin = lambda z, y, x: 0.3 - 0.7 * z + 1.1 * y + 0.45 * x
    eL = lin(2 * Kc + 1, 2 * Jc + 1, 2 * Ic + 1)
    outL = M.prolong_masked(eL, np.ones(fs, dtype=bool))
    kf, jf, if_ = np.indices(fs).astype(float)
    want = lin(kf + 0.5, jf + 0.5, if_ + 0.5)
    inner = (slice(1, -1),) * 3
    assert np.abs(outL[inner] - want[inner]).max() < 1e-13


def test_ghost_relation_returns_the_ghost_value():
    """u_b from Eq. u_i-1jk solved for it: put back into u_g = u_b - r u_b +
    r u_i (r = m_g / m_i) it returns the initial ghost value on every ghost face
    of an active cell, for any mask ratio."""
    shape = (6, 7, 8)
    m = _irregular_mask(shape, 9)
    rng = np.random.default_rng(4)
    ut = rng.normal(size=shape)
    ub = M.boundary_values(ut, m)
    act = m > 0
    n = 0
    for f, (ax, st) in enumerate(M.FACES):
        ug = np.roll(ut, -st, axis=ax)
        mg = np.roll(m, -st, axis=ax)
        ghost = act & (mg <= 0)
        assert np.array_equal(np.isfinite(ub[f]), ghost)
        r = mg[ghost] / m[ghost]
        back = ub[f][ghost] - r * ub[f][ghost] + r * ut[ghost]
        assert np.abs(back - ug[ghost]).max() < 1e-12
        n += int(ghost.sum())
    assert n > 0


def test_level_count_rule_by_hand():
    """Masked level rule (reading of Sec. V.A.2: halve while every size stays
    even and the halved size is >= 4, the coarser mask, the mean of the 8
    children, keeps its outer layer masked and has an active cell), on cases
    counted by hand."""
    def block(n, lo, hi):
        m = -np.ones((n, n, n))
        m[lo:hi, lo:hi, lo:hi] = 1.0
        return m
    # 12^3 with the central 4^3 active: 12 -> 6 (6^3 has the central 2^3
    # active); halving 6 would give 3 < 4
    assert M.num_levels(block(12, 4, 8)) == 2
    # 16^3 with a 2-cell masked margin: 16 -> 8 -> 4 (4^3: faces average to 0)
    assert M.num_levels(block(16, 2, 14)) == 3
    # 16^3 with a 1-cell margin: the 4^3 level would have active outer cells
    assert M.num_levels(block(16, 1, 15)) == 2
    # 10 -> 5 and 14 -> 7 (odd sizes end the series); 6 would halve to 3 < 4
    assert M.num_levels(block(10, 1, 9)) == 2 and M.num_levels(block(14, 1, 13)) == 2
    assert M.num_levels(block(6, 1, 5)) == 1


def test_coarse_ghosts_keep_their_initial_values():
    """On every coarse level the ghost cells (mask <= 0) hold the restriction of
    the initial fine values for the whole solve (reading of Sec. V.B.2 for
    masked levels): a V-cycle changes only active coarse cells."""
    shape = (16, 16, 16)
    rng = np.random.default_rng(8)
    k, j, i = np.indices(shape)
    r2 = ((i - 7.5) ** 2 + (j - 7.5) ** 2 + (k - 7.5) ** 2) / 20.0
    m = np.clip(2.0 * np.exp(-r2) - 0.3, -1.0, 1.0)
    m[[0, -1]], m[:, [0, -1]], m[:, :, [0, -1]] = -1.0, -1.0, -1.0
    from oracle import oracle as _O
    model = _O.Model(P["box"], 1, P["a"], P["omega_m"], P["fr0"])
    u0 = 0.3 * np.sin(0.4 * i) + 0.2 * rng.uniform(-1, 1, shape) + model.ubar
    rho = np.exp(rng.normal(0, 0.5, shape))
    H = M.Hierarchy(u0, m, rho, 1.0 / 64, model)
    assert len(H.lev) >= 2
    before = [L.u.copy() for L in H.lev]
    for _ in range(2):
        M.vcycle(H, 0, 2, 2, 1e-10)
    for L, b in zip(H.lev, before):
        assert np.array_equal(L.u[~L.act], b[~L.act])
    assert not np.array_equal(H.lev[1].u[H.lev[1].act], before[1][H.lev[1].act])


def test_hierarchy_masks_cell_sizes_and_sweep_by_hand():
    """Masked levels (reading of Sec. V.A.2): each coarse mask, density and
    initial u is the mean of the 8 children (written out as loops), and the
    cell size doubles per level.  One vectorised Newton-Gauss-Seidel sweep
    equals the sweep written cell by cell over the active cells, red
    ((i + j + k) even) in index order first, then black."""
    from oracle import oracle as _O
    shape = (8, 12, 16)
    rng = np.random.default_rng(14)
    m = _irregular_mask(shape, 15, frac=0.7)
    model = _O.Model(P["box"], 1, P["a"], P["omega_m"], P["fr0"])
    u0 = 0.2 * rng.standard_normal(shape) + model.ubar
    rho = np.exp(rng.normal(0, 0.5, shape))
    H = M.Hierarchy(u0, m, rho, 1.0 / 64, model, nlevels=2)
    F, C = H.lev
    assert C.h == 2 * F.h and C.pre == pytest.approx(F.pre / 4, rel=1e-15)
    for K in range(shape[0] // 2):
        for J in range(shape[1] // 2):
            for I in range(shape[2] // 2):
                blk = (slice(2 * K, 2 * K + 2), slice(2 * J, 2 * J + 2), slice(2 * I, 2 * I + 2))
                assert C.m[K, J, I] == pytest.approx(m[blk].sum() / 8, abs=1e-15)
                assert C.rho[K, J, I] == pytest.approx(rho[blk].sum() / 8, rel=1e-14)
                assert C.u[K, J, I] == pytest.approx(u0[blk].sum() / 8, rel=1e-14)
    # the sweep, cell by cell
    F.f = 1e-3 * rng.standard_normal(shape)
    ref = F.u.copy()
    n2, n1, n0 = shape
    for colour in (0, 1):
        for k in range(n2):
            for j in range(n1):
                for i in range(n0):
                    if (i + j + k) % 2 != colour or not F.act[k, j, i]:
                        continue
                    F.u, keep = ref, F.u
                    Lv, dL = M.cell_terms(F, model)
                    F.u = keep
                    du = -(Lv[k, j, i] - F.f[k, j, i]) / dL[k, j, i]
                    ref[k, j, i] += min(max(du, -1.0), 1.0)
    M.ngs_sweep(F, model)
    assert np.abs(F.u - ref).max() < 1e-13
