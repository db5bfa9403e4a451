"""Pins of the symmetron oracle (oracle/symmetron.py) to facts that do not come
from the oracle itself: the closed-form homogeneous solutions, the exact FFT
solution of the linearised discrete equation, brute-force Newton on the
whole grid, the algebraic (short-range) limit, finite differences of the
operator, and exactness of the multigrid transfer operators.

The model (Hinterbichler & Khoury 2010, simulated in Davis, Li, Mota &
Winther 2011; the paper's Sec. I and VII name it among the models its
solver carries over to):
    A sum_j (chi_j - chi_i) - [ (s rho_i - 1) chi_i + chi_i^3 ] = 0,
    A = 2 lambda_0^2 / (a^2 (B h)^2),  s = (a_SSB / a)^3.
"""
import numpy as np
import pytest

from oracle import symmetron as S
from paper_1110_1379_gb300 import synth

P = dict(a=1.0, a_ssb=0.5, lambda0=1.0)


def test_coefficients_closed_form():
    # 0.5 Mpc/h cells, lambda_0 = 1 Mpc/h, a = 1: A = 2 / 0.25 = 8; s = 1/8
    A, s = S.coefficients(16.0, 32, **P)
    assert A == pytest.approx(8.0, rel=1e-15) and s == pytest.approx(0.125, rel=1e-15)
    # A scales as lambda_0^2 / (a h)^2
    A2, s2 = S.coefficients(16.0, 64, a=0.8, a_ssb=0.5, lambda0=2.0)
    assert A2 == pytest.approx(8.0 * 4 * 4 / 0.64, rel=1e-14)
    assert s2 == pytest.approx((0.5 / 0.8) ** 3, rel=1e-14)


@pytest.mark.parametrize("a,expect", [(1.0, np.sqrt(1 - 0.125)), (0.4, 0.0)])
def test_homogeneous_solution_from_random_start(a, expect):
    """rho = 1: the positive root of (s - 1) chi + chi^3 = 0 after symmetry
    breaking (a > a_SSB), chi = 0 before (the field's symmetric phase)."""
    rng = np.random.default_rng(0)
    chi0 = rng.uniform(0.3, 1.5, (16, 16, 16))
    r = S.solve(np.ones((16, 16, 16)), box=8.0, a=a, a_ssb=0.5, lambda0=1.0, tol=1e-12,
                chi0=chi0)
    assert r.converged
    assert np.abs(r.chi - expect).max() < 1e-10
    assert S.background(a, 0.5) == pytest.approx(expect, abs=1e-15)


def test_linear_limit_matches_fft_solution():
    """rho = 1 + eps g: the solution is the FFT solution of the linearised
    discrete equation up to O(eps^2)."""
    n, eps = 16, 1e-5
    g = synth.gaussian_random_field((n,) * 3, 3, sigma=1.0)
    rho = 1.0 + eps * g
    r = S.solve(rho, box=8.0, tol=1e-14, **P)
    lin = S.linear_response(g, eps, box=8.0, **P)
    chib = S.background(1.0, 0.5)
    dev = np.abs(lin - chib).max()
    assert dev > 1e-7  # a real response
    assert np.abs(r.chi - lin).max() <= 1e-3 * dev


def test_fas_matches_dense_newton_brute_force():
    n = 8
    rho = synth.lognormal_density((n,) * 3, 5, sigma=1.5)
    r = S.solve(rho, box=4.0, tol=1e-13, **P)
    ref = S.dense_newton(rho, box=4.0, chi0=np.full(rho.shape, 0.9), **P)
    assert r.converged
    assert np.abs(r.chi - ref).max() < 1e-10
    # a second start on the other side of the root reaches the same root (the
    # positive branch; the field's chi -> -chi symmetry also admits the mirror
    # image and mixed-sign roots, which a start near 0 can fall into)
    ref2 = S.dense_newton(rho, box=4.0, chi0=np.full(rho.shape, 1.3), **P)
    assert np.abs(ref2 - ref).max() < 1e-10
    A, s = S.coefficients(4.0, n, **P)
    mirror = -ref
    assert np.abs(S.operator(mirror, rho, A, s)).max() < 1e-12


def test_short_range_limit_is_the_local_minimum():
    """lambda_0 much smaller than a cell: the gradient term vanishes and chi
    sits at the minimum of the effective potential, sqrt(max(0, 1 - s rho))."""
    n = 16
    rho = synth.lognormal_density((n,) * 3, 9, sigma=1.0)
    r = S.solve(rho, box=16.0 * n, a=1.0, a_ssb=0.5, lambda0=0.01, tol=1e-12)
    s = 0.125
    local = np.sqrt(np.maximum(0.0, 1.0 - s * rho))
    # A = 2e-4 / 256 ~ 8e-7: the neighbours shift chi by O(A / m^2), the mass
    # m^2 = |2 (1 - s rho)| vanishing only at the transition s rho = 1
    away = np.abs(1.0 - s * rho) > 0.05
    assert r.converged and away.mean() > 0.8
    assert np.abs(r.chi - local)[away].max() < 1e-4


def test_screening_in_dense_cells():
    """Cells with s rho > 1 are screened (chi -> 0 in the short-range limit),
    cells of low density approach the vacuum value 1."""
    n = 16
    rho = synth.lognormal_density((n,) * 3, 9, sigma=2.0)
    r = S.solve(rho, box=16.0 * n, a=1.0, a_ssb=0.5, lambda0=0.01, tol=1e-12)
    dense = 0.125 * rho > 1.5
    void = rho < 0.1
    assert dense.any() and void.any()
    assert r.chi[dense].max() < 1e-3
    assert r.chi[void].min() > 0.99


def test_newton_derivative_by_finite_differences():
    rng = np.random.default_rng(4)
    shape = (6, 6, 6)
    chi = rng.uniform(0.1, 1.2, shape)
    rho = rng.uniform(0.2, 5.0, shape)
    A, s = S.coefficients(3.0, 6, **P)
    d = S.derivative(chi, rho, A, s)
    for idx in [(0, 0, 0), (2, 3, 5), (5, 5, 1)]:
        h = 1e-6
        cp, cm = chi.copy(), chi.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (S.operator(cp, rho, A, s)[idx] - S.operator(cm, rho, A, s)[idx]) / (2 * h)
        assert fd == pytest.approx(d[idx], rel=1e-7)


def test_operator_sums_to_the_local_terms():
    """The face differences cancel in pairs on a periodic grid: sum_i L_i is
    minus the sum of the local terms."""
    rng = np.random.default_rng(6)
    chi = rng.uniform(0.1, 1.2, (8, 6, 10))
    rho = rng.uniform(0.2, 5.0, chi.shape)
    A, s = S.coefficients(5.0, 10, **P)
    tot = S.operator(chi, rho, A, s).sum()
    loc = ((s * rho - 1.0) * chi + chi ** 3).sum()
    assert tot == pytest.approx(-loc, rel=1e-12)


def test_transfer_operators():
    rng = np.random.default_rng(8)
    c = rng.standard_normal((4, 6, 8))
    # restriction of a prolonged constant, and of any field, keeps the mean
    assert np.allclose(S.restrict(np.full((8, 12, 16), 2.5)), 2.5)
    assert S.restrict(rng.standard_normal((8, 12, 16))).shape == (4, 6, 8)
    f = rng.standard_normal((8, 12, 16))
    assert S.restrict(f).mean() == pytest.approx(f.mean(), rel=1e-12)
    # prolongation: constants exactly, the 27/9/3/1 weights at one fine cell
    assert np.allclose(S.prolong(np.full((4, 6, 8), -1.25)), -1.25)
    p = S.prolong(c)
    k, j, i = 3, 5, 6  # fine cell (odd, odd, even) -> coarse (1, 2, 3)
    K, J, I = 1, 2, 3
    w = {0: 27, 1: 9, 2: 3, 3: 1}
    acc = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                kk = K + (dk if k % 2 else -dk)
                jj = J + (dj if j % 2 else -dj)
                ii = I + (di if i % 2 else -di)
                acc += w[dk + dj + di] * c[kk % 4, jj % 6, ii % 8]
    assert p[k, j, i] == pytest.approx(acc / 64.0, rel=1e-13)
    # linear fields are reproduced away from the periodic seam
    x = np.arange(8, dtype=float)
    lin = np.broadcast_to(x, (4, 6, 8)).copy()
    pl = S.prolong(lin)
    xf = (np.arange(16) + 0.5) / 2 - 0.5  # fine cell centres in coarse units
    assert np.allclose(pl[:, :, 2:14], np.broadcast_to(xf[2:14], (8, 12, 12)))


def test_manufactured_solution_through_the_multigrid():
    """A smooth chi* and the density for which it solves the discrete
    equation: the V-cycles return chi* (the transfer operators and coarse
    levels must be consistent for the fine residual to reach 1e-13)."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    chi_s = 0.7 + 0.15 * np.sin(2 * np.pi * X) * np.cos(4 * np.pi * Y) + 0.1 * np.sin(2 * np.pi * Z)
    chi_s = np.ascontiguousarray(np.transpose(chi_s, (2, 1, 0)))
    A, s = S.coefficients(16.0, n, **P)
    lap = S.laplacian_sum(chi_s)
    rho = ((A * lap - chi_s ** 3) / chi_s + 1.0) / s
    r = S.solve(rho, box=16.0, tol=1e-13, **P)
    assert r.converged and r.cycles <= 15
    assert np.abs(r.chi - chi_s).max() < 1e-11


def test_sweep_equals_cell_by_cell_red_then_black():
    """One vectorised sweep equals Newton-Gauss-Seidel written cell by cell,
    red cells ((i + j + k) even) in index order first, then black, each
    update clamped to |d chi| <= cap; a large start makes the clamp act."""
    rng = np.random.default_rng(21)
    shape = (4, 6, 8)
    rho = synth.lognormal_density(shape, 5, sigma=1.0)
    A, s = S.coefficients(4.0, shape[2], **P)
    chi0 = rng.uniform(-2.0, 3.0, shape)
    f = 0.1 * rng.standard_normal(shape)
    cap = 0.25
    got = S.smooth(chi0, rho, f, A, s, 1, cap=cap)
    ref = chi0.copy()
    n2, n1, n0 = shape
    hit = 0
    for colour in (0, 1):
        for k in range(n2):
            for j in range(n1):
                for i in range(n0):
                    if (i + j + k) % 2 != colour:
                        continue
                    nb = sum(ref[(k + dk) % n2, (j + dj) % n1, (i + di) % n0]
                             for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                                (0, 0, 1), (0, 0, -1)))
                    c = ref[k, j, i]
                    L = A * (nb - 6.0 * c) - ((s * rho[k, j, i] - 1.0) * c + c ** 3)
                    dL = -6.0 * A - ((s * rho[k, j, i] - 1.0) + 3.0 * c * c)
                    d = -(L - f[k, j, i]) / dL
                    hit += abs(d) > cap
                    ref[k, j, i] = c + min(max(d, -cap), cap)
    assert hit > 10
    assert np.abs(got - ref).max() < 1e-12


def test_level_rule_and_coarsest_rule_by_hand():
    """Readings stated in the oracle: levels halve while every size is even and
    the halved size is >= 4 (16 -> 8 -> 4; 12 -> 6, since 6 would halve to 3;
    odd sizes stop); the coarsest level is relaxed until its rms residual is
    <= max(1e-3 x its initial rms, 0.1 tol), and stops at the first sweep that
    reaches it."""
    assert S.num_levels((16, 16, 16)) == 3
    assert S.num_levels((12, 12, 12)) == 2
    assert S.num_levels((16, 8, 24)) == 2 and S.num_levels((10, 16, 16)) == 2
    assert S.num_levels((6, 16, 16)) == 1
    rho = synth.lognormal_density((4, 4, 4), 9, sigma=1.0)
    A, s = S.coefficients(2.0, 4, **P)
    chi = np.full((4, 4, 4), 2.0)
    f = np.zeros_like(rho)
    rms = lambda c: float(np.sqrt(np.mean((S.operator(c, rho, A, s) - f) ** 2)))  # noqa: E731
    r0 = rms(chi)
    out = S._coarsest(chi, rho, f, A, s, 1e-8, 1.0)
    lim = max(1e-3 * r0, 1e-9)
    assert rms(out) <= lim
    c, n = chi.copy(), 0
    while rms(c) > lim:
        c = S.smooth(c, rho, f, A, s, 1, 1.0)
        n += 1
    assert n >= 2 and np.array_equal(c, out)


def test_two_level_cycle_by_hand():
    """One two-level FAS cycle (Sec. V.B.2) written out step by step: pre
    sweeps; d = L(chi) - f; coarse chi = R chi, coarse density = the mean of
    the 8 children (loops), coarse A = A / 4 (twice the cell size); coarse
    right-hand side L^H(R chi) - R d; coarse solve; chi += P(chi^H - R chi);
    post sweeps."""
    rng = np.random.default_rng(31)
    shape = (8, 8, 12)
    rho = synth.lognormal_density(shape, 6, sigma=1.0)
    A, s = S.coefficients(6.0, shape[2], **P)
    chi0 = 0.9 + 0.1 * rng.standard_normal(shape)
    f = np.zeros(shape)
    got = S.vcycle(chi0, rho, f, A, s, 2, pre=2, post=1, cap=1.0, tol=1e-10)
    c = S.smooth(chi0, rho, f, A, s, 2)
    d = S.operator(c, rho, A, s) - f
    rhoH = np.zeros((4, 4, 6))
    for K in range(4):
        for J in range(4):
            for I in range(6):
                rhoH[K, J, I] = rho[2 * K:2 * K + 2, 2 * J:2 * J + 2, 2 * I:2 * I + 2].mean()
    uR = S.restrict(c)
    fH = S.operator(uR, rhoH, A / 4.0, s) - S.restrict(d)
    uH = S._coarsest(uR.copy(), rhoH, fH, A / 4.0, s, 1e-10, 1.0)
    ref = S.smooth(c + S.prolong(uH - uR), rho, f, A, s, 1)
    assert np.abs(got - ref).max() < 1e-13
