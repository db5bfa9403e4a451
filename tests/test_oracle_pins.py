"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test fails for a plausible mistake in the oracle: a dropped term, a wrong
sign, a wrong index or a transposed operand.
* constants: the paper's printed -Rbar = 41 m^2; the homogeneous solution.
* E1 homogeneous density -> u = 0 (Sec. VI.A.1).
* algebraic limit alpha -> 0 (pins beta, gamma and the e^{-u/2} term).
* linear limit against the exact FFT solution (pins alpha, h^2, beta/2, gamma,
  and the flux form's linearisation); the point mass of Sec. VI.A.2 included.
* sine and Gaussian closed forms converge at order 2 (Sec. VI.A.3, VI.A.4);
  these pin the nonlinear flux form b_{i+1/2} = (b_i + b_{i+1})/2.
* telescoping: the flux terms sum to zero over a periodic grid.
* Newton derivative against central differences, ghost faces included.
* FAS solution equals a dense-Jacobian Newton root (8^3, periodic and patch).
* restriction / prolongation identities; weights 27/9/3/1 over 64.
* multigrid convergence vs single-grid relaxation (Sec. VI.D.1).
* refinement patches (Sec. VI.B.1): edge error and peak improvement, two and
  three levels.
* CIC (Sec. VI.C): mean density 1, centred particle, translation, brute force.
"""
import os

import numpy as np
import pytest

import paper_fields as PF
from oracle import oracle as O
from paper_1110_1379_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(key):
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as fh:
        for line in fh:
            parts = line.split()
            if parts and not line.startswith("#") and parts[0] == key:
                return float(parts[1])
    raise KeyError(key)


F5_64 = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)


# ---------------------------------------------------------------- constants
def test_minus_rbar_41():
    m = O.Model(64.0, 32, 1.0, 0.24, 1e-5)
    three_k1 = 3.0 * m.bkg / (m.dens)  # bkg = Om a^4 K, dens = Om a, a = 1
    assert round(three_k1) == golden("minus_Rbar_over_m2")


@pytest.mark.parametrize("a", [1.0, 0.5, 0.04])
def test_background_matches_paper_fields(a):
    m = O.Model(128.0, 128, a, 0.24, 1e-5)
    assert np.exp(m.ubar) == pytest.approx(PF.fbar_tilde_abs(a, 0.24, 1e-5), rel=1e-12)
    alpha, beta, gamma = PF.coefficients(128.0, 128, a, 0.24, 1e-5)
    assert 2 * m.pre * np.exp(m.ubar) == pytest.approx(alpha, rel=1e-12)
    assert m.bkg == pytest.approx(beta, rel=1e-12)
    assert m.dens == pytest.approx(gamma, rel=1e-12)
    if a == 1.0:
        assert np.exp(m.ubar) == pytest.approx(1e-5, rel=1e-12)  # |fbar_R(1)| = |f_R0|


# ---------------------------------------------------------------- E1
@pytest.mark.parametrize("a", [0.04, 1.0])
def test_homogeneous_converges_to_background(a):
    rng = np.random.default_rng(0)
    n = 8
    u0 = rng.uniform(-1, 1, (n, n, n))
    r = O.solve(np.ones((n, n, n)), u0=u0, tol=1e-13, box=64.0, a=a, omega_m=0.24, fr0=1e-5)
    assert r.converged
    _, beta, _ = PF.coefficients(64.0, n, a, 0.24, 1e-5)
    # |u| <= rms residual / smallest eigenvalue (beta/2) up to a safety factor
    assert np.abs(r.u).max() < 100 * 1e-13 / (beta / 2)


# ---------------------------------------------------------------- algebraic limit
def test_algebraic_limit():
    rho = synth.lognormal_density((8, 8, 8), 7, sigma=1.5)
    P = dict(box=64.0, a=0.7, omega_m=0.24, fr0=1e-16)
    r = O.solve(rho, tol=1e-14, **P)
    assert r.converged
    exact = PF.algebraic_limit(rho, a=0.7, omega_m=0.24)
    assert np.abs(r.u - exact).max() < 1e-8


# ---------------------------------------------------------------- linear limit
@pytest.mark.parametrize("fr0,box", [(1e-4, 256.0), (1e-5, 64.0), (1e-6, 32.0)])
def test_linear_limit_fft(fr0, box):
    n, eps = 16, 1e-6
    g = synth.gaussian_random_field((n, n, n), 5, sigma=1.0)
    P = dict(box=box, a=1.0, omega_m=0.24, fr0=fr0)
    r = O.solve(1.0 + eps * g, tol=1e-15, max_cycles=40, **P)
    ul = PF.linear_response(g, eps, **P)
    assert np.abs(r.u - ul).max() < 1e-5 * np.abs(ul).max()


def test_point_mass_far_field_is_linear_yukawa():
    """Sec. VI.A.2 point mass at small amplitude: the solution is the discrete
    Yukawa Green's function (exact for the linearised operator)."""
    n = 16
    eps = golden("point_mass_contrast") * 1e-3
    rho = synth.point_mass_density(n)
    g = (rho - 1.0) / golden("point_mass_contrast")
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    r = O.solve(1.0 + eps * g, tol=1e-16, max_cycles=40, **P)
    ul = PF.linear_response(g, eps, **P)
    assert np.abs(r.u - ul).max() < 1e-5 * np.abs(ul).max()
    # the scalaron is most suppressed at the mass and rises monotonically away from it
    line = r.u[0, 0, : n // 2 + 1]
    assert np.all(np.diff(line) > 0)


# ---------------------------------------------------------------- closed forms
def _orders(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("fr0", [1e-4, 1e-5, 1e-6])
def test_sine_closed_form_second_order(fr0):
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=fr0)
    errs = []
    for n in (16, 32):
        rho, ue = PF.sine_field(n, **P)
        r = O.solve(rho, tol=1e-11, max_cycles=60, **P)
        assert r.converged
        errs.append(np.abs(r.u - ue).max())
    (order,) = _orders(errs)
    assert 1.8 < order < 2.2, errs
    assert errs[-1] < 1e-3


@pytest.mark.slow
def test_sine_closed_form_second_order_64():
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    errs = []
    for n in (32, 64):
        rho, ue = PF.sine_field(n, **P)
        errs.append(np.abs(O.solve(rho, tol=1e-11, **P).u - ue).max())
    assert 1.9 < _orders(errs)[0] < 2.1


def test_gaussian_closed_form_converges():
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    errs = []
    for n in (32, 64):
        rho, ue = PF.gaussian_field(n, amp=0.5, width=0.14, **P)
        r = O.solve(rho, tol=1e-11, **P)
        assert r.converged
        errs.append(np.abs(r.u - ue).max())
    assert 1.75 < _orders(errs)[0] < 2.25, errs


# ---------------------------------------------------------------- invariants
def test_flux_terms_telescope():
    rng = np.random.default_rng(3)
    n = 8
    u = rng.uniform(-2, 1, (n, n, n))
    rho = synth.lognormal_density((n, n, n), 9, sigma=1.0)
    P = dict(box=64.0, a=0.8, omega_m=0.24, fr0=1e-5)
    d = O.residual(u, rho, **P)
    _, beta, gamma = PF.coefficients(64.0, n, 0.8, 0.24, 1e-5)
    local = beta * (np.exp(-u / 2) - 1) - gamma * (rho - 1)
    assert d.sum() == pytest.approx(local.sum(), abs=1e-9 * np.abs(d).sum())
    # and the flux part is far from zero cell by cell
    assert np.abs(d - local).max() > 1.0


def _random_patch(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 0.5, (n, n, n))
    ub = rng.uniform(-1.0, 0.5, sum(O.face_sizes((n, n, n))))
    rho = synth.lognormal_density((n, n, n), seed, sigma=1.0)
    return u, ub, rho


@pytest.mark.parametrize("with_ghosts", [False, True])
def test_newton_derivative_central_difference(with_ghosts):
    n = 6
    u, ub, rho = _random_patch(n, 11)
    ub = ub if with_ghosts else None
    P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5, h=1.0 / 16, ub=ub)
    cells = [(0, 0, 0), (5, 2, 3), (2, 3, 1), (5, 5, 5), (0, 3, 5)]
    for (i, j, k) in cells:
        _, dl = O.cell_op(u, rho, i, j, k, **P)
        eps = 1e-6
        up = u.copy()
        up[k, j, i] += eps
        um = u.copy()
        um[k, j, i] -= eps
        lp, _ = O.cell_op(up, rho, i, j, k, **P)
        lm, _ = O.cell_op(um, rho, i, j, k, **P)
        assert dl == pytest.approx((lp - lm) / (2 * eps), rel=1e-6)


def test_dense_newton_matches_fas_periodic():
    n = 8
    rho = synth.lognormal_density((n, n, n), 21, sigma=1.5)
    P = dict(box=32.0, a=1.0, omega_m=0.24, fr0=1e-5)
    ub, _ = O.dense_newton(rho, **P)
    r = O.solve(rho, tol=1e-13, **P)
    assert r.converged
    assert np.abs(r.u - ub).max() < 1e-10
    # uniqueness: another start reaches the same root
    ub2, _ = O.dense_newton(rho, u0=np.full(rho.shape, -1.0), **P)
    assert np.abs(ub2 - ub).max() < 1e-10


def test_dense_newton_matches_fas_patch():
    n = 8
    _, ub, rho = _random_patch(n, 5)
    P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5, h=1.0 / 32, ub=ub)
    un, _ = O.dense_newton(rho, **P)
    r = O.solve(rho, tol=1e-13, **P)
    assert r.converged
    assert np.abs(r.u - un).max() < 1e-10


# ---------------------------------------------------------------- transfer operators
def test_restriction_identities():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((8, 12, 16))
    c = O.restrict(f)
    assert c.shape == (4, 6, 8)
    assert c.mean() == pytest.approx(f.mean(), abs=1e-14)
    assert c[1, 2, 3] == pytest.approx(f[2:4, 4:6, 6:8].mean(), abs=1e-15)
    assert np.allclose(O.restrict(np.full((4, 4, 4), 2.5)), 2.5, atol=0, rtol=0)


def test_prolongation_weights_are_the_papers():
    nf = (8, 8, 8)
    e = np.zeros((4, 4, 4))
    e[1, 1, 1] = 64.0
    uf = O.prolong_correct(np.zeros(nf), e, np.zeros_like(e))
    # fine cell (x=3,y=3,z=3) sits in coarse (1,1,1): weight 27
    assert uf[3, 3, 3] == golden("prolong_w_parent")
    # fine cell (x=4,y=3,z=3) has (1,1,1) as a face neighbour
    assert uf[3, 3, 4] == golden("prolong_w_face")
    assert uf[3, 4, 4] == golden("prolong_w_edge")
    assert uf[4, 4, 4] == golden("prolong_w_vertex")
    assert uf.sum() == 8 * golden("prolong_denominator")  # weights sum to 1 per fine cell


def test_prolongation_exact_for_linear_fields():
    nc = 8
    x = np.arange(nc) + 0.5
    zc, yc, xc = np.meshgrid(x, x, x, indexing="ij")
    e = 0.3 * xc - 0.7 * yc + 1.1 * zc
    uf = O.prolong_correct(np.zeros((2 * nc,) * 3), e, np.zeros_like(e))
    xf = (np.arange(2 * nc) + 0.5) / 2.0
    zf, yf, xf = np.meshgrid(xf, xf, xf, indexing="ij")
    ref = 0.3 * xf - 0.7 * yf + 1.1 * zf
    inner = (slice(1, -1),) * 3
    assert np.abs(uf[inner] - ref[inner]).max() < 1e-12
    const = O.prolong_correct(np.zeros((8, 8, 8)), np.full((4, 4, 4), 3.0), np.zeros((4, 4, 4)))
    assert np.abs(const - 3.0).max() < 1e-15


def test_prolongation_on_a_patch_drops_outside_cells():
    """On a patch (Sec. V.A.3: a coarse cell outside the patch is no multigrid
    cell and adds nothing; the remaining weights are not renormalised, reading
    D15) a constant correction c reaches a fine cell scaled by 3/4 for every
    axis along which the cell touches the patch boundary, since the 27/9/3/1
    weights factor into 3/4 (own coarse cell) and 1/4 (neighbour) per axis;
    periodic grids wrap and reproduce c everywhere."""
    shape = (6, 10, 8)                                # (n2, n1, n0)
    cs = tuple(v // 2 for v in shape)
    c = 2.5
    uf = O.prolong_correct(np.zeros(shape), np.full(cs, c), np.zeros(cs), dirichlet=True)
    k, j, i = np.indices(shape)
    nb = sum(((ix == 0) | (ix == n - 1)).astype(int) for ix, n in ((i, shape[2]), (j, shape[1]),
                                                                  (k, shape[0])))
    assert np.abs(uf - c * 0.75 ** nb).max() < 1e-15
    up = O.prolong_correct(np.zeros(shape), np.full(cs, c), np.zeros(cs), dirichlet=False)
    assert np.abs(up - c).max() < 1e-15


def test_face_restriction_exact_for_linear_faces():
    """Coarse patch boundary values (Sec. V.B.2 reading: the mean of the 4 fine
    face values covering a coarse face cell) reproduce a field linear along
    each face: the mean of a linear function over the 2 x 2 fine face cells is
    its value at the coarse face cell's centre.  Distinct slopes along the two
    in-face axes and unequal sizes make a swapped axis or a shifted block fail."""
    shape = (6, 10, 14)                       # (n2, n1, n0)
    n = [shape[2], shape[1], shape[0]]        # n0, n1, n2
    axes = {0: (1, 2), 1: (0, 2), 2: (0, 1)}  # in-face axes p < q of the face normal to ax

    def faces(nn, coef):
        out = []
        for f in range(6):
            p, q = axes[f // 2]
            a0, b, c = coef[f]
            P = (np.arange(nn[p]) + 0.5) / nn[p]
            Q = (np.arange(nn[q]) + 0.5) / nn[q]
            out.append((a0 + b * P[None, :] + c * Q[:, None]).ravel())  # index Q n_p + P
        return np.concatenate(out)

    rng = np.random.default_rng(11)
    coef = [tuple(rng.uniform(-2.0, 2.0, 3)) for _ in range(6)]
    fine = faces(n, coef)
    assert fine.size == sum(O.face_sizes(shape))
    coarse = O.restrict_faces(fine, shape)
    expect = faces([v // 2 for v in n], coef)
    assert np.abs(coarse - expect).max() < 1e-14


def test_sweep_equals_cell_by_cell_red_then_black():
    """One oracle sweep equals Newton-Gauss-Seidel written cell by cell from
    the single-cell operator: red cells ((i + j + k) even) in index order
    first, then black, u <- u - (L - f) / (dL/du) clamped to |du| <= cap (the
    clamp acts from this start)."""
    rng = np.random.default_rng(41)
    shape = (4, 4, 6)
    rho = synth.lognormal_density(shape, 3, sigma=1.0)
    u0 = rng.uniform(-2.0, 1.0, shape)
    f = 0.01 * rng.standard_normal(shape)
    h, cap = 1.0 / 16, 0.25
    got = O.smooth(u0, rho, 1, h=h, f=f, cap=cap, **F5_64)
    ref = u0.copy()
    hit = 0
    for colour in (0, 1):
        for k in range(shape[0]):
            for j in range(shape[1]):
                for i in range(shape[2]):
                    if (i + j + k) % 2 != colour:
                        continue
                    L, dL = O.cell_op(ref, rho, i, j, k, h=h, **F5_64)
                    du = -(L - f[k, j, i]) / dL
                    hit += abs(du) > cap
                    ref[k, j, i] += min(max(du, -cap), cap)
    assert hit > 5
    assert np.abs(got - ref).max() < 1e-12


def test_two_level_vcycle_by_hand():
    """One two-level FAS V-cycle of the oracle (Sec. V.B.2) equals its steps
    written out with the single-step entry points: pre sweeps; d = L(u);
    u^H = R u, f^H = L^H(R u) - R d at twice the cell size with density R rho;
    coarsest solve (sweeps until rms(L^H - f^H) <= max(1e-3 x its initial
    rms, 0.1 tol), at least one); u += P(u^H - R u); post sweeps."""
    rng = np.random.default_rng(42)
    shape = (8, 8, 12)
    assert O.num_levels(shape) == 2
    rho = synth.lognormal_density(shape, 4, sigma=1.0)
    u0 = 0.3 * rng.standard_normal(shape)
    h, tol, pre, post = 1.0 / 24, 1e-9, 2, 1
    got = O.solve(rho, u0=u0, h=h, tol=tol, pre=pre, post=post, ncycles=1, **F5_64).u
    rms = lambda d: float(np.sqrt(np.mean(d * d)))  # noqa: E731
    u = O.smooth(u0, rho, pre, h=h, **F5_64)
    d = O.residual(u, rho, h=h, **F5_64)
    uR, rhoH = O.restrict(u), O.restrict(rho)
    fH = O.residual(uR, rhoH, h=2 * h, **F5_64) - O.restrict(d)
    thr = max(1e-3 * rms(O.residual(uR, rhoH, h=2 * h, f=fH, **F5_64)), 0.1 * tol)
    uH = uR.copy()
    for _ in range(500):
        uH = O.smooth(uH, rhoH, 1, h=2 * h, f=fH, **F5_64)
        if rms(O.residual(uH, rhoH, h=2 * h, f=fH, **F5_64)) <= thr:
            break
    u = O.prolong_correct(u, uH, uR)
    ref = O.smooth(u, rho, post, h=h, **F5_64)
    assert np.abs(got - ref).max() < 1e-11


def test_level_count_rule():
    assert O.num_levels((32, 32, 32)) == 4  # 32 16 8 4
    assert O.num_levels((512, 512, 512)) == 8
    assert O.num_levels((48, 48, 48)) == 4  # 48 24 12 6
    assert O.num_levels((96, 96, 96)) == 5
    assert O.num_levels((10, 10, 10)) == 1


# ---------------------------------------------------------------- multigrid vs single grid
def test_vcycle_beats_single_grid():
    """Sec. VI.D.1: V-cycles reach 1e-12 within tens of finest-grid sweeps, while
    single-grid relaxation of the F4 sine field stalls."""
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-4)
    rho, _ = PF.sine_field(32, **P)
    r = O.solve(rho, tol=golden("vcycle_residual"), max_cycles=40, **P)
    assert r.converged
    assert (2 + 2) * r.cycles <= 80
    u = O.smooth(np.zeros_like(rho), rho, 80, **P)
    single = np.sqrt(np.mean(O.residual(u, rho, **P) ** 2))
    assert single > 1e4 * golden("vcycle_residual")


# ---------------------------------------------------------------- refinement patches
def test_two_level_gaussian_patch():
    """Sec. VI.B.1 with a spherical Gaussian peak (3D analogue of Eq. gaussian_dens):
    a patch over the peak is more accurate there than its parent, agrees with a
    full fine-grid solve away from its edges, and carries a small
    interpolation error at its edges."""
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    G = dict(amp=0.99, width=0.06, centre=(0.5, 0.5, 0.5))
    N, n, o = 32, 16, 12
    rho0, ue0 = PF.spherical_gaussian_field(N, **P, **G)
    rhop, uep = PF.spherical_gaussian_patch(2 * o, n, 2 * N, **P, **G)
    dom, (pat,) = O.solve_levels(rho0, [dict(parent=-1, origin=(o, o, o), rho=rhop)],
                                 tol=1e-10, **P)
    assert dom.converged and pat.converged
    err_p = np.abs(pat.u - uep)
    err_d = np.abs(dom.u - ue0)
    c, C = n // 2, N // 2
    assert err_p[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1].max() < \
        err_d[C - 1:C + 1, C - 1:C + 1, C - 1:C + 1].max()
    full_r, full_u = PF.spherical_gaussian_field(2 * N, **P, **G)
    full = O.solve(full_r, tol=1e-10, **P)
    sl = slice(2 * o, 2 * o + n)
    err_f = np.abs(full.u - full_u)[sl, sl, sl]
    inner = (slice(4, -4),) * 3
    assert err_p[inner].max() < 1.2 * err_f[inner].max() + 1e-3
    # boundary interpolation error: small, as the paper reports at refinement edges
    assert err_p.max() < 0.02
    assert err_p[0].max() < 20 * golden("refinement_edge_error")


def test_three_level_gaussian_patch():
    """Sec. VI.B's nested refinement on the spherical Gaussian: a level-2
    patch inside the level-1 patch takes its boundary from that patch (not
    from the domain grid) and is more accurate at the peak than its parent,
    with a small error at its edges."""
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    G = dict(amp=0.99, width=0.06, centre=(0.5, 0.5, 0.5))
    N, n, o1, o2 = 32, 16, 12, 4                   # level-2 patch over level-1 cells 4..11
    rho0, _ = PF.spherical_gaussian_field(N, **P, **G)
    rho1, ue1 = PF.spherical_gaussian_patch(2 * o1, n, 2 * N, **P, **G)
    lo2 = 2 * (2 * o1 + o2)
    rho2, ue2 = PF.spherical_gaussian_patch(lo2, n, 4 * N, **P, **G)
    dom, (p1, p2) = O.solve_levels(
        rho0, [dict(parent=-1, origin=(o1, o1, o1), rho=rho1),
               dict(parent=0, origin=(o2, o2, o2), rho=rho2)], tol=1e-10, **P)
    assert p1.converged and p2.converged
    e1, e2 = np.abs(p1.u - ue1), np.abs(p2.u - ue2)
    c = n // 2
    assert e2[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1].max() < \
        e1[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1].max()
    assert e2.max() < 0.02


def _faces_from(u, lo, n):
    """Packed u_b = (ghost + first interior)/2 of the block lo..lo+n of u."""
    hi = lo + n
    b = slice(lo, hi)
    out = []
    for ax in range(3):
        for side in range(2):
            g = lo - 1 if side == 0 else hi
            i = lo if side == 0 else hi - 1
            if ax == 0:
                fg, fi = u[b, b, g], u[b, b, i]
            elif ax == 1:
                fg, fi = u[b, g, b], u[b, i, b]
            else:
                fg, fi = u[g, b, b], u[i, b, b]
            out.append((0.5 * (fg + fi)).ravel())
    return np.concatenate(out)


def test_patch_with_exact_boundary_reproduces_full_grid():
    """Eq. (bc_modified_fR_op) with u_b taken from a full-grid solution: the
    patch problem's solution is that full solution restricted to the patch."""
    P = dict(box=128.0, a=0.8, omega_m=0.24, fr0=1e-5)
    rho = synth.lognormal_density((32, 32, 32), 77, sigma=1.2)
    full = O.solve(rho, tol=1e-12, **P)
    lo, n = 6, 16
    ub = _faces_from(full.u, lo, n)
    sl = slice(lo, lo + n)
    pat = O.solve(rho[sl, sl, sl].copy(), tol=1e-12, h=1.0 / 32, ub=ub, **P)
    assert pat.converged
    assert np.abs(pat.u - full.u[sl, sl, sl]).max() < 1e-9


def test_patch_bc_exact_for_linear_parent():
    """Trilinear 27/9/3/1 interpolation is exact for a linear parent field, so the
    initial patch u and u_b (at the face centres) are exact."""
    npar = (12, 10, 14)  # (n2, n1, n0)
    xs = [(np.arange(m) + 0.5) for m in (npar[2], npar[1], npar[0])]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    lin = lambda X, Y, Z: 0.2 * X - 0.3 * Y + 0.05 * Z - 1.0  # noqa: E731
    up = lin(x, y, z)
    org, n = (3, 2, 4), (6, 8, 10)  # origin (x,y,z) in parent cells; n = (n2,n1,n0)
    u0, ub = O.patch_bc(up, org, n, parent_periodic=False)
    fx = org[0] + (np.arange(n[2]) + 0.5) / 2
    fy = org[1] + (np.arange(n[1]) + 0.5) / 2
    fz = org[2] + (np.arange(n[0]) + 0.5) / 2
    Z, Y, X = np.meshgrid(fz, fy, fx, indexing="ij")
    assert np.abs(u0 - lin(X, Y, Z)).max() < 1e-13
    sizes = O.face_sizes(n)
    off = np.cumsum([0] + sizes)
    ymid, zmid = np.meshgrid(fy, fz, indexing="ij")  # -x face: index z*ny + y
    face_mx = ub[off[0]:off[1]].reshape(n[0], n[1])
    assert np.abs(face_mx - lin(org[0], ymid.T, zmid.T)).max() < 1e-13
    face_pz = ub[off[5]:off[6]].reshape(n[1], n[2])
    Yp, Xp = np.meshgrid(fy, fx, indexing="ij")
    assert np.abs(face_pz - lin(Xp, Yp, org[2] + n[0] / 2)).max() < 1e-13
    # a stencil that would leave a non-periodic parent is rejected
    with pytest.raises(ValueError):
        O.patch_bc(up, (0, 2, 4), n, parent_periodic=False)


def test_patch_bc_wraps_a_periodic_parent():
    """A patch on a periodic parent that crosses the domain edge is set up
    from the periodic continuation of the parent: the same as a non-periodic
    parent padded by one layer of wrapped cells, with the origin shifted by
    one parent cell."""
    rng = np.random.default_rng(12)
    npar = (8, 10, 12)                            # (n2, n1, n0)
    up = rng.normal(size=npar)
    n = (6, 8, 10)
    for org in [(0, 0, 0), (9, 7, 5), (8, 1, 6)]:   # (x, y, z); past the upper edge too
        u0, ub = O.patch_bc(up, org, n, parent_periodic=True)
        o2 = (org[0] % npar[2] + 1, org[1] % npar[1] + 1, org[2] % npar[0] + 1)
        big = np.pad(up, ((1, n[0]), (1, n[1]), (1, n[2])), mode="wrap")  # index 0 = cell -1
        v0, vb = O.patch_bc(big, o2, n, parent_periodic=False)
        assert np.array_equal(u0, v0) and np.array_equal(ub, vb)


# ---------------------------------------------------------------- CIC
def test_cic_mean_density_is_one():
    pos = synth.uniform_positions(5000, 3)
    rho = O.cic(pos, (8, 12, 16))
    assert rho.mean() == pytest.approx(1.0, abs=1e-13)
    assert rho.min() >= 0.0


def test_cic_centred_particle_and_translation():
    n = (8, 8, 8)
    pos = np.array([[(3 + 0.5) / 8, (5 + 0.5) / 8, (1 + 0.5) / 8]])
    rho = O.cic(pos, n)
    assert rho[1, 5, 3] == pytest.approx(512.0, abs=1e-10)
    assert np.count_nonzero(np.abs(rho) > 1e-12) == 1
    pos2 = synth.uniform_positions(300, 4)
    r1 = O.cic(pos2, n)
    shifted = np.mod(pos2 + np.array([1.0 / 8, 0, 2.0 / 8]), 1.0)
    r2 = O.cic(shifted, n)
    assert np.abs(np.roll(r1, shift=(2, 0, 1), axis=(0, 1, 2)) - r2).max() < 1e-10


def test_cic_brute_force():
    n = (4, 6, 8)
    pos = synth.uniform_positions(40, 5)
    rho = O.cic(pos, n)
    ref = np.zeros(n)
    mass = np.prod(n) / len(pos)
    for p in pos:
        for k in range(n[0]):
            for j in range(n[1]):
                for i in range(n[2]):
                    w = mass
                    for d, (c, nd) in enumerate(((i, n[2]), (j, n[1]), (k, n[0]))):
                        dx = p[d] * nd - (c + 0.5)
                        dx -= nd * np.round(dx / nd)  # minimal image
                        w *= max(0.0, 1.0 - abs(dx))
                    ref[k, j, i] += w
    assert np.abs(rho - ref).max() < 1e-12


# ---------------------------------------------------------------- truncation error (Sec. V.B.2)
def test_truncation_error_vanishes_on_homogeneous_solution():
    P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)
    tau = O.truncation_error(np.zeros((8, 8, 8)), np.ones((8, 8, 8)), **P)
    assert np.abs(tau).max() == 0.0


def test_truncation_error_is_second_order():
    """For smooth fields tau^h = O(h^2): halving h divides its rms by ~4 (the
    coarse-grid operator at 2h against the restricted fine operator)."""
    P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)

    def fields(n):
        x = (np.arange(n) + 0.5) / n
        z, y, xx = np.meshgrid(x, x, x, indexing="ij")
        u = 0.6 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * y) + 0.3 * np.sin(2 * np.pi * z)
        rho = 1.0 + 0.4 * np.cos(2 * np.pi * (xx + z))
        return u, rho

    r = []
    for n in (16, 32, 64):
        u, rho = fields(n)
        r.append(np.sqrt(np.mean(O.truncation_error(u, rho, **P) ** 2)))
    assert 3.5 < r[0] / r[1] < 4.5 and 3.7 < r[1] / r[2] < 4.3
