"""GPU general mask scheme (fr_solve_masked) against the masked-region oracle.

Both sides run the same FP64 algorithm (red-black Newton-Gauss-Seidel, masked
FAS levels), so residual histories agree to rounding and the solutions to
well below the tolerance; converged solutions are also compared with the
closed-form spherical Gaussian and with the box-patch solve of the C oracle
(the unique discrete solution of the same equations)."""
import numpy as np
import pytest

import paper_fields as PF
from gpu_common import ctx, dev, host, torch  # noqa: F401
from oracle import masked as M
from oracle import oracle as O

pytestmark = pytest.mark.gpu

P = dict(box=128.0, a=0.9, omega_m=0.24, fr0=1e-5)


@pytest.fixture(scope="module")
def C():
    return ctx()


def _blob_region(n, seed):
    """Irregular active set (a noisy blob) with masks +-1 and, on 15 % of the
    cells, +-0.5 (ghost ratios r in {-2, -1, -1/2, 0-}); coarser levels add the
    fractional masks of the restriction."""
    rng = np.random.default_rng(seed)
    k, j, i = np.indices((n, n, n))
    c = (n - 1) / 2
    r2 = ((i - c) ** 2 + (j - c) ** 2 + (k - c) ** 2) / (0.1 * n * n)
    blob = np.exp(-r2) + 0.25 * rng.uniform(-1, 1, (n, n, n))
    m = np.where(blob > 0.45, 1.0, -1.0)
    m = np.where(rng.uniform(size=(n, n, n)) < 0.15, 0.5 * m, m)
    m[[0, -1]], m[:, [0, -1]], m[:, :, [0, -1]] = -1.0, -1.0, -1.0
    u0 = 0.2 * np.sin(0.4 * i) * np.cos(0.3 * j) + 0.1 * np.cos(0.5 * k)
    rho = np.exp(rng.normal(0, 0.5, (n, n, n)))
    return m, u0, rho


@pytest.mark.parametrize("n,seed", [(16, 6), (32, 7), (24, 8)])
def test_irregular_region_matches_oracle(C, n, seed):
    """Irregular active set with fractional masks."""
    m, u0, rho = _blob_region(n, seed)
    h = 1.0 / (4 * n)
    ref = M.solve(u0, m, rho, h=h, tol=1e-11, **P)
    assert ref.converged
    u = dev(u0)
    st, s = C.solve_masked(dev(rho), dev(m), u, h=h, tol=1e-11, **P)
    assert st == 0 and s.res_rms <= 1e-11
    assert s.vcycles == ref.cycles
    # same iterates up to rounding: the residuals agree to the rounding floor of
    # the operator's terms (about 1e-12 of the initial residual here)
    np.testing.assert_allclose(list(s.hist[: s.nhist]), ref.hist, rtol=1e-6,
                               atol=1e-12 * ref.hist[0])
    got = host(u)
    act = m > 0
    assert np.abs(got[act] - ref.u[act]).max() < 1e-10
    assert np.array_equal(got[~act], u0[~act])  # ghosts untouched


def test_spherical_region_matches_oracle_and_closed_form(C):
    G = dict(amp=0.9, width=0.08, centre=(0.5, 0.5, 0.5))
    N, nb = 128, 48
    lo = N // 2 - nb // 2
    rho, ue = PF.spherical_gaussian_patch(lo, nb, N, **P, **G)
    x = (np.arange(lo, lo + nb) + 0.5) / N
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    m = np.where(np.sqrt((xx - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) < 0.15, 1.0, -1.0)
    ref = M.solve(ue, m, rho, h=1.0 / N, tol=1e-10, **P)
    u = dev(ue)
    st, s = C.solve_masked(dev(rho), dev(m), u, h=1.0 / N, tol=1e-10, **P)
    assert st == 0 and s.vcycles == ref.cycles
    got = host(u)
    act = m > 0
    assert np.abs(got[act] - ref.u[act]).max() < 1e-10
    err_gpu = np.abs(got - ue)[act].max()
    err_ref = np.abs(ref.u - ue)[act].max()
    assert err_gpu == pytest.approx(err_ref, rel=1e-6)


def test_box_mask_equals_patch_solve(C):
    """Masks +1 inside, -1 on the outer layer: the converged region equals the
    C oracle's refinement-patch solve with u_b = (ghost + first interior)/2."""
    shape = (18, 26, 34)  # interior 16 x 24 x 32: several patch levels
    rng = np.random.default_rng(11)
    rho = np.exp(rng.normal(0, 0.6, shape))
    k, j, i = np.indices(shape)
    u0 = 0.3 * np.sin(0.2 * i + 0.1 * j) * np.cos(0.15 * k)
    m = -np.ones(shape)
    m[1:-1, 1:-1, 1:-1] = 1.0
    h = 1.0 / 96
    u = dev(u0)
    st, s = C.solve_masked(dev(rho), dev(m), u, h=h, tol=1e-10, **P)
    assert st == 0
    I = (slice(1, -1),) * 3
    mid = lambda a, b: 0.5 * (a + b)
    faces = np.concatenate([f.ravel() for f in (
        mid(u0[1:-1, 1:-1, 0], u0[1:-1, 1:-1, 1]), mid(u0[1:-1, 1:-1, -1], u0[1:-1, 1:-1, -2]),
        mid(u0[1:-1, 0, 1:-1], u0[1:-1, 1, 1:-1]), mid(u0[1:-1, -1, 1:-1], u0[1:-1, -2, 1:-1]),
        mid(u0[0, 1:-1, 1:-1], u0[1, 1:-1, 1:-1]), mid(u0[-1, 1:-1, 1:-1], u0[-2, 1:-1, 1:-1]))])
    ref = O.solve(rho[I], u0=u0[I], h=h, ub=faces, tol=1e-10, **P)
    assert ref.converged
    assert np.abs(host(u)[I] - ref.u).max() < 1e-8


def test_host_pointers_relaxation_and_limits(C):
    m, u0, rho = _blob_region(16, 12)
    h = 1.0 / 64
    ud = dev(u0)
    st, s = C.solve_masked(dev(rho), dev(m), ud, h=h, tol=1e-10, **P)
    assert st == 0
    uh = torch.from_numpy(u0.copy())
    st2, s2 = C.solve_masked(torch.from_numpy(rho), torch.from_numpy(m), uh, h=h, tol=1e-10, **P)
    assert st2 == 0 and s2.vcycles == s.vcycles
    assert np.array_equal(uh.numpy(), host(ud))
    # over-relaxed sweeps reach the same discrete solution
    ur = dev(u0)
    st3, s3 = C.solve_masked(dev(rho), dev(m), ur, h=h, tol=1e-10, relax=1.15, **P)
    assert st3 == 0
    act = m > 0
    assert np.abs(host(ur)[act] - host(ud)[act]).max() < 1e-8
    # V-cycle limit
    from paper_1110_1379_gb300 import frmg
    st4, s4 = C.solve_masked(dev(rho), dev(m), dev(u0), h=h, tol=1e-14, max_vcycles=1, **P)
    assert st4 == frmg.FR_ENOCONV and s4.vcycles == 1


def test_invalid_regions_rejected(C):
    from paper_1110_1379_gb300 import frmg
    m, u0, rho = _blob_region(16, 13)
    bad = m.copy()
    bad[0, 5, 5] = 0.5  # active cell on the outer layer
    with pytest.raises(frmg.FRError) as e:
        C.solve_masked(dev(rho), dev(bad), dev(u0), h=1.0 / 64, **P)
    assert e.value.status == frmg.FR_EINVAL
    bad = m.copy()
    bad[5, 5, 5] = 1.5
    with pytest.raises(frmg.FRError):
        C.solve_masked(dev(rho), dev(bad), dev(u0), h=1.0 / 64, **P)
    r = rho.copy()
    r[4, 4, 4] = np.nan
    with pytest.raises(frmg.FRError):
        C.solve_masked(dev(r), dev(m), dev(u0), h=1.0 / 64, **P)
    with pytest.raises(frmg.FRError):
        C.solve_masked(dev(rho), dev(m), dev(u0), h=-1.0, **P)


@pytest.mark.parametrize("n,seed", [(32, 7), (24, 8)])
def test_mixed_precision_reaches_the_oracle_solution(C, n, seed):
    """prec='mixed': FP32 V-cycles of the same scheme, then FP64 ones; the
    FP64 residual meets tol and the solution is the oracle's (the unique
    discrete solution), with the ghosts untouched."""
    m, u0, rho = _blob_region(n, seed)
    h = 1.0 / (4 * n)
    ref = M.solve(u0, m, rho, h=h, tol=1e-11, **P)
    assert ref.converged
    u = dev(u0)
    st, s = C.solve_masked(dev(rho), dev(m), u, h=h, tol=1e-10, prec="mixed", **P)
    assert st == 0 and s.res_rms <= 1e-10 and s.outer >= 1
    hist = list(s.hist[: s.nhist])
    # first entry the FP64 start, then FP32 cycles (positive), then FP64
    # evaluations (negated)
    k = next(i for i, v in enumerate(hist) if v < 0)
    assert k >= 2 and all(v > 0 for v in hist[:k]) and all(v < 0 for v in hist[k:])
    assert -hist[-1] == pytest.approx(s.res_rms, rel=1e-12)
    got = host(u)
    act = m > 0
    assert np.abs(got[act] - ref.u[act]).max() < 1e-9
    assert np.array_equal(got[~act], u0[~act])


def test_mixed_precision_equals_fp64_solve_on_sphere_union(C):
    """A union of spheres in a 64^3 box (the masked bench recipe, smaller):
    the mixed and the FP64 solves reach the same solution."""
    from paper_1110_1379_gb300 import synth
    n = 64
    rho = synth.lognormal_density((n, n, n), 77, sigma=1.5)
    m = synth.sphere_union_mask(rho, 6, (4, 10), 78, margin=6)
    h = 1.0 / (2 * n)
    u64, umx = dev(np.zeros_like(rho)), dev(np.zeros_like(rho))
    st, s = C.solve_masked(dev(rho), dev(m), u64, h=h, tol=1e-9, **P)
    st2, s2 = C.solve_masked(dev(rho), dev(m), umx, h=h, tol=1e-9, prec="mixed", **P)
    assert st == 0 and st2 == 0 and s2.res_rms <= 1e-9
    act = m > 0
    assert np.abs(host(u64)[act] - host(umx)[act]).max() < 1e-8


def test_mixed_precision_respects_the_cycle_limit(C):
    """The V-cycle limit counts the FP32 and the FP64 cycles together."""
    from paper_1110_1379_gb300 import frmg
    m, u0, rho = _blob_region(16, 14)
    st, s = C.solve_masked(dev(rho), dev(m), dev(u0), h=1.0 / 64, tol=1e-14, max_vcycles=3,
                           prec="mixed", **P)
    assert st == frmg.FR_ENOCONV and s.vcycles == 3
