"""GPU modified-Poisson solve (fr_poisson_solve / fr_poisson_source) against the oracle.

Tolerances:
* source: double-float evaluation (~48-bit) of the same formula: |ds| <= 1e-12 (1 + |s|);
* periodic solve at rms(L phi - s) <= tol: the error e satisfies L e = d, and on
  a periodic grid (zero-mean e) |e|_rms <= |d|_rms / lambda_min with
  lambda_min = 4 sin^2(pi/N)/h^2 ~ 4 pi^2 (box side 1), so |e|_rms <= tol/39;
  the tests allow max|e| <= 100 tol/39 (pointwise vs rms margin);
* patch solve: the same bound with the patch's lowest Dirichlet eigenvalue
  (>= 3 pi^2 / L^2 for a cube of side L = n h), checked the same way.
"""
import numpy as np
import pytest

from gpu_common import ctx, dev, host, torch  # noqa: F401
from oracle import oracle as O
from oracle import poisson as PO
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu

P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)


@pytest.fixture(scope="module")
def C():
    return ctx()


def _u_field(shape, seed, amp=1.5):
    # smooth synthetic f(R) variable (the Poisson equation only reads it)
    g = synth.gaussian_random_field(shape, seed, sigma=1.0)
    return amp * g - 0.5


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 20, 36), (2, 4, 6)])
def test_source_matches_oracle(C, shape):
    rho = synth.lognormal_density(shape, 31, sigma=1.5)
    u = _u_field(shape, 32)
    out = torch.zeros(shape, dtype=torch.float64, device="cuda")
    C.poisson_source(dev(rho), dev(u), out, **P)
    ref = PO.source(u, rho, **P)
    assert np.abs(host(out) - ref).max() <= 1e-12 * (1 + np.abs(ref).max())


@pytest.mark.parametrize("shape", [(32, 32, 32), (12, 20, 36), (16, 8, 24)])
def test_periodic_solve_matches_fft_oracle(C, shape):
    rho = synth.lognormal_density(shape, 41, sigma=1.2)
    u = _u_field(shape, 42)
    h = 1.0 / shape[2]
    s = PO.source(u, rho, **P)
    ref, mean = PO.solve_periodic(s, h)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-10
    st, stats, gmean = C.poisson(dev(rho), dev(u), phi, tol=tol, **P)
    assert st == 0 and stats.res_rms <= tol
    assert gmean == pytest.approx(mean, abs=1e-12)
    got = host(phi)
    assert abs(got.mean()) < 1e-12
    assert np.abs(got - ref).max() <= 100 * tol / 39.0
    # the oracle's residual of the GPU solution
    assert np.sqrt(np.mean(PO.residual(got, s - mean, h) ** 2)) <= 2 * tol


def test_manufactured_eigenmode(C):
    """rho chosen so that s = L phi* for a lattice Fourier mode phi* (u = 0 gives
    s = 2 gamma (rho - 1)); the solve must return phi*."""
    shape = (24, 16, 32)
    n2, n1, n0 = shape
    h = 1.0 / n0
    k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    ks = (2, 1, 3)  # integer wave numbers along z, y, x
    arg = 2 * np.pi * (ks[0] * k / n2 + ks[1] * j / n1 + ks[2] * i / n0)
    phistar = 1e-3 * np.cos(arg + 0.4)
    lam = -4.0 / h ** 2 * (np.sin(np.pi * ks[0] / n2) ** 2 + np.sin(np.pi * ks[1] / n1) ** 2
                           + np.sin(np.pi * ks[2] / n0) ** 2)
    gamma = P["omega_m"] * P["a"]
    rho = 1.0 + lam * phistar / (2 * gamma)
    u = np.zeros(shape)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, stats, gmean = C.poisson(dev(rho), dev(u), phi, tol=1e-11,
                                 allow_negative_density=1, **P)
    assert st == 0
    assert abs(gmean) < 1e-12
    assert np.abs(host(phi) - phistar).max() <= 100 * 1e-11 / 39.0


@pytest.mark.parametrize("shape", [(16, 12, 20), (8, 8, 8)])
def test_patch_solve_matches_direct_solve(C, shape):
    rng = np.random.default_rng(9)
    rho = synth.lognormal_density(shape, 51, sigma=0.8)
    u = _u_field(shape, 52, amp=0.5)
    h = 1.0 / 128
    phib = rng.uniform(-1e-3, 1e-3, sum(O.face_sizes(shape)))
    s = PO.source(u, rho, **P)
    ref = PO.solve_patch(s, phib, h)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-8
    st, stats, gmean = C.poisson(dev(rho), dev(u), phi, tol=tol, phib=dev(phib), h=h, **P)
    assert st == 0 and stats.res_rms <= tol
    got = host(phi)
    side = min(shape) * h
    lam_min = 3 * np.pi ** 2 / side ** 2
    assert np.abs(got - ref).max() <= 100 * tol / lam_min
    assert np.sqrt(np.mean(PO.residual(got, s, h, phib) ** 2)) <= 2 * tol


def test_host_pointers_and_initial_guess(C):
    shape = (16, 16, 16)
    rho = synth.lognormal_density(shape, 61, sigma=1.0)
    u = _u_field(shape, 62)
    phi_d = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s1, m1 = C.poisson(dev(rho), dev(u), phi_d, tol=1e-10, **P)
    phi_h = torch.zeros(shape, dtype=torch.float64)
    st2, s2, m2 = C.poisson(torch.from_numpy(rho), torch.from_numpy(u), phi_h, tol=1e-10, **P)
    assert st == 0 and st2 == 0
    assert np.abs(host(phi_d) - phi_h.numpy()).max() < 1e-13
    # restarting from the solution converges at once
    st3, s3, _ = C.poisson(dev(rho), dev(u), phi_d, tol=1e-10, **P)
    assert st3 == 0 and s3.vcycles == 0 and s3.outer == 1


def test_invalid_arguments(C):
    rho = torch.ones((8, 8, 8), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(rho)
    phi = torch.zeros((8, 8, 7), dtype=torch.float64, device="cuda")
    from paper_1110_1379_gb300 import frmg
    with pytest.raises(frmg.FRError):
        C.poisson(rho, u, phi, **P)
    phi = torch.zeros_like(rho)
    with pytest.raises(frmg.FRError):
        C.poisson(rho, u, phi, tol=-1.0, **P)


def test_full_size_workload_sampled(C):
    """512^3 (the bench workload): f(R) solve, then the Poisson solve; the
    oracle's formulas evaluated at sampled cells give residuals <= 10 tol, and
    phi has zero mean."""
    n = 512
    shape = (n, n, n)
    PH = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    rho_np = synth.lognormal_density(shape, 3000, sigma=2.0)
    rho = dev(rho_np)
    u = torch.zeros_like(rho)
    st, s = C.solve(rho, u, tol=1e-8, prec="mixed", **PH)
    assert st == 0
    phi = torch.zeros_like(rho)
    tol = 1e-8
    st, ps, mean = C.poisson(rho, u, phi, tol=tol, **PH)
    assert st == 0 and ps.res_rms <= tol
    rng = np.random.default_rng(3)
    cells = rng.integers(0, n, size=(64, 3))
    h = 1.0 / n
    un = host(u)
    ph = host(phi)
    assert abs(ph.mean()) < 1e-10
    for (k, j, i) in cells:
        nb = (ph[k, j, (i + 1) % n] + ph[k, j, (i - 1) % n] + ph[k, (j + 1) % n, i]
              + ph[k, (j - 1) % n, i] + ph[(k + 1) % n, j, i] + ph[(k - 1) % n, j, i])
        lap = (nb - 6 * ph[k, j, i]) / h ** 2
        src = PO.source(un[k:k + 1, j:j + 1, i:i + 1], rho_np[k:k + 1, j:j + 1, i:i + 1],
                        **PH)[0, 0, 0]
        assert abs(lap - (src - mean)) <= 10 * tol + 1e-12 * abs(src)


def test_periodic_solve_tiled_levels_match_fft_oracle(C):
    """128^3: the fine and 64^3 levels use the tiled smoother."""
    shape = (128, 128, 128)
    rho = synth.lognormal_density(shape, 71, sigma=1.5)
    u = _u_field(shape, 72)
    h = 1.0 / shape[2]
    s = PO.source(u, rho, **P)
    ref, mean = PO.solve_periodic(s, h)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-9
    st, stats, gmean = C.poisson(dev(rho), dev(u), phi, tol=tol, **P)
    assert st == 0 and stats.res_rms <= tol
    assert np.abs(host(phi) - ref).max() <= 100 * tol / 39.0


def test_patch_solve_tiled_satisfies_oracle_equation(C):
    """A patch large enough for the tiled smoother; by uniqueness of the
    Dirichlet problem, a small oracle residual fixes the solution."""
    shape = (48, 64, 64)
    rng = np.random.default_rng(13)
    rho = synth.lognormal_density(shape, 81, sigma=1.0)
    u = _u_field(shape, 82, amp=0.5)
    h = 1.0 / 256
    phib = rng.uniform(-1e-3, 1e-3, sum(O.face_sizes(shape)))
    s = PO.source(u, rho, **P)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-8
    st, stats, _ = C.poisson(dev(rho), dev(u), phi, tol=tol, phib=dev(phib), h=h, **P)
    assert st == 0 and stats.res_rms <= tol
    assert np.sqrt(np.mean(PO.residual(host(phi), s, h, phib) ** 2)) <= 2 * tol


@pytest.mark.parametrize("relax", [1.15, 1.3])
def test_over_relaxed_poisson_solve_matches_fft_oracle(C, relax):
    """Over-relaxed red-black sweeps (periodic, tiled levels) and a patch reach
    the same discrete solutions."""
    shape = (64, 64, 64)
    rho = synth.lognormal_density(shape, 91, sigma=1.5)
    u = _u_field(shape, 92)
    h = 1.0 / shape[2]
    s = PO.source(u, rho, **P)
    ref, mean = PO.solve_periodic(s, h)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-9
    st, stats, gmean = C.poisson(dev(rho), dev(u), phi, tol=tol, relax=relax, **P)
    assert st == 0 and stats.res_rms <= tol
    assert np.abs(host(phi) - ref).max() <= 100 * tol / 39.0
    shp = (16, 12, 20)
    rng = np.random.default_rng(93)
    rp = synth.lognormal_density(shp, 94, sigma=0.8)
    up = _u_field(shp, 95, amp=0.5)
    phib = rng.uniform(-1e-3, 1e-3, sum(O.face_sizes(shp)))
    hp = 1.0 / 128
    refp = PO.solve_patch(PO.source(up, rp, **P), phib, hp)
    phip = torch.zeros(shp, dtype=torch.float64, device="cuda")
    st, stats, _ = C.poisson(dev(rp), dev(up), phip, tol=1e-8, phib=dev(phib), h=hp,
                             relax=relax, **P)
    assert st == 0
    assert np.abs(host(phip) - refp).max() <= 100 * 1e-8 / (3 * np.pi ** 2 / (12 * hp) ** 2)


@pytest.mark.parametrize("patch", [False, True])
def test_ragged_tiles_match_oracle(C, patch):
    """A fine level whose tiles (64 x 16) are cut by the grid edge in x and y,
    smoothed and corrected by the tiled kernels."""
    shape = (40, 72, 96)
    rho = synth.lognormal_density(shape, 101, sigma=1.2)
    u = _u_field(shape, 102, amp=0.5)
    h = 1.0 / 256 if patch else 1.0 / shape[2]
    s = PO.source(u, rho, **P)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tol = 1e-9
    if patch:
        rng = np.random.default_rng(103)
        phib = rng.uniform(-1e-3, 1e-3, sum(O.face_sizes(shape)))
        st, stats, _ = C.poisson(dev(rho), dev(u), phi, tol=tol, phib=dev(phib), h=h,
                                 relax=1.2, **P)
        assert st == 0 and stats.res_rms <= tol
        assert np.sqrt(np.mean(PO.residual(host(phi), s, h, phib) ** 2)) <= 2 * tol
    else:
        ref, mean = PO.solve_periodic(s, h)
        st, stats, _ = C.poisson(dev(rho), dev(u), phi, tol=tol, relax=1.2, **P)
        assert st == 0 and stats.res_rms <= tol
        assert np.abs(host(phi) - ref).max() <= 100 * tol / 39.0
