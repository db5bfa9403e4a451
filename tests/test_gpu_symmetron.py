"""The symmetron solve on the GPU (fr_symmetron_solve) against the oracle
(oracle/symmetron.py): element by element on grids the oracle solves in
seconds, its pins through the GPU path (homogeneous closed forms, the FFT
solution of the linearised equation), a 256^3 solve checked by the oracle's
pointwise residual at sampled cells, host pointers and invalid input.

Tolerance: both sides stop at rms(L) <= tol; the linearised operator's
eigenvalues are bounded away from 0 on the positive branch (mass 2(1 - s rho)
or s rho - 1, plus the Laplacian), so |chi_gpu - chi_oracle| is of the order
of tol over that mass; 1e-7 at tol 1e-10 leaves a wide margin.
"""
import numpy as np
import pytest

from gpu_common import ctx, dev, host, torch  # noqa: F401
from oracle import symmetron as S
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu
P = dict(a=1.0, a_ssb=0.5, lambda0=1.0)


@pytest.fixture(scope="module")
def C():
    return ctx()


@pytest.mark.parametrize("shape,sigma,seed", [((32, 32, 32), 1.0, 71), ((16, 24, 40), 2.0, 72),
                                              ((64, 64, 64), 2.0, 73), ((8, 8, 8), 1.5, 74)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_symmetron_matches_oracle(C, shape, sigma, seed, prec):
    rho = synth.lognormal_density(shape, seed, sigma=sigma)
    box = 0.5 * shape[2]
    ref = S.solve(rho, box=box, tol=1e-10, **P)
    assert ref.converged
    chi = torch.empty(shape, dtype=torch.float64, device="cuda")
    st, s = C.symmetron(dev(rho), chi, box=box, tol=1e-10, prec=prec, initial_guess=0, **P)
    assert st == 0 and s.res_rms <= 1e-10, s.as_dict()
    err = float(np.abs(host(chi) - ref.chi).max())
    assert err <= 1e-7, err
    if prec == "fp64":
        # the same V-cycles as the oracle's, in the same order
        assert s.vcycles == ref.cycles
        assert s.hist[0] == pytest.approx(ref.hist[0], rel=1e-9)


@pytest.mark.parametrize("ncyc", [1, 3])
@pytest.mark.parametrize("shape,sigma,seed", [((32, 32, 32), 2.0, 91), ((16, 24, 40), 1.5, 92)])
def test_fp64_vcycles_match_oracle_iterates(C, shape, sigma, seed, ncyc):
    """After exactly ncyc FP64 V-cycles the GPU iterate equals the oracle's up
    to rounding: the same sweeps, restriction (the coarse density included),
    coarse operator, prolongation and coarsest rule, not only the same
    fixed point."""
    rho = synth.lognormal_density(shape, seed, sigma=sigma)
    box = 0.5 * shape[2]
    ref = S.solve(rho, box=box, tol=1e-30, max_cycles=ncyc, **P)
    assert ref.cycles == ncyc and not ref.converged
    chi = torch.empty(shape, dtype=torch.float64, device="cuda")
    st, s = C.symmetron(dev(rho), chi, box=box, tol=1e-30, prec="fp64", initial_guess=0,
                        max_vcycles=ncyc, **P)
    assert st == 4 and s.vcycles == ncyc, s.as_dict()  # FR_ENOCONV: the iterate is returned
    assert float(np.abs(host(chi) - ref.chi).max()) < 1e-10
    assert s.res_rms == pytest.approx(ref.hist[-1], rel=1e-6)


@pytest.mark.parametrize("tiling", [1, -1])
@pytest.mark.parametrize("shape,sigma,seed", [((32, 32, 32), 2.0, 81), ((48, 34, 66), 1.5, 82),
                                              ((16, 130, 20), 1.0, 83)])
def test_register_column_sweeps_match_oracle(C, shape, sigma, seed, tiling):
    """The mixed solve with its FP32 sweeps in the register-column kernel
    (64 x 8 tiles, ragged and narrow grids that wrap a tile) and with one
    launch per colour reaches the oracle's solution."""
    rho = synth.lognormal_density(shape, seed, sigma=sigma)
    box = 0.5 * shape[2]
    ref = S.solve(rho, box=box, tol=1e-10, **P)
    chi = torch.empty(shape, dtype=torch.float64, device="cuda")
    st, s = C.symmetron(dev(rho), chi, box=box, tol=1e-10, prec="mixed", initial_guess=0,
                        tiling=tiling, **P)
    assert st == 0 and s.res_rms <= 1e-10, s.as_dict()
    assert np.abs(host(chi) - ref.chi).max() <= 1e-7


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("a,expect", [(1.0, np.sqrt(1 - 0.125)), (0.4, 0.0)])
def test_homogeneous_closed_form(C, prec, a, expect):
    rng = np.random.default_rng(1)
    chi0 = rng.uniform(0.3, 1.5, (16, 16, 16))
    chi = dev(chi0)
    st, s = C.symmetron(dev(np.ones((16, 16, 16))), chi, box=8.0, a=a, a_ssb=0.5, lambda0=1.0,
                        tol=1e-12, prec=prec)
    assert st == 0, (s.vcycles, s.outer, list(s.hist[: s.nhist]))
    assert np.abs(host(chi) - expect).max() < 1e-10


def test_linear_limit_matches_fft(C):
    n, eps = 32, 1e-5
    g = synth.gaussian_random_field((n,) * 3, 3, sigma=1.0)
    rho = 1.0 + eps * g
    lin = S.linear_response(g, eps, box=16.0, **P)
    chi = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    st, s = C.symmetron(dev(rho), chi, box=16.0, tol=1e-12, prec="mixed", initial_guess=0, **P)
    assert st == 0
    dev_ = np.abs(lin - S.background(1.0, 0.5)).max()
    assert np.abs(host(chi) - lin).max() <= 1e-3 * dev_


def test_host_pointers_and_invalid_input(C):
    from paper_1110_1379_gb300 import frmg
    shape = (16, 16, 16)
    rho = synth.lognormal_density(shape, 75, sigma=1.0)
    ref = S.solve(rho, box=8.0, tol=1e-10, **P)
    chi = np.full(shape, 0.9)
    st, s = C.symmetron(rho, chi, box=8.0, tol=1e-10, prec="mixed", **P)
    assert st == 0 and np.abs(chi - ref.chi).max() <= 1e-7
    bad = rho.copy()
    bad[1, 2, 3] = -0.5
    with pytest.raises(frmg.FRError) as ei:
        C.symmetron(bad, np.ones(shape), box=8.0, **P)
    assert ei.value.status == frmg.FR_EINVAL
    with pytest.raises(frmg.FRError) as ei:
        C.symmetron(rho, np.ones(shape), box=8.0, a=1.0, a_ssb=0.5, lambda0=-1.0)
    assert ei.value.status == frmg.FR_EINVAL


def test_256_sampled_against_oracle_residual(C):
    """256^3 (0.5 Mpc/h cells, sigma 2): the oracle's L_i at sampled cells of
    the GPU solution stays within the solve's own max residual, and the
    local terms sum to zero (the face terms telescope) within N^3 tol."""
    n = 256
    rho = synth.lognormal_density((n,) * 3, 3000, sigma=2.0)
    chi = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    st, s = C.symmetron(dev(rho), chi, box=0.5 * n, tol=1e-8, prec="mixed", initial_guess=0, **P)
    assert st == 0 and s.res_rms <= 1e-8
    x = host(chi)
    A, sv = S.coefficients(0.5 * n, n, **P)
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(300):
        k, j, i = (int(v) for v in rng.integers(0, n, 3))
        ks, js, is_ = ((np.arange(-1, 2) + c) % n for c in (k, j, i))
        blk = x[np.ix_(ks, js, is_)]
        rb = rho[np.ix_(ks, js, is_)]
        worst = max(worst, abs(S.operator(blk, rb, A, sv)[1, 1, 1]))
    assert worst <= s.res_max * (1 + 1e-6) + 1e-12
    loc = float(np.sum((sv * rho - 1.0) * x + x ** 3))
    assert abs(loc) <= n ** 3 * 1e-8
    assert (x > 0).all() and x.max() < 1.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overflowing_start_reports_divergence(C, prec):
    """A start with one cell at 1e120 overflows the cubic term: the solve
    reports FR_EDIVERGED (made on the host side, nothing faults) and the
    context keeps working."""
    from paper_1110_1379_gb300 import frmg
    shape = (16, 16, 16)
    rho = dev(synth.lognormal_density(shape, 76, sigma=1.0))
    chi0 = np.full(shape, 0.9)
    chi0[3, 4, 5] = 1e120
    chi = dev(chi0)
    st, s = C.symmetron(rho, chi, box=8.0, prec=prec, **P)
    assert st == frmg.FR_EDIVERGED
    assert b"non-finite" in frmg.load().fr_last_error()
    chi.fill_(0.9)
    st, s = C.symmetron(rho, chi, box=8.0, prec=prec, **P)
    assert st == 0
