"""GPU particle-mesh steps (fr_tsc_assign, fr_cic_assign, fr_particle_forces) against
the oracle (oracle/particles.py).

Tolerance: the GPU deposits with FP64 atomics in an order that varies, so sums
of up to 27 x (particles per cell) terms agree to ~1e-15 relative per term:
1e-12 of the largest value is allowed.  Forces are sums of 81 products in a
fixed order on both sides (different association): 1e-12 relative.
"""
import numpy as np
import pytest

from gpu_common import ctx, dev, host, torch  # noqa: F401
from oracle import particles as PM
from oracle import poisson as PO
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    return ctx()


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
@pytest.mark.parametrize("shape", [(16, 24, 32), (8, 8, 8), (6, 10, 4)])
def test_assignment_matches_oracle(C, scheme, shape):
    rng = np.random.default_rng(5)
    pos = rng.random((20000, 3))
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    getattr(C, scheme)(dev(pos), out)
    ref = PM.assign(pos, shape, scheme)
    got = host(out)
    assert np.abs(got - ref).max() <= 1e-12 * ref.max()
    assert got.mean() == pytest.approx(1.0, rel=1e-13)


def test_tsc_full_zeldovich_lattice(C):
    """The 128^3 CIC workload's particles (Zel'dovich, slope -2.5, amplitude
    60: max(rho~ - 1) of about 100) with TSC."""
    n = 128
    pos = synth.zeldovich_positions(n, 2000, amplitude=synth.ZELDOVICH_AMPLITUDE_128,
                                    slope=synth.ZELDOVICH_SLOPE_128)
    out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    C.tsc(dev(pos), out)
    ref = PM.assign(pos, (n, n, n), "tsc")
    got = host(out)
    assert np.abs(got - ref).max() <= 1e-12 * ref.max()
    assert got.mean() == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
def test_forces_match_oracle(C, scheme):
    rng = np.random.default_rng(6)
    shape = (16, 24, 32)
    phi = synth.gaussian_random_field(shape, 7, sigma=1.0)
    pos = rng.random((5000, 3))
    out = torch.empty((5000, 3), dtype=torch.float64, device="cuda")
    C.forces(dev(phi), dev(pos), out, scheme=scheme)
    ref = PM.forces(phi, pos, scheme)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
def test_no_self_force_through_gpu_steps(C, scheme):
    """GPU assignment and interpolation around the exact periodic Poisson solve:
    a lone particle feels no force from its own cloud."""
    rng = np.random.default_rng(8)
    shape = (16, 16, 16)
    p = rng.random((1, 3))
    rho = torch.empty(shape, dtype=torch.float64, device="cuda")
    getattr(C, scheme)(dev(p), rho)
    phi, _ = PO.solve_periodic(host(rho) - 1.0, 1.0 / 16)
    f = torch.empty((1, 3), dtype=torch.float64, device="cuda")
    C.forces(dev(phi), dev(p), f, scheme=scheme)
    assert np.abs(host(f)).max() < 1e-12 * np.abs(PM.gradient(phi)[0]).max()


def test_host_pointers_and_invalid_positions(C):
    rng = np.random.default_rng(9)
    shape = (8, 8, 8)
    pos = rng.random((300, 3))
    phi = rng.standard_normal(shape)
    f_host = torch.empty((300, 3), dtype=torch.float64)
    C.forces(torch.from_numpy(phi), torch.from_numpy(pos), f_host, scheme="tsc")
    assert np.abs(f_host.numpy() - PM.forces(phi, pos, "tsc")).max() <= 1e-12 * np.abs(f_host.numpy()).max()
    rho_h = torch.empty(shape, dtype=torch.float64)
    C.tsc(torch.from_numpy(pos), rho_h)
    assert np.abs(rho_h.numpy() - PM.assign(pos, shape, "tsc")).max() < 1e-12 * rho_h.numpy().max()
    from paper_1110_1379_gb300 import frmg
    bad = pos.copy()
    bad[7, 1] = 1.0
    with pytest.raises(frmg.FRError):
        C.tsc(dev(bad), torch.empty(shape, dtype=torch.float64, device="cuda"))
    with pytest.raises(frmg.FRError):
        C.forces(dev(phi), dev(bad), torch.empty((300, 3), dtype=torch.float64, device="cuda"))
