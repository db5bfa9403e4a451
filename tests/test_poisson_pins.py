"""Pins of the modified-Poisson oracle (oracle/poisson.py) to things other than itself.

* the FFT solver against the stencil (independent: spectral vs real space);
* the stencil against explicit neighbour sums at chosen cells (brute force);
* the patch ghost rule: exact for linear fields (closed form: Laplacian 0);
* the patch direct solver against a dense matrix built from the stencil applied
  to unit vectors (brute force on a tiny grid);
* the source in its two closed-form limits: delta R = 0 (u = 0) gives
  2 Om a (rho - 1), the screened limit gives the GR source 1.5 Om a (rho - 1);
* consistency of Eq. (discrete_poisson) with Eq. (discrete_fR): at a converged
  f(R) solution the mean of the Poisson source is 1.5 Om a (mean rho - 1).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import poisson as PO
from paper_1110_1379_gb300 import synth

P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 20, 8), (6, 10, 14)])
def test_fft_solution_satisfies_stencil(shape):
    rng = np.random.default_rng(3)
    h = 1.0 / shape[2]
    s = rng.standard_normal(shape)
    phi, mean = PO.solve_periodic(s, h)
    assert abs(mean - s.mean()) < 1e-15
    assert abs(phi.mean()) < 1e-12
    r = PO.laplacian(phi, h) - (s - mean)
    assert np.abs(r).max() < 1e-9 * np.abs(s).max()


def test_stencil_explicit_sums():
    rng = np.random.default_rng(5)
    shape = (6, 8, 10)
    h = 0.1
    phi = rng.standard_normal(shape)
    L = PO.laplacian(phi, h)
    n2, n1, n0 = shape
    for (k, j, i) in [(0, 0, 0), (5, 7, 9), (2, 3, 4), (0, 7, 4)]:
        nb = (phi[k, j, (i + 1) % n0] + phi[k, j, (i - 1) % n0] + phi[k, (j + 1) % n1, i]
              + phi[k, (j - 1) % n1, i] + phi[(k + 1) % n2, j, i] + phi[(k - 1) % n2, j, i])
        assert L[k, j, i] == pytest.approx((nb - 6 * phi[k, j, i]) / h ** 2, rel=1e-14, abs=1e-12)


def _linear_with_faces(shape, h, c):
    n2, n1, n0 = shape
    z, y, x = np.meshgrid((np.arange(n2) + 0.5) * h, (np.arange(n1) + 0.5) * h,
                          (np.arange(n0) + 0.5) * h, indexing="ij")
    f = lambda X, Y, Z: c[0] + c[1] * X + c[2] * Y + c[3] * Z  # noqa: E731
    phi = f(x, y, z)
    # face values at the face centres of the boundary cells, packed -x,+x,-y,+y,-z,+z
    zz, yy = np.meshgrid((np.arange(n2) + 0.5) * h, (np.arange(n1) + 0.5) * h, indexing="ij")
    zx, xx = np.meshgrid((np.arange(n2) + 0.5) * h, (np.arange(n0) + 0.5) * h, indexing="ij")
    yx, xy = np.meshgrid((np.arange(n1) + 0.5) * h, (np.arange(n0) + 0.5) * h, indexing="ij")
    faces = [f(0.0, yy, zz), f(n0 * h, yy, zz), f(xx, 0.0, zx), f(xx, n1 * h, zx),
             f(xy, yx, 0.0), f(xy, yx, n2 * h)]
    return phi, np.concatenate([a.ravel() for a in faces])


def test_patch_ghost_rule_exact_for_linear_fields():
    shape, h = (6, 8, 10), 0.05
    phi, phib = _linear_with_faces(shape, h, [0.3, 1.7, -2.1, 0.9])
    L = PO.laplacian(phi, h, phib)
    assert np.abs(L).max() < 1e-9


def test_patch_solver_against_dense_stencil_matrix():
    rng = np.random.default_rng(11)
    shape, h = (4, 4, 6), 0.25
    ncell = int(np.prod(shape))
    s = rng.standard_normal(shape)
    phib = rng.standard_normal(sum(O.face_sizes(shape)))
    # the BC-modified operator is affine in phi: columns from unit vectors
    zero = np.zeros(shape)
    c0 = PO.laplacian(zero, h, phib).ravel()
    A = np.empty((ncell, ncell))
    for q in range(ncell):
        e = np.zeros(ncell)
        e[q] = 1.0
        A[:, q] = PO.laplacian(e.reshape(shape), h, phib).ravel() - c0
    ref = np.linalg.solve(A, s.ravel() - c0).reshape(shape)
    got = PO.solve_patch(s, phib, h)
    assert np.abs(got - ref).max() < 1e-10
    assert np.abs(PO.residual(got, s, h, phib)).max() < 1e-9


@pytest.mark.parametrize("a", [0.5, 1.0])
def test_source_limits(a):
    rng = np.random.default_rng(7)
    rho = np.exp(rng.normal(0, 0.4, (8, 8, 8)))
    om = 0.24
    ol = 1 - om
    # delta R = 0 (u = 0): the unscreened source, 4/3 of the GR one
    s0 = PO.source(np.zeros_like(rho), rho, box=64.0, a=a, omega_m=om, fr0=1e-5)
    assert np.abs(s0 - 2 * om * a * (rho - 1)).max() < 1e-12
    # screened limit (alpha -> 0 pointwise solution of Eq. discrete_fR):
    # beta (e^{-u/2} - 1) = gamma (rho - 1) gives the GR source 1.5 Om a (rho - 1)
    beta = om * a ** 4 * (a ** -3 + 4 * ol / om)
    gamma = om * a
    u = -2.0 * np.log(1.0 + gamma * (rho - 1) / beta)
    s1 = PO.source(u, rho, box=64.0, a=a, omega_m=om, fr0=1e-5)
    assert np.abs(s1 - 1.5 * om * a * (rho - 1)).max() < 1e-12


def test_source_mean_at_converged_fR_solution():
    shape = (16, 16, 16)
    rho = synth.lognormal_density(shape, 77, sigma=0.8) * 1.05  # mean 1.05
    r = O.solve(rho, tol=1e-12, **P)
    s = PO.source(r.u, rho, **P)
    gamma = P["omega_m"] * P["a"]
    assert s.mean() == pytest.approx(1.5 * gamma * (rho.mean() - 1.0), abs=1e-10)
