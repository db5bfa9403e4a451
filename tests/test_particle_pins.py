"""Pins of the particle-mesh oracle (oracle/particles.py).

* mass: the mean assigned density is 1 (the check of Sec. VI.C);
* a particle at a cell centre deposits the closed-form TSC weights
  (1/8, 3/4, 1/8) per axis (CIC: all its mass into that cell);
* translating every particle by one cell translates the density exactly;
* TSC equals CIC convolved with the cell top-hat along each axis (the TSC
  cloud is the CIC cloud widened by one cell);
* the central-difference gradient of a lattice cosine mode in closed form;
* same-scheme force interpolation: a particle at a cell centre feels the
  closed-form weighted gradient; a lone particle feels no force from its own
  density (self-force 0) and a pair feels equal and opposite forces, with Phi
  from the exact FFT Poisson solve (momentum conservation).
"""
import numpy as np
import pytest

from oracle import particles as PM
from oracle import poisson as PO


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
def test_mass_conservation(scheme):
    rng = np.random.default_rng(1)
    pos = rng.random((3000, 3))
    rho = PM.assign(pos, (8, 12, 16), scheme)
    assert rho.mean() == pytest.approx(1.0, rel=1e-14)
    assert rho.min() >= 0.0


def test_cell_centre_weights():
    shape = (8, 8, 8)
    pos = np.array([[(3 + 0.5) / 8, (5 + 0.5) / 8, (6 + 0.5) / 8]])
    rho = PM.assign(pos, shape, "tsc") / 512.0  # one particle of mass 512
    w = np.array([1 / 8, 3 / 4, 1 / 8])
    ref = np.zeros(shape)
    for a, i in enumerate((2, 3, 4)):
        for b, j in enumerate((4, 5, 6)):
            for c, k in enumerate((5, 6, 7)):
                ref[k, j, i] = w[a] * w[b] * w[c]
    assert np.abs(rho - ref).max() < 1e-15
    rho_c = PM.assign(pos, shape, "cic") / 512.0
    assert rho_c[6, 5, 3] == pytest.approx(1.0, abs=1e-15) and rho_c.sum() == pytest.approx(1.0)


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
def test_translation_by_one_cell(scheme):
    rng = np.random.default_rng(2)
    shape = (6, 10, 8)
    pos = rng.random((500, 3))
    rho = PM.assign(pos, shape, scheme)
    shifted = np.mod(pos + np.array([1 / 8, 0, 2 / 6]), 1.0)
    rho2 = PM.assign(shifted, shape, scheme)
    assert np.abs(rho2 - np.roll(np.roll(rho, 1, axis=2), 2, axis=0)).max() < 1e-12


def test_tsc_is_cic_widened_by_a_cell():
    # 1D identity: W_TSC(s) = integral over |y| <= 1/2 of W_CIC(s - y) dy, so a TSC
    # deposit equals the average of CIC deposits of the particle shifted over a
    # cell; checked with a fine quadrature in all three axes for one particle
    rng = np.random.default_rng(3)
    shape = (8, 8, 8)
    p = rng.random((1, 3))
    m = 64
    y = (np.arange(m) + 0.5) / m - 0.5  # midpoint nodes over one cell
    acc = np.zeros(shape)
    for a in y:
        for b in y:
            q = np.mod(p + np.stack([np.full(m, a), np.full(m, b), y], axis=1) / 8.0, 1.0)
            acc += PM.assign(q, shape, "cic")  # the m z-shifts share one particle's mass
    acc /= m * m
    tsc = PM.assign(p, shape, "tsc")
    # midpoint rule on a piecewise-quadratic integrand: O(1/m^2)
    assert np.abs(acc - tsc).max() < 5e-3 * tsc.max()


def test_gradient_of_cosine_mode():
    shape = (8, 12, 16)
    n2, n1, n0 = shape
    k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    th = (2 * np.pi * 3 / n0, 2 * np.pi * 1 / n1, 2 * np.pi * 2 / n2)
    phi = np.cos(th[0] * i + th[1] * j + th[2] * k)
    gx, gy, gz = PM.gradient(phi)
    s = -np.sin(th[0] * i + th[1] * j + th[2] * k)
    assert np.abs(gx - s * np.sin(th[0]) * n0).max() < 1e-12
    assert np.abs(gy - s * np.sin(th[1]) * n1).max() < 1e-12
    assert np.abs(gz - s * np.sin(th[2]) * n2).max() < 1e-12


def test_force_at_cell_centre_closed_form():
    shape = (8, 12, 16)
    n2, n1, n0 = shape
    k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    th = (2 * np.pi * 3 / n0, 2 * np.pi * 1 / n1, 2 * np.pi * 2 / n2)
    phi = np.cos(th[0] * i + th[1] * j + th[2] * k)
    ci, cj, ck = 5, 7, 3
    pos = np.array([[(ci + 0.5) / n0, (cj + 0.5) / n1, (ck + 0.5) / n2]])
    ang = th[0] * ci + th[1] * cj + th[2] * ck
    g = np.array([np.sin(th[0]) * n0, np.sin(th[1]) * n1, np.sin(th[2]) * n2])
    # CIC at a cell centre: the cell's own gradient; -grad phi = sin(ang) g
    f_c = PM.forces(phi, pos, "cic")[0]
    assert np.abs(f_c - np.sin(ang) * g).max() < 1e-12
    # TSC: per axis (1/8, 3/4, 1/8) average of sin(ang + m th_d) = sin(ang)(3/4 + cos(th_d)/4)
    fac = np.prod([0.75 + 0.25 * np.cos(t) for t in th])
    f_t = PM.forces(phi, pos, "tsc")[0]
    assert np.abs(f_t - np.sin(ang) * fac * g).max() < 1e-12


@pytest.mark.parametrize("scheme", ["cic", "tsc"])
def test_no_self_force_and_equal_opposite_pair(scheme):
    rng = np.random.default_rng(4)
    shape = (16, 16, 16)
    h = 1.0 / 16
    p1 = rng.random((1, 3))
    rho = PM.assign(p1, shape, scheme)
    phi, _ = PO.solve_periodic(rho - rho.mean(), h)
    f = PM.forces(phi, p1, scheme)[0]
    scale = np.abs(PM.gradient(phi)[0]).max()
    assert np.abs(f).max() < 1e-12 * scale
    p2 = rng.random((1, 3))
    # forces on 1 from 2's density and on 2 from 1's density (equal masses)
    phi1, _ = PO.solve_periodic(PM.assign(p1, shape, scheme) - 1.0, h)
    phi2, _ = PO.solve_periodic(PM.assign(p2, shape, scheme) - 1.0, h)
    f12 = PM.forces(phi2, p1, scheme)[0]
    f21 = PM.forces(phi1, p2, scheme)[0]
    assert np.abs(f12 + f21).max() < 1e-11 * np.abs(f12).max()
