"""Test fields of Sec. VI.A with closed-form solutions, and the constants they need.

The constants are written out here from the paper's formulas, independently of
both the oracle and the library, so that the closed-form tests also pin the
constants:

* c~ = c / (B H0)                                         (Sec. III.A)
* K(a) = a^-3 + 4 OL/Om,  -Rbar = 3 m^2 K(a)              (Sec. II, III.B)
* |fbar~_R(a)| = n a^2 xi / (3 K(a))^{n+1}                (Sec. VI.A.1)
* xi from |f_R0| = |fbar_R(a=1)|
* linearised operator (Sec. IV): alpha * Laplacian_h - beta/(n+1), with
  alpha = c~^2 |fbar~_R| / h^2, beta = Om a^4 K(a), gamma = Om a.

Reading (the paper prints 1/(3 c~^2) before the density term of the continuum
equation but 1/c~^2 in Eq. discrete_fR): the discrete coefficient 1/c~^2 is the
one under which the sine and Gaussian closed forms below are exact; the tests
use it.  Reading of the Gaussian amplitude A: the exponent is n+1, so that
A = |fbar~_R| and delta -> 0 far from the peak as the paper states.
"""
from __future__ import annotations

import numpy as np

C_KMS = 299792.458
NHS = 1.0


def ctilde(box):
    return C_KMS / (100.0 * box)


def fbar_tilde_abs(a, omega_m, fr0, n=NHS):
    ol = 1.0 - omega_m
    k1 = 3.0 * (1.0 + 4.0 * ol / omega_m)
    xi = fr0 * k1 ** (n + 1) / n
    ka = 3.0 * (a ** -3 + 4.0 * ol / omega_m)
    return n * a * a * xi / ka ** (n + 1)


def coefficients(box, ncell, a, omega_m, fr0):
    """(alpha, beta, gamma) of the x c~^2 equation in u = ln(f_R/fbar_R)."""
    h = 1.0 / ncell
    alpha = ctilde(box) ** 2 * fbar_tilde_abs(a, omega_m, fr0) / h ** 2
    beta = omega_m * a ** 4 * (a ** -3 + 4.0 * (1.0 - omega_m) / omega_m)
    gamma = omega_m * a
    return alpha, beta, gamma


def cell_centres(n):
    return (np.arange(n) + 0.5) / n


def sine_field(n, *, box, a, omega_m, fr0):
    """Eq. (sine_dens), Sec. VI.A.3, as rho~ = 1 + delta on an n^3 grid (x only),
    and the exact u = ln(f_R / fbar_R) = ln(2 - sin 2 pi x)."""
    x = cell_centres(n)
    A = fbar_tilde_abs(a, omega_m, fr0)
    ol = 1.0 - omega_m
    s = np.sin(2 * np.pi * x)
    delta = (ctilde(box) ** 2 / (omega_m * a) * (2 * np.pi) ** 2 * A * s
             + (1.0 + 4.0 * a ** 3 * ol / omega_m) * ((2.0 - s) ** (-1.0 / (NHS + 1)) - 1.0))
    rho = np.broadcast_to(1.0 + delta, (n, n, n)).copy()
    u = np.broadcast_to(np.log(2.0 - s), (n, n, n)).copy()
    return rho, u


def gaussian_field(n, *, box, a, omega_m, fr0, amp, width):
    """Eq. (gaussian_dens), Sec. VI.A.4 (x only, peak at x = 0.5), and the exact
    u = ln(1 - amp exp(-(x-0.5)^2 / W^2)) from Eq. (fR_gaussian_dens)."""
    x = cell_centres(n)
    A = fbar_tilde_abs(a, omega_m, fr0)
    ol = 1.0 - omega_m
    xi = fr0 * (3.0 * (1.0 + 4.0 * ol / omega_m)) ** (NHS + 1) / NHS
    s2 = (x - 0.5) ** 2 / width ** 2
    g = np.exp(-s2)
    delta = (ctilde(box) ** 2 / (omega_m * a) * 2 * A * amp / width ** 2 * g * (1 - 2 * s2)
             + a ** 3 / 3.0 * (NHS * a * a * xi / (A * (1 - amp * g))) ** (1.0 / (NHS + 1))
             - (1.0 + 4.0 * ol / omega_m * a ** 3))
    rho = np.broadcast_to(1.0 + delta, (n, n, n)).copy()
    u = np.broadcast_to(np.log(1.0 - amp * g), (n, n, n)).copy()
    return rho, u


def linear_response(g, eps, *, box, a, omega_m, fr0):
    """Exact solution of the linearised discrete equation for rho = 1 + eps g on
    a periodic cube: u^(k) = -gamma eps g^(k) / (alpha sum_d 4 sin^2(pi k_d/N) + beta/2)."""
    n = g.shape[0]
    alpha, beta, gamma = coefficients(box, n, a, omega_m, fr0)
    k = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    lap = 4 * (np.sin(np.pi * kx / n) ** 2 + np.sin(np.pi * ky / n) ** 2
               + np.sin(np.pi * kz / n) ** 2)
    uh = -gamma * eps * np.fft.fftn(g) / (alpha * lap + beta / (NHS + 1))
    return np.fft.ifftn(uh).real


def algebraic_limit(rho, *, a, omega_m):
    """alpha -> 0 limit: beta (e^{-u/2} - 1) = gamma (rho - 1) pointwise."""
    beta = omega_m * a ** 4 * (a ** -3 + 4.0 * (1.0 - omega_m) / omega_m)
    gamma = omega_m * a
    return -(NHS + 1) * np.log1p(gamma * (rho - 1.0) / beta)


def spherical_gaussian_field(n, *, box, a, omega_m, fr0, amp, width, centre=(0.5, 0.5, 0.5),
                             offset=0.0):
    """3D analogue of Eq. (gaussian_dens): f_R = -A[1 - amp exp(-r^2/W^2)] with r
    the distance to ``centre``; the 3D Laplacian of exp(-r^2/W^2) is
    (4 r^2/W^4 - 6/W^2) exp(-r^2/W^2), which replaces (4 s^2/W^4 - 2/W^2) of the
    1D profile.  Evaluated at the centres of an n^3 grid shifted by ``offset``
    cells of size 1/n (for patches: pass the patch's fine grid)."""
    x = (np.arange(n) + 0.5 + offset) / n
    return _sph(x, x, x, box=box, a=a, omega_m=omega_m, fr0=fr0, amp=amp, width=width,
                centre=centre)


def _sph(xs, ys, zs, *, box, a, omega_m, fr0, amp, width, centre):
    A = fbar_tilde_abs(a, omega_m, fr0)
    ol = 1.0 - omega_m
    xi = fr0 * (3.0 * (1.0 + 4.0 * ol / omega_m)) ** (NHS + 1) / NHS
    z, y, x = np.meshgrid(zs, ys, xs, indexing="ij")
    r2 = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2) / width ** 2
    g = np.exp(-r2)
    delta = (ctilde(box) ** 2 / (omega_m * a) * A * amp * (6.0 - 4.0 * r2) / width ** 2 * g
             + a ** 3 / 3.0 * (NHS * a * a * xi / (A * (1 - amp * g))) ** (1.0 / (NHS + 1))
             - (1.0 + 4.0 * ol / omega_m * a ** 3))
    return 1.0 + delta, np.log(1.0 - amp * g)


def spherical_gaussian_patch(lo_fine, n_fine, n_domain_fine, **kw):
    """Same field on a sub-block of a grid of n_domain_fine^3 cells: fine cells
    lo_fine .. lo_fine + n_fine - 1 along each axis."""
    xs = (np.arange(lo_fine, lo_fine + n_fine) + 0.5) / n_domain_fine
    return _sph(xs, xs, xs, **kw)
