"""Plain FP64 CPU oracle of the symmetron field equation (a second scalar-field
model on the same FAS machinery).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The GPU library never imports it.

The paper builds its multigrid solver for f(R) gravity and states (Sec. I,
Sec. VII) that the same machinery carries over to the other screened
scalar-field models it lists, among them the symmetron of Hinterbichler &
Khoury (2010, the paper's reference hk2010), whose structure formation was
simulated with the earlier multigrid code in Davis, Li, Mota & Winther (2011,
the paper's reference dlmw2011).  The model, in our own restatement:

* potential V(phi) = -mu^2 phi^2 / 2 + lambda phi^4 / 4, coupling to matter
  A(phi) = 1 + phi^2 / (2 M^2);
* in the quasi-static limit the comoving field equation is
  laplacian phi = a^2 [ (rho_m / M^2 - mu^2) phi + lambda phi^3 ];
* with chi = phi / phi_0 (phi_0 = mu / sqrt(lambda), the vacuum value), the
  symmetry-breaking density rho_SSB = mu^2 M^2 reached by the mean matter
  density at a = a_SSB (so rho_m / rho_SSB = (a_SSB / a)^3 rho~, rho~ the
  density in units of its mean) and the vacuum range lambda_0 = 1/(sqrt 2 mu):
      laplacian chi = (a^2 / (2 lambda_0^2)) [ ((a_SSB/a)^3 rho~ - 1) chi + chi^3 ].

Discretisation as the paper does it for f(R) (Sec. IV, Eq. discrete_fR; the
7-point Laplacian of Eq. discrete_poisson), on a periodic grid of cells of
size h (box units; B h Mpc/h), divided by the coefficient of the bracket so
that the residual is measured in units of the potential's gradient (the
same scaling on every multigrid level):

    L_i(chi) = A sum_{6 faces j} (chi_j - chi_i) - [ (s rho_i - 1) chi_i + chi_i^3 ] = 0,
    A = 2 lambda_0^2 / (a^2 (B h)^2),   s = (a_SSB / a)^3,

with the Newton derivative dL_i/dchi_i = -6 A - [ (s rho_i - 1) + 3 chi_i^2 ].
The algorithm is the paper's (Sec. V.B.2): red-black Newton-Gauss-Seidel
(u_i <- u_i - (L_i - f_i) / dL_i), FAS V-cycles with the 8-child average as
restriction and the trilinear 27/9/3/1 prolongation of Sec. V.A.3, the
coarse operator being the same L with the cell size doubled (A / 4) and the
density averaged.  Readings (listed in the design notes): the symmetric
field has two branches chi -> -chi; the solution sought is the positive one
(every start is positive); an update is clamped to |d chi| <= cap as in the
f(R) solver; the coarsest level is relaxed until its rms residual has fallen
by 1e-3 (or below 0.1 tol), at most 500 sweeps.

Vectorised red-black sweeps are exact: a cell's update reads only its own
value and neighbours of the other colour, so updating every cell of one
colour at once equals updating them one by one.

Pins (tests/test_symmetron_pins.py; no function here is unpinned):
coefficients and background by test_coefficients_closed_form and
test_homogeneous_solution_from_random_start; operator and derivative by
test_operator_sums_to_the_local_terms,
test_newton_derivative_by_finite_differences,
test_linear_limit_matches_fft_solution, test_short_range_limit_is_the_local_minimum
and test_screening_in_dense_cells; smooth by
test_sweep_equals_cell_by_cell_red_then_black; restrict and prolong by
test_transfer_operators; num_levels and the coarsest rule by
test_level_rule_and_coarsest_rule_by_hand; vcycle and solve by
test_two_level_cycle_by_hand, test_fas_matches_dense_newton_brute_force and
test_manufactured_solution_through_the_multigrid.
"""
from __future__ import annotations

import numpy as np


def coefficients(box, n, a, a_ssb, lambda0):
    """(A, s) of the discrete equation on a grid of n cells per side."""
    h = box / n  # cell size in Mpc/h
    A = 2.0 * lambda0 * lambda0 / (a * a * h * h)
    s = (a_ssb / a) ** 3
    return A, s


def background(a, a_ssb):
    """Homogeneous solution (rho = 1) on the positive branch: sqrt(1 - s) after
    symmetry breaking (a > a_SSB), 0 before."""
    s = (a_ssb / a) ** 3
    return float(np.sqrt(max(0.0, 1.0 - s)))


def laplacian_sum(chi):
    """sum over the 6 periodic neighbours of (chi_j - chi_i)."""
    out = -6.0 * chi
    for ax in range(3):
        out = out + np.roll(chi, 1, ax) + np.roll(chi, -1, ax)
    return out


def operator(chi, rho, A, s):
    """L_i(chi) on a periodic grid."""
    return A * laplacian_sum(chi) - ((s * rho - 1.0) * chi + chi ** 3)


def derivative(chi, rho, A, s):
    """dL_i / dchi_i."""
    return -6.0 * A - ((s * rho - 1.0) + 3.0 * chi * chi)


def colour_mask(shape, colour):
    k, j, i = np.indices(shape)
    return ((i + j + k) & 1) == colour


def smooth(chi, rho, f, A, s, nsweeps, cap=1.0):
    """nsweeps red-black Newton-Gauss-Seidel sweeps of L(chi) = f (red first)."""
    chi = chi.copy()
    masks = [colour_mask(chi.shape, c) for c in (0, 1)]
    for _ in range(nsweeps):
        for m in masks:
            r = operator(chi, rho, A, s) - f
            d = -r / derivative(chi, rho, A, s)
            d = np.clip(d, -cap, cap)
            chi[m] += d[m]
    return chi


def restrict(a):
    """Mean of the 8 children of every coarse cell."""
    n2, n1, n0 = a.shape
    return a.reshape(n2 // 2, 2, n1 // 2, 2, n0 // 2, 2).mean(axis=(1, 3, 5))


def prolong(c):
    """Trilinear (27/9/3/1 over 64) periodic interpolation of a coarse field
    onto the grid of twice its size (Sec. V.A.3)."""
    out = c
    for ax in range(3):
        near = np.repeat(out, 2, axis=ax)
        # the farther coarse neighbour of each fine cell: -1 for even, +1 for odd
        lo = np.repeat(np.roll(out, 1, ax), 2, axis=ax)
        hi = np.repeat(np.roll(out, -1, ax), 2, axis=ax)
        idx = [slice(None)] * 3
        far = lo.copy()
        idx[ax] = slice(1, None, 2)
        far[tuple(idx)] = hi[tuple(idx)]
        out = 0.75 * near + 0.25 * far
    return out


def num_levels(shape):
    """Halve while every size stays even and >= 4 (the f(R) solver's rule)."""
    n = list(shape)
    nl = 1
    while all(v % 2 == 0 and v // 2 >= 4 for v in n):
        n = [v // 2 for v in n]
        nl += 1
    return nl


def _coarsest(chi, rho, f, A, s, tol, cap):
    r0 = np.sqrt(np.mean((operator(chi, rho, A, s) - f) ** 2))
    lim = max(1e-3 * r0, 0.1 * tol)
    for _ in range(500):
        chi = smooth(chi, rho, f, A, s, 1, cap)
        if np.sqrt(np.mean((operator(chi, rho, A, s) - f) ** 2)) <= lim:
            break
    return chi


def vcycle(chi, rho, f, A, s, nl, *, pre, post, cap, tol):
    """One FAS V-cycle (Sec. V.B.2) on L(chi) = f; rho and A of this level."""
    if nl == 1:
        return _coarsest(chi, rho, f, A, s, tol, cap)
    chi = smooth(chi, rho, f, A, s, pre, cap)
    d = operator(chi, rho, A, s) - f
    uR = restrict(chi)
    rhoH = restrict(rho)
    AH = 0.25 * A
    fH = operator(uR, rhoH, AH, s) - restrict(d)
    uH = vcycle(uR.copy(), rhoH, fH, AH, s, nl - 1, pre=pre, post=post, cap=cap, tol=tol)
    chi = chi + prolong(uH - uR)
    return smooth(chi, rho, f, A, s, post, cap)


class Result:
    def __init__(self, chi, cycles, hist, converged):
        self.chi, self.cycles, self.hist, self.converged = chi, cycles, hist, converged


def solve(rho, *, box, a, a_ssb, lambda0, tol=1e-8, chi0=None, pre=2, post=2, cap=1.0,
          max_cycles=100):
    """FAS V-cycles from chi0 (default: the homogeneous positive solution, or
    1 before symmetry breaking) until rms(L(chi)) <= tol."""
    rho = np.asarray(rho, dtype=np.float64)
    A, s = coefficients(box, rho.shape[2], a, a_ssb, lambda0)
    if chi0 is None:
        chi = np.full(rho.shape, background(a, a_ssb) or 1.0)
    else:
        chi = np.array(chi0, dtype=np.float64)
    nl = num_levels(rho.shape)
    f = np.zeros_like(rho)
    hist = [float(np.sqrt(np.mean(operator(chi, rho, A, s) ** 2)))]
    cycles = 0
    while hist[-1] > tol and cycles < max_cycles:
        chi = vcycle(chi, rho, f, A, s, nl, pre=pre, post=post, cap=cap, tol=tol)
        cycles += 1
        hist.append(float(np.sqrt(np.mean(operator(chi, rho, A, s) ** 2))))
        if not np.isfinite(hist[-1]):
            break
    return Result(chi, cycles, hist, hist[-1] <= tol)


def dense_newton(rho, *, box, a, a_ssb, lambda0, chi0, tol=1e-13, cap=1.0, max_iter=100):
    """Brute force: Newton's method on the whole grid at once with the full
    Jacobian (numpy.linalg.solve); independent of the multigrid path."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    A, s = coefficients(box, shape[2], a, a_ssb, lambda0)
    n = rho.size
    idx = np.arange(n).reshape(shape)
    chi = np.array(chi0, dtype=np.float64).copy()
    for _ in range(max_iter):
        r = operator(chi, rho, A, s).ravel()
        if np.abs(r).max() < tol:
            break
        J = np.zeros((n, n))
        J[np.arange(n), np.arange(n)] = derivative(chi, rho, A, s).ravel()
        for ax in range(3):
            for sh in (1, -1):
                nb = np.roll(idx, -sh, ax).ravel()  # neighbour j of cell i
                np.add.at(J, (np.arange(n), nb), A)
        d = np.linalg.solve(J, -r)
        d = np.clip(d, -cap, cap)
        chi = chi + d.reshape(shape)
    return chi


def linear_response(g, eps, *, box, a, a_ssb, lambda0):
    """Exact solution of the discrete equation linearised about the
    homogeneous positive solution chib for rho = 1 + eps g (a > a_SSB):
        (A Delta_h - m2) dchi = s chib eps g,   m2 = 2 (1 - s),
    solved by FFT; the nonlinear solution agrees to O(eps^2)."""
    shape = g.shape
    A, s = coefficients(box, shape[2], a, a_ssb, lambda0)
    chib = background(a, a_ssb)
    m2 = 2.0 * (1.0 - s)
    sym = np.zeros(shape)
    for ax, n in enumerate(shape):
        kk = np.fft.fftfreq(n) * n
        sh = [1, 1, 1]
        sh[ax] = n
        sym = sym + (4.0 * np.sin(np.pi * kk / n) ** 2).reshape(sh)
    ghat = np.fft.fftn(g)
    dhat = -s * chib * eps * ghat / (A * sym + m2)
    return chib + np.real(np.fft.ifftn(dhat))
