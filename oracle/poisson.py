"""Plain FP64 CPU oracle of the modified Poisson equation for Phi.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The GPU library never imports it.

Everything here follows Li, Zhao, Teyssier & Koyama (arXiv:1110.1379):

* the source is the right-hand side of Eq. (discrete_poisson) in the paper's
  variable u~ = ln(-a^2 f_R) (n = 1), evaluated as written:
      2 Om a (rho - 1) - (1/6) Om a^4 [ (n a^2 xi)^(1/(n+1)) exp(-u~/(n+1))
                                        - 3 (a^-3 + 4 OL/Om) ],
  with xi from the homogeneous solution that defines |f_R0| (Sec. VI.A.1);
* the operator is the 7-point Laplacian of the left-hand side of
  Eq. (discrete_poisson); on a refinement patch a missing neighbour is the
  ghost phi_g = 2 phi_b - phi_i (Eq. phi_b with mask ratio -1), which gives the
  left-hand side of Eq. (bc_modified_poisson);
* on a periodic grid the discrete solution is defined up to a constant and
  exists only for a source of zero mean; the oracle removes the source's mean
  and returns the solution of zero mean.  It is computed exactly (to rounding)
  with the discrete Fourier transform, whose modes are eigenvectors of the
  periodic 7-point Laplacian with eigenvalues -(4/h^2) sum_d sin^2(pi k_d/N_d);
* on a patch the BC-modified linear system is assembled and solved directly
  (``scipy.sparse.linalg.spsolve``; dense ``numpy.linalg.solve`` for tiny
  grids).

Values in and out are the shifted f(R) variable u = ln(f_R / fbar_R) (as in
``oracle.py``) and Phi in code units (box side 1, h = 1/N).

Pins (tests/test_poisson_pins.py; no function here is unpinned): source by
test_source_limits and test_source_mean_at_converged_fR_solution; laplacian
by test_stencil_explicit_sums and test_patch_ghost_rule_exact_for_linear_fields;
eigenvalues and solve_periodic by test_fft_solution_satisfies_stencil;
solve_patch by test_patch_solver_against_dense_stencil_matrix.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _orc


def source(u, rho, *, box, a, omega_m, fr0):
    """Right-hand side of Eq. (discrete_poisson), n = 1."""
    u = np.asarray(u, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    m = _orc.Model(box, u.shape[2], a, omega_m, fr0)
    ol = 1.0 - omega_m
    n = 1.0
    ut = u + m.ubar  # the paper's u~
    dr = (n * a * a * m.xi) ** (1.0 / (n + 1.0)) * np.exp(-ut / (n + 1.0)) \
        - 3.0 * (a ** -3 + 4.0 * ol / omega_m)
    return 2.0 * omega_m * a * (rho - 1.0) - omega_m * a ** 4 * dr / 6.0


def laplacian(phi, h, phib=None):
    """7-point Laplacian (1/h^2) [sum of the six neighbours - 6 phi].

    ``phib`` None: periodic grid.  Otherwise the six packed boundary faces
    (-x, +x, -y, +y, -z, +z; the layout of ``oracle.face_sizes``) of a patch:
    a neighbour outside the patch is the ghost 2 phi_b - phi_i.
    """
    phi = np.asarray(phi, dtype=np.float64)
    out = -6.0 * phi
    if phib is None:
        for ax in range(3):
            out += np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
        return out / (h * h)
    faces = _unpack_faces(phib, phi.shape)
    for ax in range(3):
        for side, sh in enumerate((1, -1)):
            nb = np.roll(phi, sh, axis=ax)
            # boundary layer of this side: the neighbour is the ghost
            idx = [slice(None)] * 3
            idx[ax] = slice(0, 1) if side == 0 else slice(phi.shape[ax] - 1, phi.shape[ax])
            idx = tuple(idx)
            nb[idx] = 2.0 * faces[2 * (2 - ax) + side] - phi[idx]
            out += nb
    return out / (h * h)


def _unpack_faces(phib, shape):
    """Packed faces -> six arrays broadcastable onto the boundary layers.

    Face f of a (n2, n1, n0) grid: f = 0, 1 (x faces) are [n2][n1], f = 2, 3
    (y) are [n2][n0], f = 4, 5 (z) are [n1][n0].  Returned in the order used
    by ``laplacian``: index 2*(2-ax) + side with ax the numpy axis (0 = z).
    """
    n2, n1, n0 = shape
    sizes = _orc.face_sizes(shape)
    off = np.concatenate([[0], np.cumsum(sizes)])
    f = [np.asarray(phib[off[i]:off[i + 1]], dtype=np.float64) for i in range(6)]
    return [f[0].reshape(n2, n1, 1), f[1].reshape(n2, n1, 1),
            f[2].reshape(n2, 1, n0), f[3].reshape(n2, 1, n0),
            f[4].reshape(1, n1, n0), f[5].reshape(1, n1, n0)]


def residual(phi, s, h, phib=None):
    """d = L(phi) - s."""
    return laplacian(phi, h, phib) - np.asarray(s, dtype=np.float64)


def eigenvalues(shape, h):
    """-(4/h^2) sum_d sin^2(pi k_d / N_d) on the FFT index grid of ``shape``."""
    lam = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = np.arange(n)
        e = -4.0 * np.sin(np.pi * k / n) ** 2 / (h * h)
        sh = [1, 1, 1]
        sh[ax] = n
        lam = lam + e.reshape(sh)
    return lam


def solve_periodic(s, h):
    """Zero-mean solution of L(phi) = s - mean(s) on a periodic grid.

    Returns (phi, mean(s)).
    """
    s = np.asarray(s, dtype=np.float64)
    mean = float(s.mean())
    sh = np.fft.fftn(s - mean)
    lam = eigenvalues(s.shape, h)
    lam[0, 0, 0] = 1.0
    ph = sh / lam
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph)), mean


def solve_patch(s, phib, h):
    """Solution of the BC-modified system L(phi) = s on a patch (direct solve)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    s = np.asarray(s, dtype=np.float64)
    shape = s.shape
    n2, n1, n0 = shape
    ncell = s.size
    # columns of the operator: L applied to unit vectors would be slow; assemble
    # the 7-point stencil with the ghost rule (diagonal -6 - 1 per missing
    # neighbour, off-diagonals +1) and move 2 phi_b / h^2 to the right-hand side
    idx = np.arange(ncell).reshape(shape)
    rows, cols, vals = [], [], []
    diag = np.full(shape, -6.0)
    rhs = s * h * h
    faces = _unpack_faces(phib, shape)
    for ax in range(3):
        for side, sh in enumerate((1, -1)):
            nbr = np.roll(idx, sh, axis=ax)
            inside = np.ones(shape, dtype=bool)
            bl = [slice(None)] * 3
            bl[ax] = slice(0, 1) if side == 0 else slice(shape[ax] - 1, shape[ax])
            bl = tuple(bl)
            inside[bl] = False
            rows.append(idx[inside])
            cols.append(nbr[inside])
            vals.append(np.ones(int(inside.sum())))
            diag[bl] -= 1.0
            rhs[bl] -= 2.0 * faces[2 * (2 - ax) + side][..., :] * np.ones_like(rhs[bl])
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ncell, ncell))
    if ncell <= 512:
        phi = np.linalg.solve(A.toarray(), rhs.ravel())
    else:
        phi = spla.spsolve(A.tocsc(), rhs.ravel())
    return phi.reshape(shape)
