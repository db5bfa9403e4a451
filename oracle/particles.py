"""Plain FP64 CPU oracle of the particle-mesh steps on either side of the solvers.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``.  The GPU library never imports it.

Sec. VI.C of Li, Zhao, Teyssier & Koyama (arXiv:1110.1379): density assignment
with the triangle-shaped-cloud (TSC) scheme, the code's default, and force
interpolation with the same scheme as the assignment (CIC with CIC, TSC with
TSC) so that momentum is conserved.  The paper gives no formulas; the schemes
are the standard ones it refers to (Hockney & Eastwood):

* positions in box units [0, 1); cell centres at (i + 1/2)/n_d; in cell-centre
  units x = pos n_d - 1/2;
* CIC: the 2 nearest cells per axis, weights 1 - t and t (t = x - floor(x));
* TSC: the nearest cell c = floor(x + 1/2) and its two neighbours per axis,
  with d = x - c in [-1/2, 1/2): weights (1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2;
* 3D weights are products over the axes, periodic wrap; every particle has
  mass n0 n1 n2 / np, so that the mean density is 1;
* the force is -grad Phi with the gradient by central differences on the grid,
  (phi_{i+1} - phi_{i-1}) / (2 h_d), h_d = 1/n_d, interpolated to the particle
  with the assignment weights.

``numpy.add.at`` (an unbuffered scatter-add) performs the deposits.

Pins (tests/test_particle_pins.py; no function here is unpinned): assign by
test_mass_conservation, test_cell_centre_weights, test_translation_by_one_cell
and test_tsc_is_cic_widened_by_a_cell; gradient by test_gradient_of_cosine_mode;
forces by test_force_at_cell_centre_closed_form and
test_no_self_force_and_equal_opposite_pair.
"""
from __future__ import annotations

import numpy as np


def _stencil(pos, n, scheme):
    """Per axis: (cell indices [np, k], weights [np, k]) of the scheme."""
    pos = np.asarray(pos, dtype=np.float64)
    idx, wts = [], []
    for d in range(3):
        x = pos[:, d] * n[d] - 0.5
        if scheme == "cic":
            c0 = np.floor(x)
            t = x - c0
            cells = np.stack([c0, c0 + 1], axis=1)
            w = np.stack([1.0 - t, t], axis=1)
        elif scheme == "tsc":
            c = np.floor(x + 0.5)
            dd = x - c
            cells = np.stack([c - 1, c, c + 1], axis=1)
            w = np.stack([0.5 * (0.5 - dd) ** 2, 0.75 - dd ** 2, 0.5 * (0.5 + dd) ** 2], axis=1)
        else:
            raise ValueError(scheme)
        idx.append(np.mod(cells.astype(np.int64), n[d]))
        wts.append(w)
    return idx, wts


def assign(pos, shape, scheme="tsc"):
    """Density rho~ on a (n2, n1, n0) grid from particles at pos [np, 3] (x, y, z)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = (shape[2], shape[1], shape[0])
    npart = pos.shape[0]
    mass = float(np.prod(shape)) / npart
    (ix, iy, iz), (wx, wy, wz) = _stencil(pos, n, scheme)
    rho = np.zeros(shape)
    k = ix.shape[1]
    for a in range(k):
        for b in range(k):
            for c in range(k):
                np.add.at(rho, (iz[:, c], iy[:, b], ix[:, a]), mass * wx[:, a] * wy[:, b] * wz[:, c])
    return rho


def gradient(phi):
    """Central-difference gradient of a periodic (n2, n1, n0) field in box units:
    returns (gx, gy, gz)."""
    phi = np.asarray(phi, dtype=np.float64)
    n2, n1, n0 = phi.shape
    gx = (np.roll(phi, -1, axis=2) - np.roll(phi, 1, axis=2)) * (n0 / 2.0)
    gy = (np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) * (n1 / 2.0)
    gz = (np.roll(phi, -1, axis=0) - np.roll(phi, 1, axis=0)) * (n2 / 2.0)
    return gx, gy, gz


def forces(phi, pos, scheme="tsc"):
    """-grad Phi interpolated to the particles: [np, 3] (x, y, z)."""
    phi = np.asarray(phi, dtype=np.float64)
    shape = phi.shape
    n = (shape[2], shape[1], shape[0])
    g = gradient(phi)
    (ix, iy, iz), (wx, wy, wz) = _stencil(pos, n, scheme)
    out = np.zeros((np.asarray(pos).shape[0], 3))
    k = ix.shape[1]
    for a in range(k):
        for b in range(k):
            for c in range(k):
                w = wx[:, a] * wy[:, b] * wz[:, c]
                for d in range(3):
                    out[:, d] -= w * g[d][iz[:, c], iy[:, b], ix[:, a]]
    return out
