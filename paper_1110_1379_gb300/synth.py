"""Seeded synthetic inputs: density fields and particle sets.

This module holds no solver arithmetic.  It only draws random numbers and
shapes them into the inputs the solver and the oracle both consume:

* Gaussian random fields with a power-law spectrum P(k) ~ k^slope
  (white noise -> rFFT -> multiply by sqrt(P) -> irFFT -> scale to sigma),
* lognormal densities rho = exp(g - sigma^2/2), renormalised to mean 1
  (rho~ has mean 1 in the paper's code units, Sec. III.A),
* Zel'dovich-displaced particle lattices (displacement s = IFFT(i k / k^2 g^)),
* the point-mass field of Sec. VI.A.2 (Eq. point_mass).

Seeds follow seed = 1000 * config + field index.  numpy only.
"""
from __future__ import annotations

import numpy as np


def _kgrid(shape):
    """Integer wavenumbers for an rFFT of a (n2, n1, n0) array."""
    n2, n1, n0 = shape
    kz = np.fft.fftfreq(n2, d=1.0 / n2)
    ky = np.fft.fftfreq(n1, d=1.0 / n1)
    kx = np.fft.rfftfreq(n0, d=1.0 / n0)
    return np.meshgrid(kz, ky, kx, indexing="ij")


def gaussian_random_field(shape, seed, sigma=1.0, slope=-1.5, dtype=np.float64):
    """Zero-mean Gaussian field with P(k) ~ |k|^slope (k in grid units), k = 0
    removed, normalised to standard deviation ``sigma`` per cell."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    wk = np.fft.rfftn(white)
    del white
    kz, ky, kx = _kgrid(shape)
    k2 = kz * kz + ky * ky + kx * kx
    del kz, ky, kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)  # sqrt(P) = |k|^(slope/2)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del amp, k2
    g = np.fft.irfftn(wk, s=shape, axes=(0, 1, 2))
    del wk
    g -= g.mean()
    std = g.std()
    if std > 0:
        g *= sigma / std
    return g.astype(dtype, copy=False)


def lognormal_density(shape, seed, sigma=1.0, slope=-1.5):
    """rho = exp(g - sigma^2/2) renormalised to an exact mean of 1 (FP64)."""
    g = gaussian_random_field(shape, seed, sigma=sigma, slope=slope)
    g -= 0.5 * sigma * sigma
    np.exp(g, out=g)
    g /= g.mean()
    return g


def point_mass_density(n):
    """Eq. (point_mass), Sec. VI.A.2: contrast 1e-4 (N^3 - 1) in cell (0,0,0) and
    -1e-4 elsewhere; returned as rho~ = 1 + contrast."""
    rho = np.full((n, n, n), 1.0 - 1e-4)
    rho[0, 0, 0] = 1.0 + 1e-4 * (n ** 3 - 1)
    return rho


def zeldovich_positions(n, seed, amplitude, slope=-1.5):
    """n^3 particles on a cell-centred lattice displaced by amplitude * s(q),
    s = IFFT(i k / k^2 g^) with g a unit-variance field of spectrum k^slope.
    Positions are in box units, wrapped into [0, 1); shape (n^3, 3) as (x, y, z)."""
    shape = (n, n, n)
    g = gaussian_random_field(shape, seed, sigma=1.0, slope=slope)
    gk = np.fft.rfftn(g)
    del g
    kz, ky, kx = _kgrid(shape)
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    disp = []
    for kd in (kx, ky, kz):
        sk = 1j * kd / k2 * gk
        sk[0, 0, 0] = 0.0
        disp.append(np.fft.irfftn(sk, s=shape, axes=(0, 1, 2)) / n)  # grid units -> box units
    del gk, kz, ky, kx, k2
    q = (np.arange(n) + 0.5) / n
    qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
    pos = np.empty((n ** 3, 3))
    for d, qd in enumerate((qx, qy, qz)):
        x = qd + amplitude * disp[d]
        pos[:, d] = np.mod(x, 1.0).ravel()
    # np.mod can return exactly 1.0 for tiny negative inputs
    pos[pos >= 1.0] = 0.0
    return pos


# Zel'dovich spectrum slope and amplitude for the 128^3, seed-2000 particle set
# of the CIC workload, written by oracle/calibrate_zeldovich.py: the first
# slope of -1.5, -2, -2.5, -3 whose best amplitude reaches the contrast of ~100
# the workload names (max(rho~ - 1) = 101.0 of the CIC density; with slope
# -1.5 a one-particle-per-cell field saturates at 43.7).
ZELDOVICH_SLOPE_128 = -2.5
ZELDOVICH_AMPLITUDE_128 = 60.0


def uniform_positions(np_, seed):
    rng = np.random.default_rng(seed)
    return rng.random((np_, 3))


def batch_specs(nfields=96, seed=5000):
    """Many independent fields of uneven size: N from {32, 48, 64, 96, 128},
    |f_R0| from {1e-4, 1e-5, 1e-6}, a ~ U[0.3, 1], lognormal sigma ~ U[0.5, 2.5],
    box = N Mpc/h (cell 1 Mpc/h); field i uses density seed seed + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nfields):
        n = int(rng.choice([32, 48, 64, 96, 128]))
        out.append(dict(n=n, fr0=float(rng.choice([1e-4, 1e-5, 1e-6])),
                        a=float(rng.uniform(0.3, 1.0)), sigma=float(rng.uniform(0.5, 2.5)),
                        box=float(n), seed=seed + i))
    return out


def refine_density(parent_block, seed, sigma=0.5):
    """Density of a refinement patch over a block of parent cells: each parent
    cell splits into 2x2x2 children whose values are the parent value times a
    seeded lognormal modulation normalised to mean 1 over the 8 children, so
    the children average exactly to their parent (mass-consistent)."""
    rng = np.random.default_rng(seed)
    p = np.asarray(parent_block, dtype=np.float64)
    mod = np.exp(sigma * rng.standard_normal((2 * p.shape[0], 2 * p.shape[1], 2 * p.shape[2])))
    m = mod.reshape(p.shape[0], 2, p.shape[1], 2, p.shape[2], 2)
    m = m / m.mean(axis=(1, 3, 5), keepdims=True)
    child = m * p[:, None, :, None, :, None]
    return child.reshape(2 * p.shape[0], 2 * p.shape[1], 2 * p.shape[2])


def patch_layout(rho, sizes, count, seed, margin=1, parent_box=None):
    """Greedy placement of `count` cubic patches of fine sizes drawn from `sizes`
    over the densest cells of the parent grid rho (n2, n1, n0): each patch's
    footprint (size/2 parent cells) plus `margin` parent cells stays inside the
    parent (or inside parent_box = (lo, hi) per axis) and does not overlap
    earlier patches.  Returns a list of (origin (x, y, z), size)."""
    rng = np.random.default_rng(seed)
    n2, n1, n0 = rho.shape
    order = np.argsort(rho, axis=None)[::-1]
    taken = np.zeros(rho.shape, dtype=bool)
    out = []
    lo = np.array([margin, margin, margin])
    hi = np.array([n0, n1, n2]) - margin
    if parent_box is not None:
        lo = np.maximum(lo, np.array(parent_box[0]) + margin)
        hi = np.minimum(hi, np.array(parent_box[1]) - margin)
    for flat in order:
        if len(out) >= count:
            break
        k, j, i = np.unravel_index(flat, rho.shape)
        s = int(rng.choice(sizes))
        half = s // 2
        org = np.array([i, j, k]) - half // 2
        org = np.minimum(np.maximum(org, lo), hi - half)
        if np.any(org < lo) or np.any(org + half > hi):
            continue
        sl = (slice(org[2], org[2] + half), slice(org[1], org[1] + half),
              slice(org[0], org[0] + half))
        if taken[sl].any():
            continue
        taken[sl] = True
        out.append((tuple(int(v) for v in org), s))
    return out


def nested_case(n, seed, sizes1, count1, sizes2, count2, sigma=2.5):
    """Domain density (lognormal) plus refinement patches: `count1` level-1
    patches of fine sizes from `sizes1` over the densest domain cells, and one
    level-2 patch (sizes from `sizes2`) inside each of the first `count2`
    level-1 patches.  Returns (rho_domain, [dict(parent, origin, rho)])."""
    rho0 = lognormal_density((n, n, n), seed, sigma=sigma)
    lay1 = patch_layout(rho0, sizes1, count1, seed + 1, margin=1)
    patches = []
    for t, (org, s) in enumerate(lay1):
        blk = rho0[org[2]:org[2] + s // 2, org[1]:org[1] + s // 2, org[0]:org[0] + s // 2]
        patches.append(dict(parent=-1, origin=org, rho=refine_density(blk, seed + 10 + t)))
    for t1 in range(min(count2, len(lay1))):
        p = patches[t1]
        lay2 = patch_layout(p["rho"], sizes2, 1, seed + 100 + t1, margin=1)
        for org, s in lay2:
            blk = p["rho"][org[2]:org[2] + s // 2, org[1]:org[1] + s // 2,
                           org[0]:org[0] + s // 2]
            patches.append(dict(parent=t1, origin=org, rho=refine_density(blk, seed + 200 + t1)))
    return rho0, patches


def sphere_union_mask(rho, count, radii, seed, margin=2):
    """Mask of an irregular refinement region: +1 inside the union of `count`
    spheres centred on the densest cells of rho (at least one minimum radius
    apart, at least the maximum radius + margin cells from the box edge), with
    radii drawn uniformly from radii = (rmin, rmax) cells; -1 elsewhere (so the
    box's outer layer is masked).  A wider masked margin lets the multigrid
    hierarchy coarsen further (each coarser level must keep its outer layer
    masked)."""
    rng = np.random.default_rng(seed)
    n2, n1, n0 = rho.shape
    rmin, rmax = radii
    edge = int(np.ceil(rmax)) + margin
    inner = np.full(rho.shape, -np.inf)
    inner[edge:n2 - edge, edge:n1 - edge, edge:n0 - edge] = \
        rho[edge:n2 - edge, edge:n1 - edge, edge:n0 - edge]
    order = np.argsort(inner, axis=None)[::-1]
    centres = []
    for c in order:
        if len(centres) == count or not np.isfinite(inner.flat[c]):
            break
        p = np.array(np.unravel_index(c, rho.shape))
        if all(np.sum((p - q) ** 2) >= rmin ** 2 for q in centres):
            centres.append(p)
    m = -np.ones(rho.shape)
    for p in centres:
        r = rng.uniform(rmin, rmax)
        R = int(np.ceil(r))
        lo = [max(0, int(p[d]) - R) for d in range(3)]
        hi = [min(rho.shape[d], int(p[d]) + R + 1) for d in range(3)]
        k, j, i = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                              np.arange(lo[2], hi[2]), indexing="ij")
        inside = (k - p[0]) ** 2 + (j - p[1]) ** 2 + (i - p[2]) ** 2 < r * r
        sub = m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        sub[inside] = 1.0
    return m
