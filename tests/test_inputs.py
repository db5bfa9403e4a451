"""The seeded input generators (paper_1110_1379_gb300/synth.py) produce the
recipe the design states: spectrum, normalisation, determinism, the batch
and nested-patch layouts, and the masked-region shape.  No GPU."""
import numpy as np
import pytest

from paper_1110_1379_gb300 import synth


def _shell_power(g, kmin=2, kmax=12):
    """Mean |g^(k)|^2 in integer shells of |k| (grid units)."""
    n = g.shape[0]
    gk = np.abs(np.fft.fftn(g)) ** 2
    k = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    ks = np.arange(kmin, kmax)
    p = np.array([gk[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in ks])
    return ks, p


@pytest.mark.parametrize("slope", [-1.5, -2.5])
def test_gaussian_field_spectrum_and_normalisation(slope):
    g = synth.gaussian_random_field((48, 48, 48), 7, sigma=1.7, slope=slope)
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.7, rel=1e-12)
    ks, p = _shell_power(g)
    fit = np.polyfit(np.log(ks), np.log(p), 1)[0]
    assert fit == pytest.approx(slope, abs=0.2)
    assert np.array_equal(g, synth.gaussian_random_field((48, 48, 48), 7, sigma=1.7, slope=slope))
    assert not np.array_equal(g, synth.gaussian_random_field((48, 48, 48), 8, sigma=1.7,
                                                              slope=slope))


def test_lognormal_density():
    rho = synth.lognormal_density((32, 24, 40), 3, sigma=2.0)
    assert rho.shape == (32, 24, 40) and rho.dtype == np.float64
    assert rho.min() > 0 and rho.mean() == pytest.approx(1.0, abs=1e-14)
    lg = np.log(rho)
    assert lg.std() == pytest.approx(2.0, rel=1e-10)   # exp(g - s^2/2) / mean: log is g + const


def test_point_mass_field():
    rho = synth.point_mass_density(8)
    assert rho.mean() == pytest.approx(1.0, abs=1e-15)
    assert rho[0, 0, 0] - 1 == pytest.approx(1e-4 * 511) and rho[1, 0, 0] - 1 == pytest.approx(-1e-4)


def test_zeldovich_positions():
    n = 16
    lat = synth.zeldovich_positions(n, 2, 0.0)
    q = (np.arange(n) + 0.5) / n
    assert lat.shape == (n ** 3, 3) and np.allclose(np.sort(np.unique(lat[:, 0])), q)
    pos = synth.zeldovich_positions(n, 2, 1.0)
    assert pos.min() >= 0.0 and pos.max() < 1.0
    d = (pos - lat + 0.5) % 1.0 - 0.5                  # displacement, periodic
    assert 0.0 < np.abs(d).max() < 0.2
    assert np.abs(d.mean(axis=0)).max() < 1e-12        # k = 0 removed: no net drift
    d2 = (synth.zeldovich_positions(n, 2, 2.0) - lat + 0.5) % 1.0 - 0.5
    assert np.allclose(d2, 2.0 * d, atol=1e-12)        # linear in the amplitude


def test_batch_specs_recipe():
    specs = synth.batch_specs()
    assert len(specs) == 96
    assert {s["n"] for s in specs} <= {32, 48, 64, 96, 128}
    assert {s["fr0"] for s in specs} == {1e-4, 1e-5, 1e-6}
    assert all(0.3 <= s["a"] <= 1.0 and 0.5 <= s["sigma"] <= 2.5 for s in specs)
    assert all(s["box"] == s["n"] for s in specs)
    assert [s["seed"] for s in specs] == list(range(5000, 5096))
    assert specs == synth.batch_specs()


def test_refined_density_is_mass_consistent():
    parent = synth.lognormal_density((4, 6, 8), 1, sigma=1.0)
    child = synth.refine_density(parent, 9)
    assert child.shape == (8, 12, 16) and child.min() > 0
    back = child.reshape(4, 2, 6, 2, 8, 2).mean(axis=(1, 3, 5))
    assert np.abs(back - parent).max() < 1e-13


def test_nested_layout_nests_and_does_not_overlap():
    rho0, patches = synth.nested_case(32, 11, (16, 24), 4, (8, 16), 2)
    lvl1 = [p for p in patches if p["parent"] < 0]
    assert len(lvl1) == 4
    occupied = np.zeros(rho0.shape, dtype=bool)
    for p in lvl1:
        o, s = p["origin"], p["rho"].shape[0] // 2
        assert all(1 <= o[d] and o[d] + s <= 31 for d in range(3))   # one-cell margin
        sl = (slice(o[2], o[2] + s), slice(o[1], o[1] + s), slice(o[0], o[0] + s))
        assert not occupied[sl].any()
        occupied[sl] = True
        blk = rho0[sl]
        back = p["rho"].reshape(s, 2, s, 2, s, 2).mean(axis=(1, 3, 5))
        assert np.abs(back - blk).max() < 1e-12
    for p in patches:
        if p["parent"] >= 0:
            par = patches[p["parent"]]["rho"]
            o, s = p["origin"], p["rho"].shape[0] // 2
            assert all(1 <= o[d] and o[d] + s <= par.shape[2 - d] - 1 for d in range(3))


def test_sphere_union_mask():
    rho = synth.lognormal_density((40, 40, 40), 4, sigma=1.5)
    m = synth.sphere_union_mask(rho, 6, (4.0, 8.0), 2, margin=2)
    assert set(np.unique(m)) == {-1.0, 1.0}
    edge = np.ones(m.shape, dtype=bool)
    edge[1:-1, 1:-1, 1:-1] = False
    assert (m[edge] < 0).all() and (m > 0).sum() > 6 * 4 ** 3
