"""Batched fields (many grids per launch) and nested refinement patches on the
GPU against the FP64 oracle.

Small cases are compared element by element with the oracle's solutions.  The
full-size batched workload (96 fields of 32^3-128^3) and the full-size nested
workload (256^3 domain, two refinement levels) are checked through properties
that hold at any size: the oracle's pointwise residual L_i(u) at sampled cells
of the GPU solution, the telescoping invariant of the flux terms, and full
oracle solves of the fields small enough to finish in seconds.
"""
import numpy as np
import pytest

import paper_fields as PF
from gpu_common import ctx, dev, host, local_block, torch  # noqa: F401
from oracle import oracle as O
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu
OM = 0.24


@pytest.fixture(scope="module")
def C():
    return ctx()


def sampled_residual(u, rho, *, box, a, fr0, h, nsample=200, seed=0, interior=0):
    """max |L_i(u)| from the oracle at sampled cells, each evaluated on the
    6^3 block centred on the cell (periodic grids, or patch cells at least
    `interior` cells from the patch edge)."""
    rng = np.random.default_rng(seed)
    n2, n1, n0 = u.shape
    worst = 0.0
    for _ in range(nsample):
        k = int(rng.integers(interior, n2 - interior))
        j = int(rng.integers(interior, n1 - interior))
        i = int(rng.integers(interior, n0 - interior))
        ub = local_block(u, k, j, i)
        rb = local_block(rho, k, j, i)
        L, _ = O.cell_op(ub, rb, 3, 3, 3, box=box, a=a, omega_m=OM, fr0=fr0, h=h)
        worst = max(worst, abs(L))
    return worst


# ------------------------------------------------------------------ batches
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_batch_matches_oracle(C, prec):
    specs = [dict(n=16, fr0=1e-4, a=0.5, sigma=1.0, box=16.0, seed=11),
             dict(n=24, fr0=1e-5, a=0.8, sigma=2.0, box=24.0, seed=12),
             dict(n=32, fr0=1e-6, a=1.0, sigma=2.5, box=32.0, seed=13),
             dict(n=48, fr0=1e-5, a=0.35, sigma=1.5, box=48.0, seed=14),
             dict(n=32, fr0=1e-4, a=0.9, sigma=0.5, box=32.0, seed=15)]
    rhos = [synth.lognormal_density((s["n"],) * 3, s["seed"], sigma=s["sigma"]) for s in specs]
    us = [torch.zeros((s["n"],) * 3, dtype=torch.float64, device="cuda") for s in specs]
    st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[s["box"] for s in specs],
                              avals=[s["a"] for s in specs], fr0s=[s["fr0"] for s in specs],
                              omega_m=OM, tol=1e-8, prec=prec)
    assert st == 0
    for s, r, u, stt in zip(specs, rhos, us, stats):
        ref = O.solve(r, tol=1e-8, box=s["box"], a=s["a"], omega_m=OM, fr0=s["fr0"])
        assert ref.converged and stt.res_rms <= 1e-8
        assert np.abs(host(u) - ref.u).max() <= 1e-6
        if prec == "fp64":
            assert stt.vcycles == ref.cycles


@pytest.mark.parametrize("pre,post", [(2, 1), (1, 2), (1, 1)])
@pytest.mark.parametrize("defect_precision", [0, 1])
def test_batch_with_odd_pass_plans_matches_oracle(C, pre, post, defect_precision):
    """Odd numbers of ping-pong passes per cycle in a batch whose fields leave
    the inner solves at different cycles (each keeps its data in the buffer it
    left with): every field still reaches the oracle's solution."""
    specs = [dict(n=16, fr0=1e-4, a=0.5, sigma=1.0, box=16.0, seed=31),
             dict(n=32, fr0=1e-6, a=1.0, sigma=2.5, box=32.0, seed=32),
             dict(n=24, fr0=1e-5, a=0.8, sigma=1.5, box=24.0, seed=33),
             dict(n=32, fr0=1e-4, a=0.35, sigma=0.5, box=16.0, seed=34)]
    rhos = [synth.lognormal_density((s["n"],) * 3, s["seed"], sigma=s["sigma"]) for s in specs]
    us = [torch.zeros((s["n"],) * 3, dtype=torch.float64, device="cuda") for s in specs]
    st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[s["box"] for s in specs],
                              avals=[s["a"] for s in specs], fr0s=[s["fr0"] for s in specs],
                              omega_m=OM, tol=1e-8, prec="mixed", pre=pre, post=post, tiling=1,
                              defect_precision=defect_precision)
    assert st == 0
    cyc = set()
    for s, r, u, stt in zip(specs, rhos, us, stats):
        ref = O.solve(r, tol=1e-8, box=s["box"], a=s["a"], omega_m=OM, fr0=s["fr0"])
        assert stt.res_rms <= 1e-8
        assert np.abs(host(u) - ref.u).max() <= 1e-6
        cyc.add(stt.vcycles)
    if (pre + post) % 2:
        assert len(cyc) > 1  # the fields did leave at different cycles


def test_batch_autotune_returns_a_converging_setting(C):
    specs = [dict(n=16, fr0=1e-4, a=0.5, sigma=1.0, box=16.0, seed=21),
             dict(n=32, fr0=1e-5, a=1.0, sigma=2.0, box=32.0, seed=22),
             dict(n=24, fr0=1e-6, a=0.8, sigma=1.5, box=24.0, seed=23)]
    rhos = [synth.lognormal_density((s["n"],) * 3, s["seed"], sigma=s["sigma"]) for s in specs]
    kw = dict(boxes=[s["box"] for s in specs], avals=[s["a"] for s in specs],
              fr0s=[s["fr0"] for s in specs], omega_m=OM, tol=1e-8)
    best, secs = C.autotune_batch([dev(r) for r in rhos], prec="mixed", **kw)
    assert secs > 0 and (best["pre"], best["post"]) in [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3)]
    assert best["relax"] in (1.0, 1.15, 1.25) and best["tiling"] in (0, 1)
    assert best["smooth_tile"] in (16, 8, -1)
    us = [torch.zeros((s["n"],) * 3, dtype=torch.float64, device="cuda") for s in specs]
    opts = {k: best[k] for k in ("pre", "post", "relax", "tiling", "smooth_tile")}
    st, stats = C.solve_batch([dev(r) for r in rhos], us, prec="mixed", **kw, **opts)
    assert st == 0
    for s, r, u in zip(specs, rhos, us):
        ref = O.solve(r, tol=1e-8, box=s["box"], a=s["a"], omega_m=OM, fr0=s["fr0"])
        assert np.abs(host(u) - ref.u).max() <= 1e-6


def test_full_batch_workload(C):
    """96 fields, N in {32..128}, mixed precision, one batched solve."""
    specs = synth.batch_specs(96, 5000)
    rhos = [synth.lognormal_density((s["n"],) * 3, s["seed"], sigma=s["sigma"]) for s in specs]
    us = [torch.zeros((s["n"],) * 3, dtype=torch.float64, device="cuda") for s in specs]
    st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[s["box"] for s in specs],
                              avals=[s["a"] for s in specs], fr0s=[s["fr0"] for s in specs],
                              omega_m=OM, tol=1e-8, prec="mixed")
    assert st == 0
    checked_full = 0
    for idx, (s, r, u, stt) in enumerate(zip(specs, rhos, us, stats)):
        assert stt.res_rms <= 1e-8
        uh = host(u)
        P = dict(box=s["box"], a=s["a"], fr0=s["fr0"])
        # telescoping: sum_i L_i = sum_i [beta (e^{-u/2} - 1) - gamma (rho - 1)]
        _, beta, gamma = PF.coefficients(s["box"], s["n"], s["a"], OM, s["fr0"])
        tel = np.sum(beta * np.expm1(-uh / 2) - gamma * (r - 1.0))
        assert abs(tel) <= 10 * uh.size * 1e-8
        if s["n"] <= 48 and checked_full < 6:
            ref = O.solve(r, tol=1e-8, omega_m=OM, **P)
            assert np.abs(uh - ref.u).max() <= 1e-6
            checked_full += 1
        elif idx % 8 == 0:
            assert sampled_residual(uh, r, h=1.0 / s["n"], nsample=40, seed=idx, **P) < 1e-6


# ------------------------------------------------------------------ nested patches
def _levels_case(N, P, sizes1, n1, sizes2, n2, seed):
    return synth.nested_case(N, seed, sizes1, n1, sizes2, n2)


@pytest.mark.parametrize("prec,relax", [("fp64", 1.0), ("mixed", 1.0), ("mixed", 1.2)])
def test_small_nested_patches_match_oracle(C, prec, relax):
    P = dict(box=64.0, a=1.0, fr0=1e-5)
    rho0, patches = _levels_case(32, P, [16, 24], 3, [16], 2, 700)
    assert len(patches) >= 4 and any(p["parent"] >= 0 for p in patches)
    dom, pres = O.solve_levels(rho0, [dict(parent=p["parent"], origin=p["origin"], rho=p["rho"])
                                      for p in patches], tol=1e-8, omega_m=OM, **P)
    u0 = torch.zeros(rho0.shape, dtype=torch.float64, device="cuda")
    gp = [dict(parent=p["parent"], origin=p["origin"], density=dev(p["rho"]),
               u=torch.zeros(p["rho"].shape, dtype=torch.float64, device="cuda"))
          for p in patches]
    st, stats = C.solve_levels(dev(rho0), u0, gp, tol=1e-8, omega_m=OM, prec=prec, relax=relax,
                               **P)
    assert st == 0
    assert np.abs(host(u0) - dom.u).max() <= 1e-6
    for g, r in zip(gp, pres):
        assert r.converged
        assert np.abs(host(g["u"]) - r.u).max() <= 1e-6


@pytest.mark.parametrize("tiling,fmg", [(-1, 0), (1, 0), (1, 1)])
def test_tiled_patch_levels_match_oracle(C, tiling, fmg):
    """Patches of 32^3 (coarse patch levels of 16^3, tiled with tiling=1: the
    tiled smoother, residual+restriction, prolongation and FAS right-hand side
    on Dirichlet grids) against the one-thread-per-cell kernels and the oracle;
    fmg=1 starts the domain solve by full multigrid (the patch starts from the
    interpolated parent solution, so it keeps its V-cycles)."""
    P = dict(box=64.0, a=1.0, fr0=1e-5)
    rho0, patches = _levels_case(32, P, [32], 2, [], 0, 720)
    assert len(patches) >= 1 and all(p["rho"].shape == (32, 32, 32) for p in patches)
    dom, pres = O.solve_levels(rho0, [dict(parent=p["parent"], origin=p["origin"], rho=p["rho"])
                                      for p in patches], tol=1e-8, omega_m=OM, **P)
    u0 = torch.zeros(rho0.shape, dtype=torch.float64, device="cuda")
    gp = [dict(parent=p["parent"], origin=p["origin"], density=dev(p["rho"]),
               u=torch.zeros(p["rho"].shape, dtype=torch.float64, device="cuda"))
          for p in patches]
    st, stats = C.solve_levels(dev(rho0), u0, gp, tol=1e-8, omega_m=OM, prec="mixed",
                               tiling=tiling, fmg=fmg, **P)
    assert st == 0
    assert np.abs(host(u0) - dom.u).max() <= 1e-6
    for g, r in zip(gp, pres):
        assert r.converged
        assert np.abs(host(g["u"]) - r.u).max() <= 1e-6


def test_full_nested_workload(C):
    """256^3 domain, 8-32 level-1 patches of 32^3-64^3 and level-2 patches inside
    them (lognormal sigma 2.5, |f_R0| = 1e-5), mixed precision."""
    N = 256
    P = dict(box=256.0, a=1.0, fr0=1e-5)
    rho0, patches = _levels_case(N, P, [32, 48, 64], 16, [32, 48], 12, 4000)
    u0 = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    gp = [dict(parent=p["parent"], origin=p["origin"], density=dev(p["rho"]),
               u=torch.zeros(p["rho"].shape, dtype=torch.float64, device="cuda"))
          for p in patches]
    st, stats = C.solve_levels(dev(rho0), u0, gp, tol=1e-8, omega_m=OM, prec="mixed", **P)
    assert st == 0
    assert all(s.res_rms <= 1e-8 for s in stats)
    ud = host(u0)
    assert sampled_residual(ud, rho0, h=1.0 / N, nsample=100, seed=1, **P) < 1e-6
    hs = []
    for t, (p, g) in enumerate(zip(patches, gp)):
        hp = (1.0 / N if p["parent"] < 0 else hs[p["parent"]]) / 2
        hs.append(hp)
        if t % 4 == 0:
            assert sampled_residual(host(g["u"]), p["rho"], h=hp, nsample=20, seed=t,
                                    interior=4, **P) < 1e-6


def test_batch_of_small_grids_with_forced_tiling(C):
    """Grids smaller than the shared-memory tiles (16^3, 32^3) in one batch with
    the tiled kernels forced on: halo coordinates wrap over several periods."""
    specs = [dict(n=16, fr0=1e-5, a=1.0, sigma=1.0, box=16.0, seed=31),
             dict(n=32, fr0=1e-5, a=0.7, sigma=2.0, box=32.0, seed=32),
             dict(n=16, fr0=1e-6, a=0.5, sigma=1.5, box=16.0, seed=33)]
    rhos = [synth.lognormal_density((s["n"],) * 3, s["seed"], sigma=s["sigma"]) for s in specs]
    us = [torch.zeros((s["n"],) * 3, dtype=torch.float64, device="cuda") for s in specs]
    st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[s["box"] for s in specs],
                              avals=[s["a"] for s in specs], fr0s=[s["fr0"] for s in specs],
                              omega_m=OM, tol=1e-8, prec="mixed", tiling=1)
    assert st == 0
    for s, r, u in zip(specs, rhos, us):
        ref = O.solve(r, tol=1e-8, box=s["box"], a=s["a"], omega_m=OM, fr0=s["fr0"])
        assert np.abs(host(u) - ref.u).max() <= 1e-6
