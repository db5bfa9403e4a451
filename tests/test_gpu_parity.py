"""GPU (CUDA, C ABI) against the FP64 oracle, step by step and end to end.

Tolerances:
* one FP64 step (sweep, residual, restriction, prolongation, boundary set-up):
  the two sides evaluate the same formulas in a different rounding order, so
  they agree to ~1e-12 relative; tests use 1e-10 (absolute in u, relative to
  the largest term for residuals).
* a converged solve at rms residual <= 1e-8: both sides sit within
  tol / (beta/2) ~ 1e-8 of the unique discrete solution, so |u_gpu - u_oracle|
  <= 1e-6 (the stated target) with a large margin.
"""
import numpy as np
import pytest

import paper_fields as PF
from gpu_common import ctx, dev, host, local_block, torch  # noqa: F401
from oracle import oracle as O
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu

CFG1 = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)


@pytest.fixture(scope="module")
def C():
    return ctx()


def _field(shape, seed, sigma=1.0):
    return synth.lognormal_density(shape, seed, sigma=sigma)


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("shape", [(32, 32, 32), (12, 20, 36), (4, 4, 4), (2, 2, 2)])
@pytest.mark.parametrize("nsweeps", [1, 3])
def test_smooth_matches_oracle(C, shape, nsweeps):
    rho = _field(shape, 11, sigma=1.5)
    rng = np.random.default_rng(2)
    u0 = rng.uniform(-0.5, 0.3, shape)
    f = rng.standard_normal(shape) * 0.1
    h = 1.0 / shape[2]
    ref = O.smooth(u0, rho, nsweeps, h=h, f=f, **CFG1)
    u = dev(u0)
    C.smooth(u, dev(rho), nsweeps, h=h, f=dev(f), **CFG1)
    assert np.abs(host(u) - ref).max() < 1e-10


def test_smooth_patch_faces_match_oracle(C):
    shape = (10, 8, 12)
    rho = _field(shape, 3)
    rng = np.random.default_rng(5)
    u0 = rng.uniform(-0.5, 0.3, shape)
    ub = rng.uniform(-0.8, 0.4, sum(O.face_sizes(shape)))
    h = 1.0 / 64
    ref = O.smooth(u0, rho, 2, h=h, ub=ub, **CFG1)
    u = dev(u0)
    C.smooth(u, dev(rho), 2, h=h, ub=dev(ub), **CFG1)
    assert np.abs(host(u) - ref).max() < 1e-10


@pytest.mark.parametrize("with_faces", [False, True])
def test_residual_matches_oracle(C, with_faces):
    shape = (16, 12, 20)
    rho = _field(shape, 8, sigma=2.0)
    rng = np.random.default_rng(9)
    u0 = rng.uniform(-2.0, 0.5, shape)
    f = rng.standard_normal(shape)
    ub = rng.uniform(-1, 0.5, sum(O.face_sizes(shape))) if with_faces else None
    P = dict(h=1.0 / 40, f=f, ub=ub, **CFG1)
    ref = O.residual(u0, rho, **P)
    d = torch.empty(shape, dtype=torch.float64, device="cuda")
    C.residual(dev(u0), dev(rho), d, h=P["h"], f=dev(f),
               ub=None if ub is None else dev(ub), **CFG1)
    scale = np.abs(ref).max()
    assert np.abs(host(d) - ref).max() < 1e-12 * max(scale, 1.0)


def test_restrict_and_prolong_match_oracle(C):
    rng = np.random.default_rng(4)
    fine = rng.standard_normal((12, 8, 16))
    c = torch.empty((6, 4, 8), dtype=torch.float64, device="cuda")
    C.restrict(dev(fine), c)
    assert np.abs(host(c) - O.restrict(fine)).max() < 1e-15
    uH = rng.standard_normal((6, 4, 8))
    uR = rng.standard_normal((6, 4, 8))
    for dirichlet in (False, True):
        uf = dev(fine)
        C.prolong_correct(uf, dev(uH), dev(uR), dirichlet=dirichlet)
        ref = O.prolong_correct(fine, uH, uR, dirichlet=dirichlet)
        assert np.abs(host(uf) - ref).max() < 1e-14


@pytest.mark.parametrize("periodic,origin", [(True, (0, 3, 14)), (False, (2, 3, 4))])
def test_patch_bc_matches_oracle(C, periodic, origin):
    rng = np.random.default_rng(6)
    up = rng.standard_normal((14, 12, 16))
    n = (6, 8, 10)
    ui_ref, ub_ref = O.patch_bc(up, origin, n, parent_periodic=periodic)
    ui = torch.empty(n, dtype=torch.float64, device="cuda")
    ub = torch.empty(sum(O.face_sizes(n)), dtype=torch.float64, device="cuda")
    C.patch_bc(dev(up), origin, ui, ub, periodic=periodic)
    assert np.abs(host(ui) - ui_ref).max() < 1e-14
    assert np.abs(host(ub) - ub_ref).max() < 1e-14


# ------------------------------------------------------------------ V-cycles
@pytest.mark.parametrize("shape", [(32, 32, 32), (40, 24, 48), (48, 48, 48)])
@pytest.mark.parametrize("ncyc", [1, 3])
def test_fp64_vcycles_match_oracle(C, shape, ncyc):
    """Identical V-cycles (same ordering, restriction, coarsest rule) give the
    same iterate up to rounding."""
    rho = _field(shape, 1000, sigma=1.0)
    P = dict(box=64.0 * shape[2] / 32, a=1.0, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho, ncycles=ncyc, **P)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    s = C.vcycles(dev(rho), u, ncyc, **P)
    assert np.abs(host(u) - ref.u).max() < 1e-10
    # the library reduces norms in FP32 per block (a stopping signal): 1e-5 relative
    assert s.res_rms == pytest.approx(ref.hist[-1], rel=1e-5, abs=1e-13)


# ------------------------------------------------------------------ full solves
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_config1_matches_oracle(C, prec):
    shape = (32, 32, 32)
    rho = _field(shape, 1000, sigma=1.0)
    ref = O.solve(rho, tol=1e-8, **CFG1)
    assert ref.converged
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec=prec, **CFG1)
    assert st == 0
    assert s.res_rms <= 1e-8
    assert np.abs(host(u) - ref.u).max() <= 1e-6
    if prec == "fp64":
        assert s.vcycles == ref.cycles
        assert np.abs(host(u) - ref.u).max() <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("fr0,box,sigma", [(1e-4, 256.0, 2.0), (1e-6, 256.0, 2.0),
                                           (1e-5, 128.0, 2.5)])
def test_solve_screened_regimes_match_oracle(C, prec, fr0, box, sigma):
    shape = (48, 48, 48)
    rho = _field(shape, 3000 + int(-np.log10(fr0)), sigma=sigma)
    P = dict(box=box, a=1.0, omega_m=0.24, fr0=fr0)
    ref = O.solve(rho, tol=1e-8, **P)
    assert ref.converged
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec=prec, **P)
    assert st == 0 and s.res_rms <= 1e-8
    assert np.abs(host(u) - ref.u).max() <= 1e-6


@pytest.mark.parametrize("a", [0.5, 1.0])
def test_solve_cic_config_matches_oracle(C, a):
    """Particles -> CIC density -> solve, both sides from the same positions."""
    n = 32
    pos = synth.zeldovich_positions(n, 2000, amplitude=0.02)
    rho_ref = O.cic(pos, (n, n, n))
    rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    C.cic(dev(pos), rho)
    assert np.abs(host(rho) - rho_ref).max() < 1e-12 * rho_ref.max()
    P = dict(box=32.0, a=a, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho_ref, tol=1e-8, **P)
    u = torch.zeros_like(rho)
    st, s = C.solve(rho, u, tol=1e-8, **P)
    assert st == 0
    assert np.abs(host(u) - ref.u).max() <= 1e-6


def test_sine_closed_form_on_gpu(C):
    """Sec. VI.A.3 on the GPU: same second-order approach to the closed form."""
    P = dict(box=256.0, a=1.0, omega_m=0.24, fr0=1e-5)
    errs = []
    for n in (32, 64):
        rho, ue = PF.sine_field(n, **P)
        u = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        st, _ = C.solve(dev(rho), u, tol=1e-11, allow_negative_density=1, **P)
        assert st == 0
        errs.append(np.abs(host(u) - ue).max())
    assert 1.9 < np.log2(errs[0] / errs[1]) < 2.1


# ------------------------------------------------------------------ host memory path
def test_host_pointers_same_as_device(C):
    shape = (16, 16, 16)
    rho = _field(shape, 5)
    u_host = np.zeros(shape)
    st, _ = C.solve(rho, u_host, tol=1e-9, **CFG1)
    assert st == 0
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    C.solve(dev(rho), u, tol=1e-9, **CFG1)
    assert np.abs(host(u) - u_host).max() < 1e-14


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("initial_guess", [0, 1])
def test_mixed_host_output_equals_device(C, pinned, initial_guess):
    """A host u (page-locked: copied out early, while the last defect is
    checked; pageable: copied at the end) receives exactly the device result,
    also when the solve needs more than one outer step."""
    shape = (48, 32, 64)
    rho = _field(shape, 4300, sigma=2.0)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    ud = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, sd = C.solve(dev(rho), ud, tol=1e-9, prec="mixed", initial_guess=initial_guess, **P)
    assert st == 0 and sd.outer >= 2
    uh = torch.zeros(shape, dtype=torch.float64, pin_memory=pinned)
    rh = torch.from_numpy(rho)
    if pinned:
        rh = rh.pin_memory()
    st, sh = C.solve(rh, uh, tol=1e-9, prec="mixed", initial_guess=initial_guess, **P)
    assert st == 0 and sh.vcycles == sd.vcycles and sh.outer == sd.outer
    assert np.array_equal(uh.numpy(), host(ud))
    assert sd.host_copies == 0 and sh.host_copies >= 1
    if not pinned:
        assert sh.host_copies == 1  # pageable memory: copied once, at the end


# ------------------------------------------------------------------ edge cases
def test_invalid_arguments(C):
    from paper_1110_1379_gb300 import frmg
    rho = torch.ones((8, 8, 7), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(rho)
    with pytest.raises(frmg.FRError) as e:
        C.solve(rho, u, **CFG1)
    assert e.value.status == frmg.FR_EINVAL
    rho = torch.ones((8, 8, 8), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(rho)
    rho[1, 2, 3] = float("nan")
    with pytest.raises(frmg.FRError):
        C.solve(rho, u, **CFG1)
    rho[1, 2, 3] = -0.5
    with pytest.raises(frmg.FRError):
        C.solve(rho, u, **CFG1)
    st, _ = C.solve(rho, u, allow_negative_density=1, **CFG1)
    assert st == 0
    with pytest.raises(frmg.FRError):
        C.solve(torch.ones_like(rho), u, box=64.0, a=-1.0, omega_m=0.24, fr0=1e-5)


def test_no_convergence_reports_and_writes_u(C):
    from paper_1110_1379_gb300 import frmg
    shape = (16, 16, 16)
    rho = _field(shape, 7, sigma=1.5)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-12, max_vcycles=1, **CFG1)
    assert st == frmg.FR_ENOCONV
    assert s.vcycles == 1
    ref = O.solve(rho, ncycles=1, **CFG1)
    assert np.abs(host(u) - ref.u).max() < 1e-10


def test_homogeneous_and_tiny_grids(C):
    for shape in [(2, 2, 2), (4, 4, 4), (6, 6, 6)]:
        rng = np.random.default_rng(1)
        u = dev(rng.uniform(-1, 1, shape))
        st, s = C.solve(dev(np.ones(shape)), u, tol=1e-12, **CFG1)
        assert st == 0
        assert np.abs(host(u)).max() < 1e-10


# ------------------------------------------------------------------ FP32 smoothing (mixed path)
def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


F32_SHAPES = [(32, 32, 32), (20, 36, 70), (16, 18, 130)]


@pytest.mark.parametrize("shape", F32_SHAPES)
@pytest.mark.parametrize("bg", [False, True])
@pytest.mark.parametrize("faces", [False, True])
@pytest.mark.parametrize("nsweeps", [1, 2, 3])
def test_f32_tiled_smoother_equals_simple(C, shape, bg, faces, nsweeps):
    """The shared-memory temporally blocked kernel performs the same sweeps as
    the one-colour-per-launch kernel (same formulas; FP32 rounding only)."""
    rng = np.random.default_rng(17)
    u0 = rng.uniform(-0.3, 0.3, shape) if bg else rng.uniform(-1.5, 0.3, shape)
    f = rng.standard_normal(shape) * 0.3
    b = rng.uniform(-1.5, 0.3, shape) if bg else None
    ub = rng.uniform(-1.5, 0.3, sum(O.face_sizes(shape))) if faces else None
    P = dict(box=128.0, a=0.9, omega_m=0.24, fr0=1e-5, h=1.0 / 48)
    outs = []
    for tiled in (False, True):
        u = _f32(u0)
        C.smooth_f32(u, nsweeps, bg=None if b is None else _f32(b), f=_f32(f),
                     ub=None if ub is None else _f32(ub), tiled=tiled, **P)
        outs.append(host(u).astype(np.float64))
    assert np.abs(outs[0] - outs[1]).max() < 2e-6


@pytest.mark.parametrize("shape", F32_SHAPES + [(64, 48, 256), (40, 130, 66)])
@pytest.mark.parametrize("bg", [False, True])
@pytest.mark.parametrize("faces", [False, True])
@pytest.mark.parametrize("nsweeps", [1, 2, 3])
def test_register_column_smoother_is_the_ring_smoother(C, shape, bg, faces, nsweeps):
    """The register-column one-sweep kernels (plain form on 64 x 8 and 64 x 16
    tiles, correction form on 64 x 8) perform the same sweeps as the
    shared-memory plane-ring kernels, bit for bit: same cells, same face order,
    same arithmetic (x = expm1(u) recomputed from u equals the cached x).  The
    patch faces of the correction form are the exception: there the compiler
    contracts the ghost terms into fused multiply-adds differently in the two
    kernels, so they agree to FP32 rounding."""
    rng = np.random.default_rng(31)
    u0 = rng.uniform(-0.3, 0.3, shape) if bg else rng.uniform(-1.5, 0.3, shape)
    f = rng.standard_normal(shape) * 0.3
    b = rng.uniform(-1.5, 0.3, shape) if bg else None
    ub = rng.uniform(-1.5, 0.3, sum(O.face_sizes(shape))) if faces else None
    P = dict(box=128.0, a=0.9, omega_m=0.24, fr0=1e-5, h=1.0 / 48)
    outs = {}
    for tiled in (1, 8, 16):
        u = _f32(u0)
        C.smooth_f32(u, nsweeps, bg=None if b is None else _f32(b), f=_f32(f),
                     ub=None if ub is None else _f32(ub), tiled=tiled, **P)
        outs[tiled] = host(u)
    if bg and faces:
        for t in (8, 16):
            assert np.abs(outs[1].astype(np.float64) - outs[t]).max() < 2e-6
        return
    assert np.array_equal(outs[1], outs[8])
    assert np.array_equal(outs[1], outs[16])


@pytest.mark.parametrize("bg", [False, True])
@pytest.mark.parametrize("faces", [False, True])
def test_f32_smoother_matches_oracle(C, bg, faces):
    """FP32 sweeps (plain, and in the correction form on a background) track
    the FP64 oracle's sweeps of the same full-variable equation."""
    shape = (24, 20, 36)
    rng = np.random.default_rng(23)
    P = dict(box=128.0, a=1.0, omega_m=0.24, fr0=1e-5, h=1.0 / 40)
    ub = rng.uniform(-1.2, 0.3, sum(O.face_sizes(shape))) if faces else None
    ones = np.ones(shape)
    if bg:
        b = rng.uniform(-1.2, 0.3, shape).astype(np.float32).astype(np.float64)
        d0 = rng.uniform(-0.05, 0.05, shape).astype(np.float32).astype(np.float64)
        r = (rng.standard_normal(shape) * 0.05).astype(np.float32).astype(np.float64)
        # full-variable equation A(u) = r + A(bg) with u0 = bg + d0
        Abg = O.residual(b, ones, ub=ub, **P)
        ref = O.smooth(b + d0, ones, 2, f=r + Abg, ub=ub, **P)
        u = _f32(d0)
        C.smooth_f32(u, 2, bg=_f32(b), f=_f32(r), ub=None if ub is None else _f32(ub), **P)
        got = b + host(u).astype(np.float64)
    else:
        u0 = rng.uniform(-1.2, 0.3, shape).astype(np.float32).astype(np.float64)
        f = (rng.standard_normal(shape) * 0.3).astype(np.float32).astype(np.float64)
        ref = O.smooth(u0, ones, 2, f=f, ub=ub, **P)
        u = _f32(u0)
        C.smooth_f32(u, 2, f=_f32(f), ub=None if ub is None else _f32(ub), **P)
        got = host(u).astype(np.float64)
    assert np.abs(got - ref).max() < 2e-5


@pytest.mark.parametrize("tiling", [-1, 1])
@pytest.mark.parametrize("tdepth", [1, 2])
@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 40, 96)])
def test_mixed_tiled_and_plain_kernels_match_oracle(C, tiling, tdepth, shape):
    """The shared-memory FP32 kernels (smoother with 1 or 2 sweeps per pass,
    residual + restriction) and the one-thread-per-cell kernels both drive the
    mixed solve to the oracle's solution."""
    rho = _field(shape, 4000, sigma=2.0)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho, tol=1e-8, **P)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec="mixed", tiling=tiling, temporal_depth=tdepth,
                    **P)
    assert st == 0 and s.res_rms <= 1e-8
    assert np.abs(host(u) - ref.u).max() <= 1e-6
    assert s.vcycles <= 2 * ref.cycles + 4


# ------------------------------------------------------------------ double-float defect
@pytest.mark.parametrize("fr0,box", [(1e-4, 256.0), (1e-5, 128.0), (1e-6, 64.0)])
@pytest.mark.parametrize("faces", [False, True])
@pytest.mark.parametrize("shape", [(24, 20, 32), (6, 10, 14)])
def test_double_float_defect_matches_fp64(C, fr0, box, faces, shape):
    """The mixed loop's defect in double-float arithmetic agrees with the FP64
    oracle residual to ~1e-13 of the size of the operator's terms, both for a
    random u (large residual) and, on the first shape, at a converged solution
    (the cancellation the convergence test depends on).  Two cells per
    thread in packed pairs; the last block of (6, 10, 14) is part-filled."""
    rho = _field(shape, 77, sigma=2.0)
    P = dict(box=box, a=1.0, omega_m=0.24, fr0=fr0)
    rng = np.random.default_rng(8)
    ub = rng.uniform(-2.0, 0.5, sum(O.face_sizes(shape))) if faces else None
    alpha, beta, gamma = PF.coefficients(box, shape[2], 1.0, 0.24, fr0)
    us = [rng.uniform(-3.0, 0.8, shape)]
    if shape == (24, 20, 32):
        us.append(O.solve(rho, tol=1e-12, ub=ub, h=1.0 / shape[2], **P).u)
    for u in us:
        ref = O.residual(u, rho, ub=ub, **P)
        d = torch.empty(shape, dtype=torch.float64, device="cuda")
        C.residual_df(dev(u), dev(rho), d, ub=None if ub is None else dev(ub), **P)
        # size of the largest flux term, alpha e^u |du| with |du| up to ~4
        term = alpha * np.exp(np.abs(u).max()) * 4.0
        assert np.abs(host(d) - ref).max() < 2e-13 * term + 1e-12


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 40, 96)])
def test_mixed_defect_precisions_agree(C, shape):
    """Double-float and FP64 defects drive the mixed loop to the same solution."""
    rho = _field(shape, 5000, sigma=2.0)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    outs = []
    for dp in (0, 1):
        u = torch.zeros(shape, dtype=torch.float64, device="cuda")
        st, s = C.solve(dev(rho), u, tol=1e-10, prec="mixed", defect_precision=dp, **P)
        assert st == 0 and s.res_rms <= 1e-10
        outs.append(host(u))
    assert np.abs(outs[0] - outs[1]).max() < 1e-9


def test_autotune_returns_a_converging_setting(C):
    shape = (32, 32, 32)
    rho = _field(shape, 1000, sigma=1.0)
    best, secs = C.autotune(dev(rho), tol=1e-8, prec="mixed", **CFG1)
    assert (best["pre"], best["post"]) in [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3)]
    assert best["temporal_depth"] in (1, 2) and secs > 0
    assert best["relax"] in (1.0, 1.15, 1.25)
    assert best["smooth_tile"] in (16, 8, -1)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec="mixed", pre=best["pre"], post=best["post"],
                    temporal_depth=best["temporal_depth"], relax=best["relax"],
                    smooth_tile=best["smooth_tile"], **CFG1)
    assert st == 0
    assert np.abs(host(u) - O.solve(rho, tol=1e-8, **CFG1).u).max() <= 1e-6


# ------------------------------------------------------------------ over-relaxation
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("relax", [1.15, 1.25])
@pytest.mark.parametrize("tiling", [-1, 1])
def test_over_relaxed_solve_reaches_oracle_solution(C, prec, relax, tiling):
    """u += w du in every Newton-GS update changes the path, not the discrete
    solution: the solve still ends at the oracle's (plain Newton-GS) solution."""
    shape = (48, 32, 64)
    rho = _field(shape, 4100, sigma=2.0)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho, tol=1e-8, **P)
    assert ref.converged
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec=prec, relax=relax, tiling=tiling, **P)
    assert st == 0 and s.res_rms <= 1e-8
    assert np.abs(host(u) - ref.u).max() <= 1e-6


@pytest.mark.parametrize("shape,relax", [((48, 32, 64), 1.0), ((48, 32, 64), 1.15),
                                         ((32, 32, 32), 1.25), ((12, 20, 36), 1.0)])
def test_fmg_start_reaches_oracle_solution(C, shape, relax):
    """The full-multigrid start changes the first iterate, not the solution."""
    rho = _field(shape, 4200, sigma=2.0)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho, tol=1e-8, **P)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-8, prec="mixed", relax=relax, fmg=1, **P)
    assert st == 0 and s.res_rms <= 1e-8
    assert np.abs(host(u) - ref.u).max() <= 1e-6
    # the first entry of the residual history (first V-cycle after the start)
    # lies well below the residual of u = 0
    assert s.hist[0] < 0.5 * s.res0_rms


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_initial_guess_zero_does_not_read_u(C, prec):
    """initial_guess=0: u is output only (host NaNs are neither copied in nor
    read); the result equals the solve from a zeroed u, bit for bit."""
    shape = (32, 32, 32)
    rho = _field(shape, 1000, sigma=1.0)
    u0 = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s0 = C.solve(dev(rho), u0, tol=1e-8, prec=prec, **CFG1)
    assert st == 0
    for host_u in (False, True):
        u1 = torch.full(shape, float("nan"), dtype=torch.float64,
                        device="cpu" if host_u else "cuda")
        st, s1 = C.solve(dev(rho), u1, tol=1e-8, prec=prec, initial_guess=0, **CFG1)
        assert st == 0 and s1.vcycles == s0.vcycles
        assert np.array_equal(host(u1), host(u0))
    from paper_1110_1379_gb300 import frmg
    with pytest.raises(frmg.FRError):
        C.solve(dev(rho), u0, initial_guess=2, **CFG1)


def test_zero_start_validates_density(C):
    """The mixed zero start validates rho in its fused first pass: NaN and
    (unless allowed) negative values are rejected as on every other path."""
    from paper_1110_1379_gb300 import frmg
    shape = (16, 16, 16)
    rho = _field(shape, 1500, sigma=0.5)
    for bad, allow, ok in ((np.nan, 0, False), (np.inf, 0, False), (-0.2, 0, False),
                           (-0.2, 1, True), (-0.0, 0, True)):
        r = rho.copy()
        r[3, 4, 5] = bad
        u = torch.zeros(shape, dtype=torch.float64, device="cuda")
        if ok:
            st, s = C.solve(dev(r), u, tol=1e-8, prec="mixed", initial_guess=0,
                            allow_negative_density=allow, **CFG1)
            assert st == 0
        else:
            with pytest.raises(frmg.FRError) as e:
                C.solve(dev(r), u, tol=1e-8, prec="mixed", initial_guess=0,
                        allow_negative_density=allow, **CFG1)
            assert e.value.status == frmg.FR_EINVAL


def test_relax_out_of_range_rejected(C):
    from paper_1110_1379_gb300 import frmg
    rho = torch.ones((8, 8, 8), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(rho)
    for w in (0.0, -0.5, 2.0, float("nan")):
        with pytest.raises(frmg.FRError) as e:
            C.solve(rho, u, relax=w, **CFG1)
        assert e.value.status == frmg.FR_EINVAL


# ------------------------------------------------------------------ CUDA graphs
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("on_side_stream", [False, True])
def test_graph_replay_is_bit_identical(C, prec, on_side_stream):
    """V-cycles replayed from a captured graph give the same bits and the same
    kernel count as direct launches, on the legacy default stream (the solve
    moves to the context's own stream) and on a caller's stream."""
    shape = (32, 32, 32)
    rho = _field(shape, 1200, sigma=1.5)
    d = dev(rho)
    outs, counts = [], []
    s = torch.cuda.Stream() if on_side_stream else None
    for g in (0, 1):
        u = torch.zeros(shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        n0 = C.launches
        if s is not None:
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                st, stats = C.solve(d, u, tol=1e-9, prec=prec, use_graph=g, **CFG1)
            torch.cuda.current_stream().wait_stream(s)
        else:
            st, stats = C.solve(d, u, tol=1e-9, prec=prec, use_graph=g, **CFG1)
        assert st == 0 and stats.vcycles >= 3
        counts.append(C.launches - n0)
        outs.append(host(u))
    assert np.array_equal(outs[0], outs[1])
    assert counts[0] == counts[1]


@pytest.mark.parametrize("pre,post,tdepth", [(2, 1, 1), (1, 2, 1), (1, 0, 1), (3, 2, 2)])
def test_odd_pass_plans_single_field(C, pre, post, tdepth):
    """A V-cycle with an odd number of ping-pong smoother passes per level leaves
    each level in its other buffer; graph replay (one graph per buffer-parity
    state) gives the same bits as direct launches, and both reach the oracle's
    solution."""
    shape = (32, 48, 64)
    rho = _field(shape, 1250, sigma=1.5)
    P = dict(box=2.0 * shape[2], a=1.0, omega_m=0.24, fr0=1e-5)
    ref = O.solve(rho, tol=1e-8, **P)
    outs, counts = [], []
    for g in (0, 1):
        u = torch.zeros(shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        n0 = C.launches
        st, stats = C.solve(dev(rho), u, tol=1e-8, prec="mixed", pre=pre, post=post,
                            temporal_depth=tdepth, tiling=1, use_graph=g,
                            stream=torch.cuda.current_stream(), **P)
        assert st == 0 and stats.res_rms <= 1e-8 and stats.vcycles >= 4
        counts.append(C.launches - n0)
        outs.append(host(u))
    assert np.array_equal(outs[0], outs[1])
    assert counts[0] == counts[1]
    assert np.abs(outs[1] - ref.u).max() <= 1e-6


def test_odd_pass_plan_batch_matches_oracle(C):
    """A batch with V(2,1) runs the in-place smoother (the parity of a field
    that has left the inner solve must not flip) and still reaches every
    field's oracle solution."""
    rhos = [_field((16, 16, 16), 1400 + i, sigma=0.5 + 0.6 * i) for i in range(3)]
    us = [torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda") for _ in rhos]
    st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[32.0] * 3, avals=[1.0] * 3,
                              fr0s=[1e-5] * 3, omega_m=0.24, tol=1e-8, prec="mixed", pre=2,
                              post=1, tiling=1)
    assert st == 0
    for r, u in zip(rhos, us):
        ref = O.solve(r, tol=1e-8, box=32.0, a=1.0, omega_m=0.24, fr0=1e-5)
        assert np.abs(host(u) - ref.u).max() <= 1e-6


def test_graph_replay_batch_with_fields_leaving(C):
    """Batched solve where fields stop at different cycles: the graph reads the
    per-field active flags from device memory, so replay stays exact."""
    rhos = [_field((16, 16, 16), 1300 + i, sigma=0.5 + 0.6 * i) for i in range(4)]
    res = []
    for g in (0, 1):
        us = [torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda") for _ in rhos]
        st, stats = C.solve_batch([dev(r) for r in rhos], us, boxes=[32.0] * 4,
                                  avals=[1.0] * 4, fr0s=[1e-5] * 4, omega_m=0.24, tol=1e-9,
                                  prec="mixed", use_graph=g)
        assert st == 0
        res.append(([host(u) for u in us], [x.vcycles for x in stats]))
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    assert res[0][1] == res[1][1]


# ------------------------------------------------------- truncation-error rule (Sec. V.B.2)
def test_truncation_error_rule_fp64_matches_oracle(C):
    """FP64 solve with tau_alpha = 1/3: the reported tau is the oracle's
    L^H(R u) - R L^h(u) at the returned u (same arithmetic class, FP64), and the
    solve stops once rms(d) <= tau_alpha rms(tau), before a tight tolerance."""
    shape = (32, 32, 32)
    rho = _field(shape, 1000, sigma=1.0)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-13, prec="fp64", tau_alpha=1.0 / 3.0, **CFG1)
    assert st == 0
    tau = O.truncation_error(host(u), rho, **CFG1)
    tref = float(np.sqrt(np.mean(tau ** 2)))
    # the GPU sums tau^2 per block in FP32 (256 terms): ~1e-6 relative on the norm
    assert s.tau_rms == pytest.approx(tref, rel=1e-5)
    assert s.res_rms <= max(1e-13, s.tau_rms / 3.0)
    u2 = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st2, s2 = C.solve(dev(rho), u2, tol=1e-13, prec="fp64", **CFG1)
    assert st2 == 0 and s2.vcycles > s.vcycles and np.isnan(s2.tau_rms)


def test_truncation_error_rule_mixed(C):
    """Mixed solve: tau from the FP32 full-variable phase, close to the oracle's
    tau at the returned u; the defect ends below tau_alpha rms(tau)."""
    shape = (32, 32, 32)
    rho = _field(shape, 1000, sigma=1.0)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, s = C.solve(dev(rho), u, tol=1e-13, prec="mixed", tau_alpha=1.0 / 3.0, **CFG1)
    assert st == 0
    tref = float(np.sqrt(np.mean(O.truncation_error(host(u), rho, **CFG1) ** 2)))
    assert s.tau_rms == pytest.approx(tref, rel=2e-2)
    assert s.res_rms <= s.tau_rms / 3.0
