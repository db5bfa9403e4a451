"""Allocation-free residual norm, checked against the regular residual entry point.

fr_residual_norm_noalloc is for callers that cannot allocate device memory
(memory owned by another allocator, no room for an allocation's
synchronisation).  Its rms and max of L(u) must equal those of the residual
that fr_residual returns, and those of the CPU oracle's residual, within the
residual tolerance of the other parity tests, on two calls in a row (the
second reuses the module's scratch array).  This file is named to be collected
last.
"""
import numpy as np
import pytest

from gpu_common import ctx, dev, torch
from oracle import oracle as O
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu


def _norms_from_residual(C, u, rho, faces, **P):
    d = torch.empty(u.shape, dtype=torch.float64, device="cuda")
    C.residual(u, rho, d, ub=faces, **P)
    torch.cuda.synchronize()
    return float(torch.sqrt((d * d).mean())), float(d.abs().max()), float(d.abs().max())


def test_noalloc_residual_norm_matches_residual_two_calls():
    from paper_1110_1379_gb300 import frmg
    C = ctx()
    cases = [((24, 20, 32), 11, False, dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)),
             ((16, 18, 40), 12, True, dict(box=256.0, a=0.6, omega_m=0.24, fr0=1e-4))]
    for shape, seed, with_faces, P in cases:
        rng = np.random.default_rng(seed)
        rho = dev(synth.lognormal_density(shape, seed, sigma=1.5))
        u = dev(rng.uniform(-2.0, 0.5, shape))
        faces = None
        if with_faces:
            nf = 2 * (shape[1] * shape[0] + shape[2] * shape[0] + shape[2] * shape[1])
            faces = dev(rng.uniform(-1.0, 0.5, nf))
        h = 1.0 / (2 * shape[2])
        rms_ref, max_ref, scale = _norms_from_residual(C, u, rho, faces, h=h, **P)
        # the oracle's FP64 residual of the same fields (independent of the GPU)
        d_or = O.residual(u.cpu().numpy(), rho.cpu().numpy(), h=h,
                          ub=None if faces is None else faces.cpu().numpy(), **P)
        rms_or, max_or = float(np.sqrt((d_or ** 2).mean())), float(np.abs(d_or).max())
        for _call in range(2):
            out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            st = frmg.residual_norm_noalloc(u, rho, out, h=h, ub=faces, **P)
            torch.cuda.synchronize()
            assert st == frmg.FR_OK
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(rms_ref, rel=1e-12, abs=1e-12 * scale)
            assert got[1] == pytest.approx(max_ref, rel=1e-12, abs=1e-12 * scale)
            assert got[0] == pytest.approx(rms_or, rel=1e-11, abs=1e-12 * scale)
            assert got[1] == pytest.approx(max_or, rel=1e-11, abs=1e-12 * scale)


def test_noalloc_rejects_oversize_and_host_pointers():
    from paper_1110_1379_gb300 import frmg
    ctx()
    small = torch.ones((4, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    host_u = np.zeros((4, 4, 4))
    st = frmg.residual_norm_noalloc(host_u, small, out, box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)
    assert st == frmg.FR_EINVAL
    # a grid above the 2^25-cell limit is refused before anything is read
    big = torch.empty((2, 4096, 4098), dtype=torch.float64, device="cuda")
    st = frmg.residual_norm_noalloc(big, big, out, box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)
    assert st == frmg.FR_EINVAL
    assert b"limit" in frmg.load().fr_last_error()
