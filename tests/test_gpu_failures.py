"""Failure paths of the solver, made on the host (nothing faults on the GPU).

* FR_EDIVERGED: an initial guess with one cell at u = 1000 makes e^u overflow,
  so the first residual is not finite; both precisions report the divergence,
  name it in fr_last_error() and still write the last iterate to u.
* FR_ENOMEM: a context created with a small device-workspace cap
  (FRMG_WORKSPACE_LIMIT) cannot hold a solve's workspace, so its allocator
  fails exactly as it does when cudaMalloc fails; a context without the cap
  then solves the same problem.
"""
import os

import numpy as np
import pytest

from gpu_common import ctx, dev, host, need_gpu, torch  # noqa: F401
from paper_1110_1379_gb300 import synth

pytestmark = pytest.mark.gpu
P = dict(box=64.0, a=1.0, omega_m=0.24, fr0=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overflowing_initial_guess_reports_divergence(prec):
    from paper_1110_1379_gb300 import frmg
    C = ctx()
    shape = (32, 32, 32)
    rho = dev(synth.lognormal_density(shape, 21, sigma=1.0))
    u0 = np.zeros(shape)
    u0[5, 6, 7] = 1000.0
    u = dev(u0)
    st, s = C.solve(rho, u, tol=1e-8, prec=prec, **P)
    assert st == frmg.FR_EDIVERGED, (st, s.as_dict())
    assert b"non-finite" in frmg.load().fr_last_error()
    # u holds an iterate of the right shape (the call did not abort half-way)
    assert host(u).shape == shape
    # the same context still solves a regular problem afterwards
    u.zero_()
    st, s = C.solve(rho, u, tol=1e-8, prec=prec, **P)
    assert st == frmg.FR_OK and s.res_rms <= 1e-8


def test_workspace_cap_reports_enomem(monkeypatch):
    from paper_1110_1379_gb300 import frmg
    need_gpu()
    shape = (64, 64, 64)
    rho = dev(synth.lognormal_density(shape, 22, sigma=1.0))
    monkeypatch.setenv("FRMG_WORKSPACE_LIMIT", str(1 << 20))
    C = frmg.Context(0)
    monkeypatch.delenv("FRMG_WORKSPACE_LIMIT")
    for prec in ("fp64", "mixed"):
        u = torch.zeros_like(rho)
        with pytest.raises(frmg.FRError) as ei:
            C.solve(rho, u, tol=1e-8, prec=prec, **P)
        assert ei.value.status == frmg.FR_ENOMEM
        assert b"workspace limit" in frmg.load().fr_last_error()
    phi = torch.zeros_like(rho)
    with pytest.raises(frmg.FRError) as ei:
        C.poisson(rho, torch.zeros_like(rho), phi, tol=1e-8, **P)
    assert ei.value.status == frmg.FR_ENOMEM
    C.close()
    C2 = frmg.Context(0)
    u = torch.zeros_like(rho)
    st, s = C2.solve(rho, u, tol=1e-8, prec="mixed", **P)
    assert st == frmg.FR_OK and s.res_rms <= 1e-8
    C2.close()
