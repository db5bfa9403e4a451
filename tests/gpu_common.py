"""Shared helpers for the GPU tests: a context fixture and array round trips."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx():
    need_gpu()
    from paper_1110_1379_gb300 import frmg
    return frmg.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def local_block(u, k, j, i, r=3):
    """Periodic 2r^3 block of u centred so that cell (k,j,i) sits at (r,r,r)."""
    n2, n1, n0 = u.shape
    ks = (np.arange(k - r, k + r)) % n2
    js = (np.arange(j - r, j + r)) % n1
    is_ = (np.arange(i - r, i + r)) % n0
    return u[np.ix_(ks, js, is_)]
