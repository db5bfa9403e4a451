"""The C-ABI library loads and exports every function include/frmg.h declares.
No GPU needed: nothing here calls into compute."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "frmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fr_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_1379_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fr_solve", "fr_solve_levels", "fr_solve_batch", "fr_cic_assign",
                     "fr_ctx_create", "fr_ctx_destroy", "fr_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    h = ctypes.CDLL(lib)
    for name in declared_functions():
        assert hasattr(h, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header():
    from paper_1110_1379_gb300 import frmg
    assert set(frmg.EXPORTS) == set(declared_functions())


def test_product_library_does_not_contain_the_oracle(lib):
    out = subprocess.run(["nm", "-D", lib], capture_output=True, text=True).stdout
    assert "orc_" not in out
    for fn in ("frmg.py", "build.py"):
        txt = open(os.path.join(ROOT, "paper_1110_1379_gb300", fn)).read()
        assert "oracle" not in txt.lower().replace("no cpu fallback", "")


def test_constants_without_gpu(lib):
    from paper_1110_1379_gb300 import frmg
    import paper_fields as PF
    al, be, ga, ct, fb, ub = frmg.constants(256.0, 512, 1.0, 0.24, 1e-4)
    ra, rb, rg = PF.coefficients(256.0, 512, 1.0, 0.24, 1e-4)
    assert al == pytest.approx(ra, rel=1e-13)
    assert be == pytest.approx(rb, rel=1e-13)
    assert ga == pytest.approx(rg, rel=1e-13)
    assert ct == pytest.approx(PF.ctilde(256.0), rel=1e-14)
    with pytest.raises(frmg.FRError):
        frmg.constants(-1.0, 32, 1.0, 0.24, 1e-5)
