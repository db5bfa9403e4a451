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


def test_options_struct_matches_the_header(lib):
    """fr_opts_default through the binding's struct: every documented default
    lands in its field (a layout mismatch would scramble them), and the struct
    fields follow the header's member order."""
    from paper_1110_1379_gb300 import frmg
    o = frmg.Context.opts()
    assert (o.tol, o.max_vcycles, o.pre, o.post, o.prec) == (1e-8, 100, 2, 2, frmg.FR_FP64)
    assert (o.newton_step_cap, o.inner_cycles, o.max_outer) == (1.0, 2, 40)
    assert (o.allow_negative_density, o.use_graph, o.temporal_depth, o.tiling) == (0, 1, 0, 0)
    assert (o.defect_precision, o.tau_alpha, o.relax, o.fmg, o.initial_guess) == (0, 0.0, 1.0, 0, 1)
    assert o.smooth_tile == 0
    src = open(os.path.join(ROOT, "include", "frmg.h")).read()
    body = src[src.index("typedef struct {\n    double tol;"):src.index("} fr_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    members = re.findall(r"\b(?:double|int|fr_precision)\s+([a-z_0-9, ]+);", body)
    names = [m.strip() for grp in members for m in grp.split(",")]
    assert names == [f for f, _ in frmg.fr_opts._fields_]


def test_stats_struct_matches_the_header():
    from paper_1110_1379_gb300 import frmg
    src = open(os.path.join(ROOT, "include", "frmg.h")).read()
    body = src[src.index("typedef struct {\n    int vcycles;"):src.index("} fr_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(?:double|int)\s+([a-z_0-9]+)(?:\[[A-Z_]+\])?;", body)
    assert names == [f for f, _ in frmg.fr_stats._fields_]
    assert frmg.FR_HIST == int(re.search(r"#define FR_HIST (\d+)", src).group(1))


def test_no_gpu_fails_loudly(lib):
    """Without a usable GPU the library refuses to create a context (FR_ECUDA
    with the CUDA error in the message) instead of computing anywhere else."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1110_1379_gb300 import frmg
    with pytest.raises(frmg.FRError) as ei:
        frmg.Context(0)
    assert ei.value.status == frmg.FR_ECUDA
    assert "fr_ctx_create" in str(ei.value)


def test_status_strings_name_every_code(lib):
    """fr_status_string names each fr_status code of the header and falls back
    for unknown values; the binding's constants match the header's enum."""
    from paper_1110_1379_gb300 import frmg
    h = frmg.load()
    src = open(os.path.join(ROOT, "include", "frmg.h")).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"\b(FR_E?[A-Z]+) = (\d+)", src))
    assert codes["FR_OK"] == 0 and len(codes) >= 7
    for name, v in codes.items():
        if name in ("FR_FP64", "FR_MIXED"):
            continue
        assert getattr(frmg, name) == v
        assert h.fr_status_string(v).decode().startswith(name)
    for v in (-1, 99):
        assert h.fr_status_string(v) == b"unknown status"
