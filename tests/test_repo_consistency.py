"""Host-side consistency of the repository's own references (no GPU).

* every `python bench.py ...` command in the profile summaries parses with
  bench.py's own argument parser (the summaries give runnable commands);
* every repository path that README.md name exists.
"""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _profile_bench_commands():
    cmds = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            i = line.find("python bench.py")
            if i >= 0:
                cmds.append((os.path.basename(path), line[i + len("python bench.py"):].strip()))
    return cmds


def test_profile_commands_parse(monkeypatch):
    import bench
    cmds = _profile_bench_commands()
    assert len(cmds) >= 5
    for name, tail in cmds:
        argv = shlex.split(tail.split(">")[0])
        monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
        args = bench.parse_args()
        assert args.steps >= 1, name
        if args.options:
            assert bench.parse_options(args.options), name


@pytest.mark.parametrize("doc", ["DESIGN.md", "README.md"])
def test_named_paths_exist(doc):
    text = open(os.path.join(ROOT, doc)).read()
    names = set(re.findall(r"`((?:tests|oracle|profiles|include|paper_1110_1379_gb300|csrc)/"
                           r"[A-Za-z0-9_./-]+\.(?:py|md|c|h|cu|cuh|txt))`", text))
    assert names
    missing = []
    for n in names:
        cands = [os.path.join(ROOT, n), os.path.join(ROOT, "paper_1110_1379_gb300", n)]
        if not any(os.path.exists(c) for c in cands):
            missing.append(n)
    assert not missing, missing


def test_oracle_pin_maps_name_existing_tests():
    """The pin maps in the oracle files' headers name pin tests that exist."""
    tests = ""
    for path in glob.glob(os.path.join(ROOT, "tests", "test_*.py")):
        tests += open(path).read()
    defined = set(re.findall(r"^def (test_\w+)", tests, flags=re.M))
    for name in ("fr_oracle.c", "oracle.py", "masked.py", "symmetron.py", "poisson.py",
                 "particles.py"):
        head = open(os.path.join(ROOT, "oracle", name)).read()[:6000]
        named = set(re.findall(r"\b(test_\w+)(?!\.py)\b", head))
        named = {n for n in named if not n.endswith("_") and not n.endswith("_pins")}
        assert named, name
        missing = sorted(n for n in named if n not in defined
                         and not any(d.startswith(n) for d in defined))
        assert not missing, (name, missing)
