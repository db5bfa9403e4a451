"""Host-side helpers of bench.py (no GPU): the --options parser, the
untimed option search and the clock sampler."""
import bench


def test_parse_options_types():
    o = bench.parse_options("pre=3, post=1,relax=1.25,prec=mixed,tiling=-1,fmg=1")
    assert o == {"pre": 3, "post": 1, "relax": 1.25, "prec": "mixed", "tiling": -1, "fmg": 1}
    assert isinstance(o["pre"], int) and isinstance(o["relax"], float)
    assert bench.parse_options("") == {}


def test_pick_options_takes_the_fastest_converging_candidate(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    clock = [0.0]
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])
    cost = {(2, 2, 1.0, "fp64"): 3.0, (2, 2, 1.0, "mixed"): 1.0, (1, 1, 1.15, "mixed"): 0.5}

    def run(pre, post, relax, prec):
        if (pre, post, relax, prec) == (1, 1, 1.15, "mixed"):
            raise AssertionError("no convergence")  # skipped
        clock[0] += cost[(pre, post, relax, prec)]

    cands = [dict(pre=2, post=2, relax=1.0, prec=p) for p in ("fp64", "mixed")]
    cands.append(dict(pre=1, post=1, relax=1.15, prec="mixed"))
    best, times = bench.pick_options(run, cands)
    assert best == dict(pre=2, post=2, relax=1.0, prec="mixed")
    assert times == {"V(2,2) w=1.0 fp64": 3.0, "V(2,2) w=1.0 mixed": 1.0}


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    """ClockSampler against a stand-in nvidia-smi on PATH that prints four
    sample lines: the first (taken before the timed region) is dropped, the
    median SM clock and the active throttle reasons of the rest are reported."""
    fake = tmp_path / "nvidia-smi"
    lines = ["0, 1500, 2070, 600.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{l}'\n" for l in lines) + "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{bench.os.environ.get('PATH', '')}")
    s = bench.ClockSampler(0)
    s.start()
    bench.time.sleep(0.2)
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_reports_the_headline_config(monkeypatch, capsys):
    """Both arms print the same metric, unit and config, so the two lines can
    be compared; the reference arm's bounded sample is named in cpu_baseline.
    The oracle solve is replaced by a stand-in (this checks the line, not the
    oracle)."""
    import json
    import types
    import bench
    from oracle import oracle as O
    calls = []

    def fake_solve(rho, **kw):
        calls.append(rho.shape)
        return types.SimpleNamespace(converged=True)

    monkeypatch.setattr(O, "solve", fake_solve)
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(gpus=2, steps=2, warmup=1, n=bench.N)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "cells/s" and line["higher_is_better"] is True
    assert line["config"] == bench.headline_config(bench.N, 2)
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert calls == [(bench.SAMPLE_N,) * 3] * 3
