"""Host-side helpers of bench.py (no GPU): the --options parser and the
untimed option search."""
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
