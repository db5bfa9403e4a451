"""Host side of the multi-GPU path (one process per GPU, replicas / independent
batch units), run as world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest

from paper_1110_1379_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_greedy_partition_properties():
    w = [s["n"] ** 3 for s in synth.batch_specs(96, 5000)]
    for parts in (1, 2, 3, 4, 8):
        p = shard.greedy_partition(w, parts)
        flat = sorted(i for q in p for i in q)
        assert flat == list(range(len(w)))  # every unit exactly once
        loads = [sum(w[i] for i in q) for q in p]
        assert max(loads) <= sum(w) / parts + max(w)  # LPT bound
        assert p == shard.greedy_partition(w, parts)  # deterministic on every rank


def test_rank_info_environment(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "2")
    monkeypatch.setenv("LOCAL_RANK", "2")
    assert shard.rank_info() == (2, 4, 2)
    monkeypatch.setenv("RANK", "4")
    with pytest.raises(ValueError):
        shard.rank_info()


def _worker(rank, world, port, outdir):
    import json

    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, wsz, local = shard.rank_info()
    specs = synth.batch_specs(96, 5000)
    mine = shard.greedy_partition([s["n"] ** 3 for s in specs], wsz)[r]
    gathered = [None] * wsz
    dist.all_gather_object(gathered, mine)
    # the job's time is the slowest rank's
    tmax = shard.max_over_ranks(1.5 + r)
    with open(os.path.join(outdir, f"rank{r}.json"), "w") as fh:
        json.dump({"rank": r, "world": wsz, "local": local, "mine": mine,
                   "gathered": gathered, "tmax": tmax}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing(tmp_path):
    import json

    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert res[0]["gathered"] == res[1]["gathered"]
    assert res[0]["gathered"][1] == res[1]["mine"]
    allidx = sorted(res[0]["mine"] + res[1]["mine"])
    assert allidx == list(range(96)) and not set(res[0]["mine"]) & set(res[1]["mine"])
    assert all(x["tmax"] == 2.5 for x in res)
