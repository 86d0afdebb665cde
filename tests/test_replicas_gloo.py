"""The multi-GPU path of bench.py (independent replicas, one stream per
GPU, no collective on the data path): the whole-job aggregation over ranks,
run as two gloo processes on the CPU."""
import json
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    line = {"ms_per_step": 4.0 + rank, "value": 0.0, "n_gpus": 1,
            "config": {"workload": "w", "symbols_per_pol": 1 << 20},
            "e2e": {"ms_per_step": 7.0 - rank, "value": 0.0, "unit": "Gsamples/s",
                    "h2d_bytes_per_step": 100, "d2h_bytes_per_step": 10}}

    def reduce_max(vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.tolist()

    res = bench.combine_replicas(line, world, reduce_max)
    with open(os.path.join(out, f"rank{rank}.json"), "w") as fh:
        json.dump(res, fh)
    dist.destroy_process_group()


def test_replica_aggregation_takes_the_slowest_rank(tmp_path):
    world = 2
    port = _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as fh:
            line = json.load(fh)
        assert line["n_gpus"] == world
        assert line["ms_per_step"] == 5.0                       # max over ranks
        assert line["e2e"]["ms_per_step"] == 7.0
        assert line["value"] == pytest.approx(world * 4 * (1 << 20) / 5e-3 / 1e9, rel=1e-3)
        assert line["e2e"]["h2d_bytes_per_step"] == 200
        assert line["config"]["parallelism"] == "replicas x2"


def test_streams_shard_greedily_by_cost():
    costs = [5.0, 1.0, 4.0, 3.0, 3.0, 2.0, 2.0]
    sh = bench.shard_streams(costs, 3)
    assert sorted(i for s in sh for i in s) == list(range(len(costs)))  # every stream exactly once
    loads = [sum(costs[i] for i in s) for s in sh]
    assert max(loads) - min(loads) <= max(costs)
    # costliest first to the least-loaded rank: 5 -> r0, 4 -> r1, 3 -> r2, 3 -> r2 (6),
    # 2 -> r1 (6), 2 -> r0 (7), 1 -> r1 (the lower of the two ranks at 6)
    assert sh == [[0, 6], [1, 2, 5], [3, 4]]
    assert bench.shard_streams([1.0] * 64, 2) == [list(range(0, 64, 2)), list(range(1, 64, 2))]
    assert bench.shard_streams([1.0] * 3, 4)[3] == []


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = {"form": "batch_default_fft", "wall_ms": 10.0 + rank, "ber_max": 1e-3 * (rank + 1),
            "samples": 1000000 * (rank + 1), "streams": 32, "synced_streams": 32 - rank, "cycle_slips": rank,
            "launches": 400 + rank, "symbols_per_pol_per_stream": 1 << 19}

    def op(o):
        def f(vals):
            t = torch.tensor(vals, dtype=torch.float64)
            dist.all_reduce(t, op=o)
            return t.tolist()
        return f

    res = bench.combine_shards(part, world, op(dist.ReduceOp.MAX), op(dist.ReduceOp.SUM))
    with open(os.path.join(out, f"shard{rank}.json"), "w") as fh:
        json.dump(res, fh)
    dist.destroy_process_group()


def test_sharded_streams_aggregate_on_the_host(tmp_path):
    """Stream-sharded multi-GPU form: the slowest rank's wall time, every
    rank's samples and streams, the worst BER."""
    world = 2
    port = _free_port()
    mp.spawn(_shard_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"shard{r}.json") as fh:
            line = json.load(fh)
        assert line["n_gpus"] == world and line["scaling"] == "strong"
        assert line["wall_ms"] == 11.0
        assert line["value"] == pytest.approx(3e6 / 11e-3 / 1e9, rel=1e-3)
        assert line["config"]["streams"] == 64 and line["synced_streams"] == 63
        assert line["ber_max"] == pytest.approx(2e-3) and line["cycle_slips"] == 1 and line["launches"] == 801
