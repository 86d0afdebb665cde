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
