"""The N > 1 launch logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

Checks what the GPU runs rely on when bench.py runs under torchrun: the rank
and world size from the environment, the barrier, the max-over-ranks time and
the summed work of the whole-job throughput, the partition of the ensemble
members over the ranks, and that only rank 0 runs the reference arm.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank = bench.dist_info()
        bench.barrier(ws)
        t_max = bench.max_over_ranks(ws, 1.5 + rank)
        total = bench.sum_over_ranks(ws, 10.0 * (rank + 1))
        # rank r processed 100 (r + 1) units in 1 + r seconds
        value, t_job = bench.job_throughput(ws, 100 * (rank + 1), 1.0 + rank)
        members = bench.shard(list(range(64)), ws, rank)
        rc = bench.run_reference(None) if rank != 0 else None   # rank > 0: returns before any work
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(ws=got_ws, rank=got_rank, t_max=t_max, total=total, value=value, t_job=t_job,
                       members=members, rc=rc), f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r, d in enumerate(res):
        assert (d["ws"], d["rank"]) == (ws, r)
        assert d["t_max"] == 2.5                       # max of 1.5 and 2.5
        assert d["total"] == 30.0                      # 10 + 20
        assert d["t_job"] == 2.0                       # the slower rank's time
        assert d["value"] == pytest.approx(300.0 / 2.0)  # all units over the slowest rank
    assert res[1]["rc"] == 0
    shares = [set(d["members"]) for d in res]
    assert shares[0].isdisjoint(shares[1])
    assert shares[0] | shares[1] == set(range(64))
    assert abs(len(shares[0]) - len(shares[1])) <= 1
