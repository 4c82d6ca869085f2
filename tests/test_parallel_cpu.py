"""The multi-GPU host logic on CPU: world-size-2 gloo process groups (no GPU needed).

Events are independent, so ranks shard them without a data-path collective; the process group
only carries the barrier and the max-over-ranks timing reduction.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

from paper_1608_06577_gb300.parallel import shard_events
from workload.problem import batch_shapes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_events_covers_and_balances():
    cells = [n * n * nz for n, nz, _ in batch_shapes(64)]
    for world in (1, 2, 3, 4, 8):
        shards = shard_events(cells, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(cells)))  # every event exactly once
        loads = [sum(cells[i] for i in s) for s in shards]
        # largest-first greedy: no rank exceeds the mean by more than one event
        assert max(loads) <= sum(cells) / world + max(cells)
        assert shard_events(cells, world) == shards  # deterministic
    assert shard_events([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard_events(cells, 0)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_1608_06577_gb300 import parallel
    w, r, _ = parallel.init("gloo")
    cells = [n * n * nz for n, nz, _ in batch_shapes(64)]
    mine, total_cells = parallel.rank_share(cells, w, r)  # the selection bench.py --batch makes
    assert mine == shard_events(cells, w)[r] and total_cells == sum(cells)
    if r == 1:  # the events a rank builds are the ones of the full batch with those indices
        from workload.problem import batch_problems
        small = dict(nx_choices=(8, 12), neta_choices=(4, 8), hot_range=(2, 4))
        full = batch_problems(6, **small)
        part = batch_problems(6, events=[4, 1], **small)
        assert [p.name for p in part] == [full[4].name, full[1].name]
        assert all((a.e == b.e).all() for a, b in zip(part, [full[4], full[1]]))
    parallel.barrier(w)
    t = parallel.max_over_ranks(float(10 + r), w)
    total = parallel.sum_over_ranks(float(sum(cells[i] for i in mine)), w)
    gathered = [None] * w
    dist.all_gather_object(gathered, mine)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "max": t, "total": total, "cells": sum(cells), "shards": gathered}, f)
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_reductions(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["world"] == 2
        assert r["max"] == 11.0  # max over ranks of 10 + rank
        assert r["total"] == r["cells"]  # the ranks' shards add up to the whole batch
        assert sorted(i for s in r["shards"] for i in s) == list(range(64))
    assert res[0]["shards"] == res[1]["shards"]


def test_bench_reference_arm_under_torchrun():
    """The launch the driver uses for N > 1, on CPU: rank 0 alone prints the reference line,
    the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
