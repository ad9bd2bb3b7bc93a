"""The N > 1 host path on CPU: world-size-2 process groups over gloo.

Cases are independent, so the multi-GPU layer is whole-case sharding with a
host-side gather of results and the bench's max/sum timing reduction; these
run here exactly as they do under torchrun on GPUs (gloo instead of NCCL).
"""
import os
import socket

import pytest

from paper_2512_09904_b300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # timing: slowest rank's time, all ranks' units
        ms, units = shard.reduce_timing(10.0 + rank, 1000 * (rank + 1), world)
        # sharded sweep bookkeeping: every case on exactly one rank, results merged on rank 0
        sizes = [500, 40, 300, 300, 20, 900, 60]
        owner = shard.assign_cases(sizes, world)
        local = {i: dict(rank=rank, size=sizes[i]) for i in range(len(sizes)) if owner[i] == rank}
        merged = shard.gather_results(local, rank, world)
        q.put((rank, ms, units, owner, merged))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduce_and_gather():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r = q.get(timeout=120)
        out[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        _, ms, units, owner, merged = out[r]
        assert ms == 11.0 and units == 3000.0
        assert owner == out[0][3]  # same assignment on every rank
    merged = out[0][4]
    assert out[1][4] is None
    assert sorted(merged) == list(range(7))
    for i, v in merged.items():
        assert v["rank"] == out[0][3][i]


def test_assign_cases_balances_and_is_deterministic():
    sizes = [500, 40, 300, 300, 20, 900, 60]
    owner = shard.assign_cases(sizes, 2)
    assert owner == shard.assign_cases(sizes, 2)
    load = [sum(s for s, o in zip(sizes, owner) if o == r) for r in range(2)]
    # longest first to the least-loaded rank: 900 | 500 300 300 | 60 40 20
    assert load == [1020, 1100]
    # list-scheduling bound: no rank exceeds the mean load by more than one case
    assert max(load) <= sum(sizes) / 2 + max(sizes)
    assert shard.assign_cases(sizes, 1) == [0] * 7
    with pytest.raises(ValueError):
        shard.assign_cases(sizes, 0)
