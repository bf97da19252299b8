"""Host-side multi-rank logic on the CPU: LPT assignment, and world-size-2 gloo runs
of the timing aggregation and record gathering that bench.py and batched runs use."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2107_02737_gb300 import inputs, shard


def test_lpt_assignment_is_complete_disjoint_and_balanced():
    sizes = inputs.batch_sizes(64, inputs.rng_for(2, 10_000))
    parts = shard.lpt_assign([shard.solve_cost(n) for n in sizes], 4)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))
    loads = [sum(shard.solve_cost(sizes[i]) for i in p) for p in parts]
    # LPT bound: max load <= total/world + largest item
    assert max(loads) <= sum(loads) / 4 + max(shard.solve_cost(n) for n in sizes)
    # by hand: 0->r0, 1->r1, 2->r0 (tie), 3->r1, 4->r0 (tie)
    assert shard.lpt_assign([3, 3, 2, 2, 2], 2) == [[0, 2, 4], [1, 3]]


def test_lpt_single_rank_and_more_ranks_than_items():
    assert shard.lpt_assign([5.0, 1.0], 1) == [[0, 1]]
    assert shard.lpt_assign([5.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.lpt_assign([1.0], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [128, 2048, 256, 1024, 512, 640]
        mine = shard.shard_instances(sizes, rank, world)
        ms, val = shard.aggregate_step_time(10.0 + rank, 100.0 * (rank + 1))
        recs = shard.gather_records({i: {"n": sizes[i], "rank": rank} for i in mine}, world)
        out[rank] = (mine, ms, val, sorted(recs), {i: r["rank"] for i, r in recs.items()})
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_two():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    mine0, ms0, val0, keys0, owner0 = res[0]
    mine1, ms1, val1, keys1, owner1 = res[1]
    assert sorted(mine0 + mine1) == list(range(6)) and not set(mine0) & set(mine1)
    assert ms0 == ms1 == 11.0
    assert val0 == val1 == 300.0
    assert keys0 == keys1 == list(range(6))
    assert owner0 == owner1 and all(owner0[i] == 0 for i in mine0)


def _batch_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = inputs.batch_sizes(64, inputs.rng_for(2, 10_000))

        def solve(idx):
            # stand-in for one grouped launch: L = 30 layers each, time proportional to the work
            recs = {i: {"n": sizes[i], "layers": 30, "rank": rank} for i in idx}
            work = sum(30 * 2.0 * sizes[i] ** 3 for i in idx)
            return recs, work / 1e12, work

        merged, mine, ms, work = shard.run_sharded_batch(sizes, solve, rank, world)
        out[rank] = (sorted(mine), ms, work, {i: (r["n"], r["rank"]) for i, r in merged.items()})
    finally:
        dist.destroy_process_group()


def test_sharded_batch_runner_gloo_world_size_two():
    """The 64-instance batch across two ranks: a disjoint LPT split, every record on
    both ranks, the slowest rank's time and the sum of the work."""
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    sizes = inputs.batch_sizes(64, inputs.rng_for(2, 10_000))
    (m0, ms0, w0, rec0), (m1, ms1, w1, rec1) = res[0], res[1]
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    total = sum(30 * 2.0 * n ** 3 for n in sizes)
    assert w0 == w1 == pytest.approx(total)
    loads = [sum(30 * 2.0 * sizes[i] ** 3 for i in m) / 1e12 for m in (m0, m1)]
    assert ms0 == ms1 == pytest.approx(max(loads))
    assert rec0 == rec1 and sorted(rec0) == list(range(64))
    assert all(rec0[i] == (sizes[i], 0) for i in m0) and all(rec0[i] == (sizes[i], 1) for i in m1)
    # LPT keeps the two ranks' shares within one largest instance of each other
    assert abs(loads[0] - loads[1]) <= 30 * 2.0 * max(sizes) ** 3 / 1e12


def test_sharded_batch_runner_rejects_missing_records():
    with pytest.raises(ValueError):
        shard.run_sharded_batch([128, 256], lambda idx: ({}, 1.0, 1.0), 0, 1)
