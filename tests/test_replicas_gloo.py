"""The N > 1 path on CPU: world-size-2 gloo process groups run the replica
sharding and the timing reductions bench.py uses (no GPU, no NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_22684_gb300.replicas import shard_units, unit_cost
from workloads import batch_jobs


def test_shard_is_a_partition_and_balanced():
    jobs = batch_jobs(4000, count=64, lmin=10, lmax=20)
    log_ns = [j.log_n for j in jobs]
    for world in (1, 2, 3, 4, 8):
        parts = shard_units(log_ns, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(jobs)))
        loads = [sum(unit_cost(log_ns[i]) for i in p) for p in parts]
        biggest = max(unit_cost(L) for L in log_ns)
        assert max(loads) - min(loads) <= biggest   # greedy bound


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2509_22684_gb300.replicas import max_over_ranks, my_units, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = batch_jobs(4000, count=64, lmin=10, lmax=20)
    mine = my_units([j.log_n for j in jobs], rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    elems = sum(1 << jobs[i].log_n for i in mine)
    total = sum_over_ranks(float(elems))
    slowest = max_over_ranks(float(rank + 1) * 1.5)
    dist.barrier()
    out[rank] = (gathered, total, slowest)
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_reductions():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    jobs = batch_jobs(4000, count=64, lmin=10, lmax=20)
    g0, total0, slow0 = out[0]
    g1, total1, slow1 = out[1]
    assert g0 == g1                                   # every rank sees the same assignment
    assert sorted(g0[0] + g0[1]) == list(range(64))   # disjoint cover
    assert total0 == total1 == float(sum(1 << j.log_n for j in jobs))
    assert slow0 == slow1 == 3.0


def test_shard_properties_over_generated_inputs():
    """For generated unit lists and world sizes: the shards partition the
    units, every rank computes the same assignment, and the load imbalance is
    at most the largest unit (the greedy largest-first bound)."""
    hypothesis = pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=60, deadline=None)
    @given(log_ns=st.lists(st.integers(1, 24), min_size=0, max_size=80), world=st.integers(1, 9))
    def check(log_ns, world):
        parts = shard_units(log_ns, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(len(log_ns)))
        assert parts == shard_units(list(log_ns), world)      # deterministic
        if log_ns:
            loads = [sum(unit_cost(log_ns[i]) for i in p) for p in parts]
            assert max(loads) - min(loads) <= max(unit_cost(L) for L in log_ns)

    check()
