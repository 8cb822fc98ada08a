"""Host logic of the multi-GPU path on CPU ranks (gloo, world size 2).

Queries are independent, so a batch shards across GPUs with no exchange but
the final gather. Here each rank aligns its shard with the oracle (standing
in for its GPU), the shards cover the batch exactly once, the gathered
results equal the single-process results, and the max-over-ranks timing
reduction behaves as the benchmark uses it.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2211_07340_gb300 as haru
    w = synth.workload("sars_uneven_8192", nq=24)
    ref = oracle.ref_levels(w.genome, w.model, w.k)[:4000]
    q = w.queries
    lo, hi = haru.shard_queries(q.offsets, world, rank)
    sub = q.subset(np.arange(lo, hi))
    r = oracle.batch(oracle.PREC_I16, ref, sub.events, sub.offsets, threads=1)
    # gather variable-length shards: sizes first, then padded payloads
    n = torch.tensor([hi - lo])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    m = int(max(s.item() for s in sizes))
    pay = torch.full((m, 2), -1.0, dtype=torch.float64)
    pay[: hi - lo, 0] = torch.from_numpy(r.cost)
    pay[: hi - lo, 1] = torch.from_numpy(r.col.astype(np.float64))
    parts = [torch.zeros_like(pay) for _ in range(world)]
    dist.all_gather(parts, pay)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)  # per-rank step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        got = torch.cat([p[: int(s.item())] for p, s in zip(parts, sizes)]).numpy()
        out.put((got, float(t.item()), [int(s.item()) for s in sizes]))
    dist.destroy_process_group()


def test_two_ranks_shard_and_gather():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax, sizes = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.workload("sars_uneven_8192", nq=24)
    ref = oracle.ref_levels(w.genome, w.model, w.k)[:4000]
    full = oracle.batch(oracle.PREC_I16, ref, w.queries.events, w.queries.offsets)
    np.testing.assert_array_equal(got[:, 0], full.cost)
    np.testing.assert_array_equal(got[:, 1], full.col)
    assert tmax == 2.0 and sum(sizes) == 24 and min(sizes) > 0


def test_shards_balance_events():
    import paper_2211_07340_gb300 as haru
    q = synth.workload("sars_uneven_8192", nq=1000).queries
    for world in (1, 2, 3, 8):
        cuts = [haru.shard_queries(q.offsets, world, r) for r in range(world)]
        assert cuts[0][0] == 0 and cuts[-1][1] == q.nq
        assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
        ev = [int(q.offsets[h] - q.offsets[l]) for l, h in cuts]
        assert max(ev) - min(ev) <= 2 * 500  # each cut is within one query of even
    assert haru.shard_queries(np.array([0], np.uint32), 4, 2) == (0, 0)
