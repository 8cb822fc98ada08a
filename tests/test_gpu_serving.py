"""The serving loop: continuous batching of Read Until decisions.

Reads arrive as chunks from a simulated flow cell; every decision must equal
the same read's prefix aligned alone in a batch of one (same kernels, same
arithmetic), whatever batch it shared on the GPU, and every decided read is
also checked against the oracle.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def haru():
    import paper_2211_07340_gb300 as h
    h.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return h


@pytest.fixture(scope="module")
def ref():
    return oracle.ref_levels(synth.genome(synth.SARS_COV_2_BASES, synth.SEED_GENOME_ON), synth.pore_model(6), 6)


def run_schedule(ctx, chunks, speed, signal=False):
    results = []
    done = threading.Event()

    def poller():
        while not done.is_set():
            results.extend(ctx.stream_poll(4096, 2000))

    th = threading.Thread(target=poller)
    th.start()

    def submit(c, t):
        if signal:
            return ctx.stream_submit_signal(c.read_id, c.channel, c.events, t, c.last)
        return ctx.stream_submit(c.read_id, c.channel, c.events, t, c.last)

    synth.replay(chunks, submit, speed=speed)
    n_reads = len({c.read_id for c in chunks})
    deadline = time.monotonic() + 30
    while len(results) < n_reads and time.monotonic() < deadline:
        time.sleep(0.01)
    done.set()
    th.join()
    results.extend(ctx.stream_poll(4096, 0))
    return results


@pytest.mark.parametrize("prec,budget", [(1, 64 << 20), (0, 64 << 20), (1, 8 * 1024)])
def test_decisions_match_alone(haru, ref, prec, budget):
    chunks, q = synth.flowcell_schedule(48, 4.0, seed=105)
    with haru.Context(serve_precision=prec, serve_budget_bytes=budget, threshold=60.0) as ctx:
        ctx.ref_load(ref)
        res = run_schedule(ctx, chunks, speed=4.0)
        stats = ctx.stream_stats()
        assert len(res) == q.nq, (len(res), q.nq, stats)
        by_id = {r.read_id: r for r in res}
        assert sorted(by_id) == list(range(q.nq))
        assert all(r.status == 0 for r in res)
        cost, col = ctx.sdtw_batch(prec, q.events, q.offsets)  # one batch, for reference below
        for i in range(q.nq):
            alone_c, alone_j = ctx.sdtw_batch(prec, q.query(i), np.array([0, 250], np.uint32))
            r = by_id[i]
            assert r.cost == alone_c[0] and r.end_col == alone_j[0], i
            assert r.cost == cost[i] and r.end_col == col[i]
            assert r.decision == int(r.cost <= (np.floor(60.0 * 64) / 64 if prec == 1 else 60.0))
            assert r.t_done_ns >= r.t_arrival_ns
    if budget < 64 << 20:
        assert stats["slots"] == 8 and stats["reads_submitted"] == q.nq
    idx = np.arange(q.nq)  # every decided read
    sub = q.subset(idx)
    o = oracle.batch(oracle.PREC_I16 if prec == 1 else oracle.PREC_F32, ref, sub.events, sub.offsets)
    np.testing.assert_array_equal([by_id[i].end_col for i in idx], o.col)
    np.testing.assert_array_equal(np.array([by_id[i].cost for i in idx], np.float64),
                                  o.cost if prec == 1 else o.cost.astype(np.float32).astype(np.float64))


def test_flat_and_short_reads_are_rejected_alone(haru, ref):
    with haru.Context() as ctx:
        ctx.ref_load(ref)
        t = time.monotonic_ns()
        assert ctx.stream_submit(1, 0, np.full(250, 80.0, np.float32), t, True) == 0
        assert ctx.stream_submit(2, 1, np.array([80.0], np.float32), t, True) == 0
        good = synth.flowcell_schedule(1, 2.0, seed=7)[1].query(0)
        assert ctx.stream_submit(3, 2, good, t, True) == 0
        got = {}
        deadline = time.monotonic() + 10
        while len(got) < 3 and time.monotonic() < deadline:
            for r in ctx.stream_poll(16, 1000):
                got[r.read_id] = r
        assert got[1].status == haru.HARU_EINVAL and got[1].decision == 0
        assert got[2].status == haru.HARU_EINVAL
        assert got[3].status == 0
        assert ctx.stream_poll(16, 1000) == []  # nothing pending: times out empty
        # the serving loop keeps the reference it started with: replacing it
        # is refused on the host, and serving goes on with the old one
        for replace in (lambda: ctx.ref_load(ref[:1000]),
                        lambda: ctx.ref_build(np.zeros(100, np.uint8), synth.pore_model(6), 6)):
            with pytest.raises(haru.HaruError) as err:
                replace()
            assert err.value.code == haru.HARU_EBUSY
        assert ctx.ref_length == ref.shape[0]
        assert ctx.stream_submit(4, 3, good, time.monotonic_ns(), True) == 0
        again = ctx.stream_poll(16, 10 ** 7)
        assert [r.read_id for r in again] == [4]
        assert again[0].cost == got[3].cost and again[0].end_col == got[3].end_col


def test_oversized_chunk_is_cut_to_the_prefix(haru, ref):
    """A chunk far larger than the staging budget (a whole read's events at
    once, here with 8 slots) is accepted, and only its first serve_prefix
    events are used: the decision equals that prefix aligned alone."""
    q = synth.flowcell_schedule(1, 2.0, seed=7)[1].query(0)
    chunk = np.concatenate([q, synth.random_signal(70_000, seed=13)]).astype(np.float32)
    # (a batch limit far above the 8 slots is cut to them: the loop does not
    # reserve batch buffers for 10^8 requests)
    with haru.Context(serve_budget_bytes=8 * 1024, serve_max_batch=10 ** 8) as ctx:
        ctx.ref_load(ref)
        assert ctx.stream_submit(1, 0, chunk, time.monotonic_ns(), True) == 0
        got = ctx.stream_poll(16, 10 ** 7)
        assert [r.read_id for r in got] == [1]
        assert got[0].status == 0 and got[0].events == 250
        c, j = ctx.sdtw_batch(haru.HARU_INT16, q[:250], np.array([0, 250], np.uint32))
        assert got[0].cost == c[0] and got[0].end_col == j[0]


def test_stage_counters_and_idle_sleeping_worker(haru, ref):
    """With serve_spin_us < 0 the worker sleeps between turns; decisions
    still come back, and the per-stage counters account for them."""
    q = synth.flowcell_schedule(4, 3.0, seed=9)[1]
    with haru.Context(serve_spin_us=-1) as ctx:
        ctx.ref_load(ref)
        t = time.monotonic_ns()
        for i in range(min(q.nq, 6)):
            assert ctx.stream_submit(100 + i, i, q.query(i), t, True) == 0
        got = {}
        deadline = time.monotonic() + 10
        while len(got) < min(q.nq, 6) and time.monotonic() < deadline:
            for r in ctx.stream_poll(16, 1000):
                got[r.read_id] = r
        st = ctx.stream_stats()
    assert len(got) == min(q.nq, 6)
    assert all(r.t_arrival_ns <= r.t_received_ns <= r.t_done_ns for r in got.values())
    assert st["reads_decided"] == len(got) and st["batches"] >= 1
    assert st["max_gpu_ns"] > 0 and st["max_turn_gap_ns"] > 0
    # (read while the worker keeps turning, so only bounds that a later turn
    # cannot break): the slowest turn started inside the loop's run
    assert 0 <= st["worst_turn_at_ns"] < 60 * 10 ** 9
    assert st["max_upload_host_ns"] > 0 and st["max_upload_calls_ns"] > 0
    assert st["max_detect_calls_ns"] == 0  # event chunks: no detection launches


@pytest.mark.parametrize("prec,budget", [(1, 64 << 20), (0, 64 << 20), (1, 12 * 34 * 1024)])
def test_signal_decisions_match_batch(haru, ref, prec, budget):
    """A flow cell that delivers raw samples: every decision equals the
    raw-signal batch path on the read's whole signal (detection's final
    events do not depend on how the signal was chunked) and the oracle's
    events through the oracle's sDTW; a small budget (12 slots) makes reads
    wait for admission."""
    chunks, R = synth.flowcell_signal_schedule(48, 4.0, seed=205)
    with haru.Context(serve_precision=prec, serve_budget_bytes=budget, threshold=60.0) as ctx:
        ctx.ref_load(ref)
        res = run_schedule(ctx, chunks, speed=4.0, signal=True)
        stats = ctx.stream_stats()
        assert len(res) == R.nreads, (len(res), R.nreads, stats)
        by_id = {r.read_id: r for r in res}
        assert sorted(by_id) == list(range(R.nreads))
        assert all(r.status == 0 for r in res)
        cost, col, nev = ctx.sdtw_batch_signal(prec, R.samples, R.offsets)
        # a context serving samples refuses event chunks
        assert ctx.stream_submit(10 ** 9, 0, np.ones(4, np.float32), 0, True) == haru.HARU_EINVAL
    if budget < 64 << 20:
        assert stats["slots"] == 12
    thr = np.floor(60.0 * 64) / 64 if prec == 1 else 60.0
    for i in range(R.nreads):
        r = by_id[i]
        assert r.cost == cost[i] and r.end_col == col[i] and r.events == nev[i], i
        assert r.decision == int(r.cost <= thr)
        assert r.t_done_ns >= r.t_arrival_ns
    oev, ooff = oracle.signal_events(R.samples, R.offsets)
    np.testing.assert_array_equal(nev, np.diff(ooff.astype(np.int64)))
    o = oracle.batch(oracle.PREC_I16 if prec == 1 else oracle.PREC_F32, ref, oev, ooff)
    np.testing.assert_array_equal(col, o.col)
    np.testing.assert_array_equal(cost.astype(np.float64), o.cost if prec == 1 else
                                  o.cost.astype(np.float32).astype(np.float64))
