"""Parity of the CUDA path (through the C ABI) with the oracle.

int16: bit-exact cost and end column. FP32: bitwise equal to the FP32
oracle (sub, abs, add and min round identically), within 1e-5 relative of
FP64, same column as FP64 unless the FP64 runner-up ties within 1e-5.
Sizes span several reference tiles and ragged tails; the benchmark-sized
workloads are checked in full in test_gpu_full_size.py.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import compare_fp32, compare_int16, subset

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
def sars():
    w = synth.workload("sars_32x250")
    ref = oracle.ref_levels(w.genome, w.model, w.k)
    return w, ref


def offsets_of(lengths):
    off = np.zeros(len(lengths) + 1, dtype=np.uint32)
    off[1:] = np.cumsum(lengths)
    return off


def test_reference_build_and_normalisation(haru, sars):
    w, ref = sars
    with haru.Context() as ctx:
        ctx.ref_build(w.genome, w.model, 6, scale_log2=6)
        assert ctx.ref_length == 59_796
        z, q = ctx.ref_read()
        np.testing.assert_array_equal(z, oracle.zscore(ref))
        np.testing.assert_array_equal(q, oracle.quantise(oracle.zscore(ref), 6))
        ctx.ref_load(ref, normalize=True, scale_log2=5)
        z2, q2 = ctx.ref_read()
        np.testing.assert_array_equal(z2, z)
        np.testing.assert_array_equal(q2, oracle.quantise(z, 5))


def test_sars_32x250_both_forms(haru, sars):
    w, ref = sars
    qs = w.queries
    with haru.Context() as ctx:
        ctx.ref_load(ref)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, qs.events, qs.offsets)
        compare_int16(c16, j16, ref, qs.events, qs.offsets)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, qs.events, qs.offsets)
        compare_fp32(c32, j32, ref, qs.events, qs.offsets)
    # on-target queries end near where they were planted
    on = qs.on_target
    assert (np.abs(j32[on] - qs.truth_end[on]) <= 8).mean() >= 0.9


@pytest.mark.parametrize("tile,warps,stack", [(2048, 8, 1), (4096, 4, -1), (16384, 2, 1), (4096, 8, -1), (8192, 12, 1)])
def test_ragged_sizes_span_tiles(haru, tile, warps, stack):
    rng = np.random.default_rng(tile + warps)
    N = 9_001  # several tiles plus a ragged tail
    ref = synth.random_signal(N, seed=5)
    lengths = [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 250, 255, 256, 257, 300, 383, 384, 385,
               448, 480, 500, 511, 512] + list(rng.integers(1, 513, size=14))
    off = offsets_of(lengths)
    # queries given as z-values (a 1-event query has no z-score of its own)
    ev = synth.random_signal(int(off[-1]), seed=6, scale=1.0, loc=0.0)
    with haru.Context(tile_cols=tile, warps_per_cta=warps, stack_short=stack) as ctx:
        ctx.ref_load(ref)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off, raw=False)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev, off, raw=False)
    compare_int16(c16, j16, ref, ev, off, normalize_q=False)
    compare_fp32(c32, j32, ref, ev, off, normalize_q=False)
    # and the same lengths as raw currents (z-scored on the device), 2+ events
    lengths = [m for m in lengths if m >= 2]
    off = offsets_of(lengths)
    ev = synth.random_signal(int(off[-1]), seed=7)
    with haru.Context(tile_cols=tile, warps_per_cta=warps, stack_short=stack) as ctx:
        ctx.ref_load(ref)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev, off)
    compare_int16(c16, j16, ref, ev, off)
    compare_fp32(c32, j32, ref, ev, off)


@pytest.mark.parametrize("stack", [-1, 1])
def test_every_query_length_1_to_512(haru, stack):
    """One batch holding a query of every length 1..512 in shuffled order
    (every strip height with every pad-row count; the short ones in stacked
    strips when stacking is forced), on a reference of a few tiles with a
    ragged tail: all four forms against the oracle."""
    N = 6_007
    ref = synth.random_signal(N, seed=21)
    lengths = np.arange(1, haru.HARU_MAX_QUERY + 1)
    np.random.default_rng(22).shuffle(lengths)
    off = offsets_of(lengths)
    ev = synth.random_signal(int(off[-1]), seed=23, scale=1.0, loc=0.0)
    with haru.Context(stack_short=stack) as ctx:
        ctx.ref_load(ref)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off, raw=False)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev, off, raw=False)
        cw, jw = ctx.sdtw_batch(haru.HARU_INT16_ACC32, ev, off, raw=False)
        cs, js, ss = ctx.sdtw_batch_span(haru.HARU_FP32, ev, off, raw=False)
    compare_int16(c16, j16, ref, ev, off, normalize_q=False)
    compare_fp32(c32, j32, ref, ev, off, normalize_q=False)
    compare_int16(cw, jw, ref, ev, off, normalize_q=False, prec=oracle.PREC_I32)
    np.testing.assert_array_equal(cs, c32)
    np.testing.assert_array_equal(js, j32)
    o = oracle.batch(oracle.PREC_F32, ref, ev, off, normalize_q=False, start=True)
    np.testing.assert_array_equal(ss, o.start)


def test_planted_copies_end_at_planted_column(haru):
    N = 5000
    ref = synth.random_signal(N, seed=8, scale=1.0, loc=0.0)  # z-values: within the int16 range at 2^6
    starts = [0, 1, 777, 2500, N - 300]
    lens = [300, 250, 129, 32, 300]
    ev = np.concatenate([ref[s:s + m] for s, m in zip(starts, lens)]).astype(np.float32)
    off = offsets_of(lens)
    with haru.Context() as ctx:
        ctx.ref_load(ref, normalize=False)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev, off, raw=False)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off, raw=False)
    np.testing.assert_array_equal(c32, 0.0)
    np.testing.assert_array_equal(j32, [s + m - 1 for s, m in zip(starts, lens)])
    np.testing.assert_array_equal(c16, 0.0)
    np.testing.assert_array_equal(j16, [s + m - 1 for s, m in zip(starts, lens)])


def test_single_event_and_full_length_queries(haru):
    ref = synth.random_signal(600, seed=9)
    lens = [1, 512, 1, 300, 600 - 88]
    off = offsets_of(lens)
    ev = synth.random_signal(int(off[-1]), seed=10, scale=1.0, loc=0.0)
    with haru.Context() as ctx:
        ctx.ref_load(ref)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev, off, raw=False)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off, raw=False)
    compare_fp32(c32, j32, ref, ev, off, normalize_q=False)
    compare_int16(c16, j16, ref, ev, off, normalize_q=False)
    # M == N: a query as long as the reference
    ref2 = synth.random_signal(300, seed=11)
    ev2 = synth.random_signal(300, seed=12)
    off2 = offsets_of([300])
    with haru.Context() as ctx:
        ctx.ref_load(ref2)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, ev2, off2)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev2, off2)
    compare_fp32(c32, j32, ref2, ev2, off2)
    compare_int16(c16, j16, ref2, ev2, off2)


def test_errors_and_empty(haru, sars):
    w, ref = sars
    ev = synth.random_signal(100, seed=1)
    with haru.Context() as ctx:
        cost = np.zeros(2, np.float32)
        col = np.zeros(2, np.int64)
        assert ctx.sdtw_batch_raw(0, ev, offsets_of([50, 50]), 2, cost, col) == haru.HARU_ENOREF
        ctx.ref_load(ref[:400])
        assert ctx.sdtw_batch_raw(0, ev, offsets_of([50, 50]), 0, cost, col) == haru.HARU_OK
        assert ctx.sdtw_batch_raw(0, ev, np.array([0, 0, 100], np.uint32), 2, cost, col) == haru.HARU_EINVAL
        big = synth.random_signal(600, seed=2)
        assert ctx.sdtw_batch_raw(0, big, offsets_of([600]), 1, cost, col) == haru.HARU_EINVAL  # M > N
        assert ctx.sdtw_batch_raw(7, ev, offsets_of([50, 50]), 2, cost, col) == haru.HARU_EINVAL
        flat = np.full(50, 3.0, np.float32)  # zero spread: z-score undefined
        assert ctx.sdtw_batch_raw(0, flat, offsets_of([50]), 1, cost, col, 0, haru.HARU_RAW) == haru.HARU_EINVAL
        # the context still works after rejected calls
        c, j = ctx.sdtw_batch(haru.HARU_FP32, ev, offsets_of([50, 50]))
        assert np.isfinite(c).all()
        with pytest.raises(haru.HaruError):
            ctx.ref_load(np.full(10, 1.0, np.float32))  # zero spread


def test_device_pointers_match_host_path(haru, sars):
    w, ref = sars
    qs = w.queries
    dev = torch.device("cuda:0")
    ev = torch.from_numpy(qs.events).to(dev)
    off = torch.from_numpy(qs.offsets.astype(np.int32)).to(dev)
    with haru.Context() as ctx:
        ctx.ref_load(ref)
        for prec in (haru.HARU_INT16, haru.HARU_FP32):
            hc, hj = ctx.sdtw_batch(prec, qs.events, qs.offsets)
            dc = torch.empty(qs.nq, dtype=torch.float32, device=dev)
            dj = torch.empty(qs.nq, dtype=torch.int64, device=dev)
            s = torch.cuda.current_stream().cuda_stream
            ctx.sdtw_batch_device(prec, ev, off, dc, dj, stream=s)
            np.testing.assert_array_equal(dc.cpu().numpy(), hc)
            np.testing.assert_array_equal(dj.cpu().numpy(), hj)
            ctx.sdtw_batch_device(prec, ev, off, dc, dj, stream=s, asynchronous=True)
            torch.cuda.synchronize()
            assert ctx.last_status() == haru.HARU_OK
            np.testing.assert_array_equal(dj.cpu().numpy(), hj)


@pytest.mark.parametrize("units", [1, 4096, 100_000])
def test_reference_segments_are_exact(haru, sars, units):
    """Splitting every sweep into speculative reference segments (verified
    and, where needed, recomputed) gives the unsplit results bit for bit."""
    _, ref = sars
    w = synth.workload("sars_uneven_8192", nq=300)
    qs = w.queries
    with haru.Context(units_target=1) as ctx:
        ctx.ref_load(ref)
        base16 = ctx.sdtw_batch(haru.HARU_INT16, qs.events, qs.offsets)
        base32 = ctx.sdtw_batch(haru.HARU_FP32, qs.events, qs.offsets)
        assert ctx.last_stats()["max_segments"] == 1
    with haru.Context(units_target=units) as ctx:
        ctx.ref_load(ref)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, qs.events, qs.offsets)
        st16 = ctx.last_stats()
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, qs.events, qs.offsets)
        st32 = ctx.last_stats()
    np.testing.assert_array_equal(c16, base16[0])
    np.testing.assert_array_equal(j16, base16[1])
    np.testing.assert_array_equal(c32, base32[0])
    np.testing.assert_array_equal(j32, base32[1])
    if units > 1:
        assert st16["max_segments"] > 1 and st32["max_segments"] > 1
    idx = np.arange(0, 300, 37)
    compare_int16(c16, j16, ref, qs.events, qs.offsets, idx=idx)
    compare_fp32(c32, j32, ref, qs.events, qs.offsets, idx=idx)


def test_autotuner_keeps_results(haru, sars):
    _, ref = sars
    qs = synth.workload("sars_uneven_8192", nq=600).queries
    with haru.Context() as ctx:
        ctx.ref_load(ref)
        forms = (haru.HARU_INT16, haru.HARU_FP32, haru.HARU_INT16_ACC32)
        before = [ctx.sdtw_batch(p, qs.events, qs.offsets) for p in forms]
        for i, p in enumerate(forms):
            chosen = ctx.autotune(p, qs.events, qs.offsets)
            assert chosen["warps_per_cta"] in (4, 8, 12) and chosen["tile_cols"] in (2048, 4096, 8192, 16384)
            c, j = ctx.sdtw_batch(p, qs.events, qs.offsets)
            np.testing.assert_array_equal(c, before[i][0])
            np.testing.assert_array_equal(j, before[i][1])


@pytest.mark.parametrize("units", [1, 4096])
def test_int16_saturation_extremes(haru, units):
    """Codes at the clamp limits (|q - r| up to 4094 per cell) and costs
    around CAP: the int16 form saturates exactly like the oracle's
    all-saturating recurrence, with and without reference segments."""
    rng = np.random.default_rng(21)
    N = 7000
    ref = np.where(rng.random(N) < 0.5, rng.choice([-40.0, 40.0], N), rng.uniform(-40.0, 40.0, N))
    lens = np.concatenate([np.full(8, 512), np.full(4, 480), rng.integers(1, 513, 36)])
    parts = []
    for i, m in enumerate(lens):
        s = int(rng.integers(0, N - m + 1))
        if i % 3 == 0:
            parts.append(rng.choice([-40.0, 40.0], m))                    # extremes everywhere
        elif i % 3 == 1:
            parts.append(ref[s:s + m] + rng.normal(0.0, rng.uniform(0.5, 2.0), m))  # cost near CAP
        else:
            parts.append(-ref[s:s + m])                                    # |q - r| = 2 |r|
    ev = np.concatenate(parts).astype(np.float32)
    off = offsets_of(lens)
    with haru.Context(units_target=units) as ctx:
        ctx.ref_load(ref, normalize=False)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, ev, off, raw=False)
    o = compare_int16(c16, j16, ref, ev, off, normalize_ref=False, normalize_q=False)
    capped = o.icost >= oracle.cap()
    assert capped.sum() >= 10 and (~capped).sum() >= 10


@pytest.mark.parametrize("units", [1, 4096])
def test_stacked_strips_are_identical(haru, sars, units):
    """Short queries stacked two to a warp strip (lanes 0-15 and 16-31) give
    the unstacked results bit for bit, for both forms, with and without
    reference segments; a sample matches the oracle."""
    _, ref = sars
    qs = synth.workload("sars_uneven_8192", nq=701).queries
    out, items = {}, {}
    for stack in (-1, 1):
        with haru.Context(stack_short=stack, units_target=units) as ctx:
            ctx.ref_load(ref)
            out[stack] = [ctx.sdtw_batch(haru.HARU_INT16, qs.events, qs.offsets)]
            items[stack] = ctx.last_stats()["items"]
            out[stack].append(ctx.sdtw_batch(haru.HARU_FP32, qs.events, qs.offsets))
            if units > 1:
                assert ctx.last_stats()["max_segments"] > 1
    assert items[1] < items[-1]  # four short queries per stacked int16 item, two per plain one
    for p in range(2):
        np.testing.assert_array_equal(out[1][p][0], out[-1][p][0])
        np.testing.assert_array_equal(out[1][p][1], out[-1][p][1])
    idx = np.flatnonzero(qs.lengths <= 256)[::23]
    compare_int16(out[1][0][0], out[1][0][1], ref, qs.events, qs.offsets, idx=idx)
    compare_fp32(out[1][1][0], out[1][1][1], ref, qs.events, qs.offsets, idx=idx)


@pytest.mark.parametrize("stack,units", [(-1, 1), (1, 1), (1, 4096), (-1, 4096)])
def test_wide_accumulation_form(haru, sars, stack, units):
    """int16 inputs with wide accumulation (Section 4.3's PE): bit-exact to the
    oracle's unsaturated integer DP, equal to the saturating int16 form
    wherever the exact cost is below CAP, identical with and without stacking
    and reference segments."""
    _, ref = sars
    qs = synth.workload("sars_uneven_8192", nq=257).queries
    with haru.Context(stack_short=stack, units_target=units) as ctx:
        ctx.ref_load(ref)
        cw, jw = ctx.sdtw_batch(haru.HARU_INT16_ACC32, qs.events, qs.offsets)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, qs.events, qs.offsets)
    o = compare_int16(cw, jw, ref, qs.events, qs.offsets, prec=oracle.PREC_I32)
    below = o.icost < oracle.cap()
    np.testing.assert_array_equal(c16[below], cw[below])
    np.testing.assert_array_equal(j16[below], jw[below])
    np.testing.assert_array_equal(c16[~below], oracle.cap() / 64.0)


def test_wide_accumulation_above_cap(haru):
    """Costs far above CAP are reported exactly by the wide form: queries at
    +2047 against a reference at -2047 with a short run of zeros cost
    M * 2047 (a vertical path in the first zero column), 34,799 and more."""
    N = 5000
    ref = np.full(N, -40.0)
    ref[2000:2010] = 0.0
    lens = [512, 480, 300, 100, 17]
    ev = np.full(sum(lens), 40.0, dtype=np.float32)
    off = offsets_of(lens)
    with haru.Context() as ctx:
        ctx.ref_load(ref, normalize=False)
        cw, jw = ctx.sdtw_batch(haru.HARU_INT16_ACC32, ev, off, raw=False)
    o = compare_int16(cw, jw, ref, ev, off, normalize_ref=False, normalize_q=False, prec=oracle.PREC_I32)
    np.testing.assert_array_equal(o.icost, np.array(lens) * 2047)
    np.testing.assert_array_equal(jw, 2000)


@pytest.mark.parametrize("stack", [-1, 1])
def test_start_columns(haru, sars, stack):
    """haru_sdtw_batch_span: costs and end columns equal haru_sdtw_batch's;
    start columns equal the oracle's (FP32 and wide accumulation), stacked
    and not, over ragged lengths."""
    _, ref = sars
    qs = synth.workload("sars_uneven_8192", nq=199).queries
    rng = np.random.default_rng(41)
    lengths = [1, 2, 31, 32, 33, 100, 255, 256, 257, 511, 512] + list(rng.integers(1, 513, size=12))
    off = offsets_of(lengths)
    ev = synth.random_signal(int(off[-1]), seed=42, scale=1.0, loc=0.0)
    with haru.Context(stack_short=stack) as ctx:
        ctx.ref_load(ref)
        for prec, oprec in ((haru.HARU_FP32, oracle.PREC_F32), (haru.HARU_INT16_ACC32, oracle.PREC_I32)):
            c, j = ctx.sdtw_batch(prec, qs.events, qs.offsets)
            cs, js, ss = ctx.sdtw_batch_span(prec, qs.events, qs.offsets)
            np.testing.assert_array_equal(cs, c)
            np.testing.assert_array_equal(js, j)
            o = oracle.batch(oprec, ref, qs.events, qs.offsets, start=True)
            np.testing.assert_array_equal(ss, o.start)
            assert ((ss >= 0) & (ss <= js)).all()
            cs, js, ss = ctx.sdtw_batch_span(prec, ev, off, raw=False)
            o = oracle.batch(oprec, ref, ev, off, normalize_q=False, start=True)
            np.testing.assert_array_equal(js, o.col)
            np.testing.assert_array_equal(ss, o.start)
        with pytest.raises(haru.HaruError):
            ctx.sdtw_batch_span(haru.HARU_INT16, qs.events, qs.offsets)


@pytest.mark.parametrize("stack", [-1, 1])
def test_start_columns_across_segments(haru, stack):
    """Start columns stay exact when a sweep is cut into speculative reference
    segments: the only zero-cost path of the first query enters a 10,000-column
    plateau two columns before it and crosses it on one row, so every segment
    boundary inside the plateau fails verification and is recomputed. The same
    batch cut into many segments and not cut at all, with short queries stacked
    two to a warp and not, gives the oracle's costs, end columns and start
    columns."""
    N = 60000
    ref = synth.random_signal(N, seed=44, scale=1.0, loc=0.0)
    c, e = np.float32(0.25), np.float32(-1.5)
    ref[20000:30000] = c
    ref[30000] = e
    a, b = ref[19998], ref[19999]
    rng = np.random.default_rng(45)
    lengths = [4, 1, 33, 250, 511] + list(rng.integers(2, 513, size=11))
    off = offsets_of(lengths)
    ev = synth.random_signal(int(off[-1]), seed=46, scale=1.0, loc=0.0)
    ev[:4] = [a, b, c, e]
    for prec, oprec in ((haru.HARU_FP32, oracle.PREC_F32), (haru.HARU_INT16_ACC32, oracle.PREC_I32)):
        o = oracle.batch(oprec, ref, ev, off, normalize_ref=False, normalize_q=False, start=True)
        if prec == haru.HARU_FP32:
            assert (o.cost[0], o.col[0], o.start[0]) == (0.0, 30000, 19998)
        for units, segmented in ((1, False), (20000, True)):
            with haru.Context(units_target=units, stack_short=stack) as ctx:
                ctx.ref_load(ref, normalize=False)
                cs, js, ss = ctx.sdtw_batch_span(prec, ev, off, raw=False)
                st = ctx.last_stats()
            assert (st["max_segments"] > 1) == segmented
            if segmented:
                assert st["fixups"] > 0
            np.testing.assert_array_equal(cs, o.cost)
            np.testing.assert_array_equal(js, o.col)
            np.testing.assert_array_equal(ss, o.start)


def test_start_columns_of_planted_copies(haru):
    N = 6000
    ref = synth.random_signal(N, seed=43, scale=1.0, loc=0.0)
    starts = [0, 1, 777, 2500, N - 300, 4000]
    lens = [300, 250, 129, 32, 300, 60]
    parts = [ref[s:s + m] for s, m in zip(starts, lens)]
    parts[-1] = np.repeat(parts[-1], 2)  # dwelled: every sample twice
    lens[-1] *= 2
    ev = np.concatenate(parts).astype(np.float32)
    off = offsets_of(lens)
    with haru.Context() as ctx:
        ctx.ref_load(ref, normalize=False)
        c, j, st = ctx.sdtw_batch_span(haru.HARU_FP32, ev, off, raw=False)
    np.testing.assert_array_equal(c, 0.0)
    np.testing.assert_array_equal(st, starts)
    np.testing.assert_array_equal(j, [s + m - 1 for s, m in zip(starts, [300, 250, 129, 32, 300, 60])])
