"""Event detection on the device (Section 4.1 pre-processing) against the
event oracle, and the raw-signal path (detection, then sDTW) against the
oracle's events run through the oracle's sDTW.

Events and their offsets are compared bit for bit: boundaries come from
exact integer statistics on both sides, and each event mean is one
correctly rounded division in double, rounded once to float. The decisions
of the raw-signal path equal those of the event path on the same events.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import compare_fp32, compare_int16

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
def sars_ref():
    g, m, k, _ = synth.signal_workload("sars_signal_32x250", nreads=1)
    return g, m, k, oracle.ref_levels(g, m, k)


def csr(parts):
    off = np.zeros(len(parts) + 1, dtype=np.uint32)
    off[1:] = np.cumsum([p.shape[0] for p in parts])
    smp = np.concatenate(parts).astype(np.int16) if parts else np.zeros(0, np.int16)
    return smp, off


def edge_reads():
    """Ragged and degenerate reads: empty, 1-3 samples, flat, noiseless steps,
    pure noise, a read at the length limit, short ones with few events."""
    rng = np.random.default_rng(51)
    parts = [np.zeros(0, np.int16), np.array([7], np.int16), np.array([1, 9], np.int16),
             np.array([5, 5, 5], np.int16), np.full(500, 612, np.int16)]
    lengths = rng.integers(13, 40, 80)
    levels = np.cumsum(rng.choice([-1, 1], 80) * rng.integers(1, 300, 80)) + 2000
    parts.append(np.repeat(levels, lengths).astype(np.int16))
    parts.append(synth.to_adc(rng.normal(90, 2.5, 3001)))
    # equal statistics at neighbouring positions (the tie of the event oracle's
    # pins), repeated: exercises the exact comparison behind the float one
    parts.append(np.tile(np.array([100] * 20 + [150] + [200] * 20, np.int16), 30))
    _, _, _, R = synth.signal_workload("sars_signal_32x250", nreads=4, seed=57)
    parts += [R.read(r) for r in range(R.nreads)]
    long = synth.signal_workload("sars_signal_32x250", nreads=1, seed=58)[3].read(0)
    parts.append(np.resize(long, synth.SAMPLE_RATE_HZ * 4))  # 16,000 samples
    parts.append(np.resize(long, 16384))                      # the limit
    for n in (1023, 1024, 1025, 2047, 2049):                   # around the kernel's tile
        parts.append(synth.to_adc(rng.normal(90, 2.5, n) + np.repeat(rng.normal(0, 12, n // 8 + 1), 8)[:n]))
    return parts


@pytest.mark.parametrize("params", [{}, {"trim_events": 0, "max_events": 512},
                                    {"window_short": 2, "window_long": 16, "threshold_short_centi": 90,
                                     "threshold_long_centi": 1500, "trim_events": 3, "max_events": 40},
                                    {"window_short": 5, "window_long": 5, "trim_events": 400, "max_events": 7}])
def test_detect_events_bit_exact(haru, params):
    smp, off = csr(edge_reads())
    with haru.Context() as ctx:
        p = ctx.event_params(**params)
        ev, eoff = ctx.detect_events(smp, off, p)
    kw = {"w1": p.window_short, "w2": p.window_long, "tau1_centi": p.threshold_short_centi,
          "tau2_centi": p.threshold_long_centi, "trim": p.trim_events, "max_events": p.max_events}
    oev, ooff = oracle.signal_events(smp, off, **kw)
    np.testing.assert_array_equal(eoff, ooff)
    np.testing.assert_array_equal(ev, oev)
    assert eoff[-1] > 0


def test_detect_events_device_pointers(haru):
    smp, off = csr(edge_reads())
    dev = torch.device("cuda:0")
    with haru.Context() as ctx:
        p = ctx.event_params()
        hev, hoff = ctx.detect_events(smp, off, p)
        d_smp = torch.from_numpy(smp).to(dev)
        d_off = torch.from_numpy(off.astype(np.int32)).to(dev)
        d_ev = torch.full((len(off) * p.max_events,), -1.0, dtype=torch.float32, device=dev)
        d_eoff = torch.zeros(len(off), dtype=torch.int32, device=dev)
        ctx.detect_events_device(d_smp, d_off, d_ev, d_eoff, p, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        eoff = d_eoff.cpu().numpy().astype(np.uint32)
        np.testing.assert_array_equal(eoff, hoff)
        np.testing.assert_array_equal(d_ev.cpu().numpy()[:int(eoff[-1])], hev)


def test_signal_batch_equals_event_path(haru, sars_ref):
    """Raw samples -> decisions equals the oracle's events through the event
    path (haru_sdtw_batch with HARU_RAW) and through the oracle's sDTW."""
    g, m, k, ref = sars_ref
    _, _, _, R = synth.signal_workload("sars_signal_32x250")
    oev, ooff = oracle.signal_events(R.samples, R.offsets)
    with haru.Context() as ctx:
        ctx.ref_build(g, m, k, scale_log2=6)
        for prec in (haru.HARU_INT16, haru.HARU_FP32, haru.HARU_INT16_ACC32):
            c, j, nev = ctx.sdtw_batch_signal(prec, R.samples, R.offsets)
            np.testing.assert_array_equal(nev, np.diff(ooff.astype(np.int64)))
            ce, je = ctx.sdtw_batch(prec, oev, ooff)
            np.testing.assert_array_equal(c, ce)
            np.testing.assert_array_equal(j, je)
            if prec == haru.HARU_FP32:
                compare_fp32(c, j, ref, oev, ooff)
            else:
                compare_int16(c, j, ref, oev, ooff, prec=oracle.PREC_I16 if prec == haru.HARU_INT16 else
                              oracle.PREC_I32)
    # on-target reads end where the level behind their last query event sits
    on = R.on_target
    truth = np.full(R.nreads, -1, dtype=np.int64)
    for r in np.flatnonzero(on):
        b = oracle.event_boundaries(R.read(r))
        last_start = b[50 + 250 - 2]  # event 299 starts at boundary 299
        truth[r] = R.level_pos[R.offsets[r] + last_start]
    assert (np.abs(j[on] - truth[on]) <= 8).mean() >= 0.9


def test_signal_uneven_8192_every_read(haru):
    """The benchmark-sized raw-signal batch (8,192 reads) on device pointers:
    every read's events and the int16 alignment of every read against the
    oracle."""
    g, m, k, R = synth.signal_workload("sars_signal_uneven_8192")
    ref = oracle.ref_levels(g, m, k)
    oev, ooff = oracle.signal_events(R.samples, R.offsets)
    dev = torch.device("cuda:0")
    with haru.Context() as ctx:
        ctx.ref_build(g, m, k, scale_log2=6)
        d_smp = torch.from_numpy(R.samples).to(dev)
        d_off = torch.from_numpy(R.offsets.astype(np.int32)).to(dev)
        cost = torch.empty(R.nreads, dtype=torch.float32, device=dev)
        col = torch.empty(R.nreads, dtype=torch.int64, device=dev)
        nev = torch.empty(R.nreads, dtype=torch.int32, device=dev)
        s = torch.cuda.current_stream().cuda_stream
        ctx.sdtw_batch_signal_device(haru.HARU_INT16, d_smp, d_off, cost, col, nev, stream=s)
        p = ctx.event_params()
        d_ev = torch.empty(R.nreads * p.max_events, dtype=torch.float32, device=dev)
        d_eoff = torch.empty(R.nreads + 1, dtype=torch.int32, device=dev)
        ctx.detect_events_device(d_smp, d_off, d_ev, d_eoff, p, stream=s)
        torch.cuda.synchronize()
        eoff = d_eoff.cpu().numpy().astype(np.uint32)
        np.testing.assert_array_equal(eoff, ooff)
        np.testing.assert_array_equal(d_ev.cpu().numpy()[:int(eoff[-1])], oev)
        np.testing.assert_array_equal(nev.cpu().numpy(), np.diff(ooff.astype(np.int64)))
        compare_int16(cost.cpu().numpy(), col.cpu().numpy(), ref, oev, ooff)


def test_signal_errors(haru, sars_ref):
    g, m, k, _ = sars_ref
    _, _, _, R = synth.signal_workload("sars_signal_32x250", nreads=3)
    cost = np.zeros(3, np.float32)
    col = np.zeros(3, np.int64)
    with haru.Context() as ctx:
        assert ctx.sdtw_batch_signal_raw(haru.HARU_INT16, R.samples, R.offsets, 3, None, cost, col, None) == \
            haru.HARU_ENOREF
        ctx.ref_build(g, m, k, scale_log2=6)
        too_long, off = csr([np.zeros(haru.HARU_MAX_READ_SAMPLES + 1, np.int16)])
        assert ctx.sdtw_batch_signal_raw(haru.HARU_INT16, too_long, off, 1, None, cost, col, None) == \
            haru.HARU_EINVAL
        bad = ctx.event_params(window_short=1)
        assert ctx.sdtw_batch_signal_raw(haru.HARU_INT16, R.samples, R.offsets, 3, bad, cost, col, None) == \
            haru.HARU_EINVAL
        # a read too short to leave a query after the adaptor trim
        short, off = csr([R.read(0), R.read(1)[:200], R.read(2)])
        assert ctx.sdtw_batch_signal_raw(haru.HARU_INT16, short, off, 3, None, cost, col, None) == \
            haru.HARU_EINVAL
        # the context still works
        c, j, nev = ctx.sdtw_batch_signal(haru.HARU_INT16, R.samples, R.offsets)
        assert (nev == 250).all() and np.isfinite(c).all()
