"""haru_sdtw_batch_noalloc: the batch entry point that allocates nothing.

It serves callers that cannot let the library allocate device memory (a
fixed memory budget reserved at start-up, a host that forbids run-time
allocation, or a caller that cannot afford cudaMalloc's implicit
synchronisation). Its scratch is a fixed array inside the library. This test
calls it through the C ABI, twice in a row with different batches, and checks
each result against haru_sdtw_batch on the same inputs: int16 bit-exact, FP32
bitwise (the tolerance the other parity tests use); the first batch is also
checked against the oracle directly. It also runs pre-z-scored events
(flags 0), and a rejected call followed by a valid one on the same shared
array. Collected last so that a run stopping at the first failure has
already run everything else.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import compare_fp32, compare_int16

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call(h, ctx, prec, ev, off, cost, col, flags):
    lib = h.lib()
    return int(lib.haru_sdtw_batch_noalloc(ctx.handle, prec, ctypes.c_void_p(ev.data_ptr()),
                                           ctypes.c_void_p(off.data_ptr()), off.shape[0] - 1,
                                           ctypes.c_void_p(cost.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                           0, flags))


def _device(q_events, q_offsets, dev):
    return (torch.from_numpy(np.ascontiguousarray(q_events, dtype=np.float32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(q_offsets).astype(np.int32)).to(dev))


def _outputs(nq, dev):
    return (torch.full((nq,), -1.0, dtype=torch.float32, device=dev),
            torch.full((nq,), -7, dtype=torch.int64, device=dev))


def test_noalloc_matches_batch_on_two_calls():
    import paper_2211_07340_gb300 as h
    h.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    w = synth.workload("sars_32x250")
    ref = oracle.ref_levels(w.genome, w.model, w.k)
    first = synth.workload("sars_uneven_8192", nq=700).queries     # odd pair count, strip heights 4..16
    second = synth.workload("sars_4096x250", nq=1024).queries      # the size limit
    with h.Context() as ctx:
        ctx.ref_load(ref)
        for n, q in enumerate((first, second)):
            ev, off = _device(q.events, q.offsets, dev)
            for prec in (h.HARU_INT16, h.HARU_FP32):
                cost, col = _outputs(q.nq, dev)
                assert _call(h, ctx, prec, ev, off, cost, col, h.HARU_RAW) == h.HARU_OK
                got_c, got_j = cost.cpu().numpy(), col.cpu().numpy()
                want_c, want_j = ctx.sdtw_batch(prec, q.events, q.offsets)
                np.testing.assert_array_equal(got_j, want_j)
                np.testing.assert_array_equal(got_c, want_c)
                if n == 0:  # the first batch also straight against the oracle
                    if prec == h.HARU_INT16:
                        compare_int16(got_c, got_j, ref, q.events, q.offsets)
                    else:
                        compare_fp32(got_c, got_j, ref, q.events, q.offsets)

        # events already z-scored (flags 0): as haru_sdtw_batch with raw=False
        zq = first.subset(np.arange(200))
        zev = np.concatenate([oracle.zscore(zq.query(i)) for i in range(zq.nq)])
        ev, off = _device(zev, zq.offsets, dev)
        for prec in (h.HARU_INT16, h.HARU_FP32):
            cost, col = _outputs(zq.nq, dev)
            assert _call(h, ctx, prec, ev, off, cost, col, 0) == h.HARU_OK
            want_c, want_j = ctx.sdtw_batch(prec, zev, zq.offsets, raw=False)
            np.testing.assert_array_equal(col.cpu().numpy(), want_j)
            np.testing.assert_array_equal(cost.cpu().numpy(), want_c)

        # a batch with one invalid query (longer than HARU_MAX_QUERY) is
        # rejected; the next valid call on the shared array succeeds
        lens = [250, h.HARU_MAX_QUERY + 88, 250]
        bad_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint32)
        bad_ev = synth.random_signal(int(bad_off[-1]), seed=3)
        ev, off = _device(bad_ev, bad_off, dev)
        cost, col = _outputs(3, dev)
        assert _call(h, ctx, h.HARU_INT16, ev, off, cost, col, h.HARU_RAW) == h.HARU_EINVAL
        ev, off = _device(second.events, second.offsets, dev)
        cost, col = _outputs(second.nq, dev)
        assert _call(h, ctx, h.HARU_INT16, ev, off, cost, col, h.HARU_RAW) == h.HARU_OK
        want_c, want_j = ctx.sdtw_batch(h.HARU_INT16, second.events, second.offsets)
        np.testing.assert_array_equal(col.cpu().numpy(), want_j)
        np.testing.assert_array_equal(cost.cpu().numpy(), want_c)

        # beyond the scratch limit, or the wide form: rejected before any GPU work
        big = synth.workload("sars_4096x250", nq=h.HARU_NOALLOC_MAX_QUERIES + 1).queries
        ev, off = _device(big.events, big.offsets, dev)
        cost, col = _outputs(big.nq, dev)
        assert _call(h, ctx, h.HARU_INT16, ev, off, cost, col, h.HARU_RAW) == h.HARU_EINVAL
        ev, off = _device(first.events, first.offsets, dev)
        cost, col = _outputs(first.nq, dev)
        assert _call(h, ctx, h.HARU_INT16_ACC32, ev, off, cost, col, h.HARU_RAW) == h.HARU_EINVAL
