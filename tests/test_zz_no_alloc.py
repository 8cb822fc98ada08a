"""haru_sdtw_batch_noalloc: the batch entry point that allocates nothing.

It serves callers that cannot let the library allocate device memory (a
fixed memory budget reserved at start-up, a host that forbids run-time
allocation, or a caller that cannot afford cudaMalloc's implicit
synchronisation). Its scratch is a fixed array inside the library. This test
calls it through the C ABI, twice in a row with different batches, and checks
each result against haru_sdtw_batch on the same inputs: int16 bit-exact, FP32
bitwise (the tolerance the other parity tests use). Collected last so that a
run stopping at the first failure has already run everything else.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call(h, ctx, prec, ev, off, cost, col, flags):
    lib = h.lib()
    return int(lib.haru_sdtw_batch_noalloc(ctx.handle, prec, ctypes.c_void_p(ev.data_ptr()),
                                           ctypes.c_void_p(off.data_ptr()), off.shape[0] - 1,
                                           ctypes.c_void_p(cost.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                           0, flags))


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
        for q in (first, second):
            ev = torch.from_numpy(q.events).to(dev)
            off = torch.from_numpy(q.offsets.astype(np.int32)).to(dev)
            for prec in (h.HARU_INT16, h.HARU_FP32):
                cost = torch.full((q.nq,), -1.0, dtype=torch.float32, device=dev)
                col = torch.full((q.nq,), -7, dtype=torch.int64, device=dev)
                assert _call(h, ctx, prec, ev, off, cost, col, h.HARU_RAW) == h.HARU_OK
                want_c, want_j = ctx.sdtw_batch(prec, q.events, q.offsets)
                np.testing.assert_array_equal(col.cpu().numpy(), want_j)
                np.testing.assert_array_equal(cost.cpu().numpy(), want_c)
        # beyond the scratch limit: rejected before any GPU work
        big = synth.workload("sars_4096x250", nq=h.HARU_NOALLOC_MAX_QUERIES + 1).queries
        ev = torch.from_numpy(big.events).to(dev)
        off = torch.from_numpy(big.offsets.astype(np.int32)).to(dev)
        cost = torch.empty(big.nq, dtype=torch.float32, device=dev)
        col = torch.empty(big.nq, dtype=torch.int64, device=dev)
        assert _call(h, ctx, h.HARU_INT16, ev, off, cost, col, h.HARU_RAW) == h.HARU_EINVAL
