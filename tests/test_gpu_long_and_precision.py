"""The long reference (5,000,000 bases, ~10M columns on both strands) and
the precision study (int16 and FP32 against the FP64 oracle).
"""
import json
import os

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


def test_long_reference_512x250(haru):
    w = synth.workload("long_512x250")
    q = w.queries
    ref = oracle.ref_levels(w.genome, w.model, w.k)
    assert ref.shape[0] == 9_999_990
    with haru.Context() as ctx:
        ctx.ref_build(w.genome, w.model, w.k, scale_log2=6)
        assert ctx.ref_length == ref.shape[0]
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, q.events, q.offsets)
        st16 = ctx.last_stats()
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, q.events, q.offsets)
        st32 = ctx.last_stats()
    # the sweep was split into many verified segments
    assert st16["max_segments"] > 4 and st32["max_segments"] > 4
    idx = np.array([0, 1, 2, 3, 255, 256, 510, 511])
    compare_int16(c16, j16, ref, q.events, q.offsets, idx=idx)
    compare_fp32(c32, j32, ref, q.events, q.offsets, idx=idx)
    on = q.on_target
    assert (np.abs(j32[on] - q.truth_end[on]) <= 8).mean() >= 0.9
    print(json.dumps({"long_reference": {"int16": st16, "fp32": st32}}))


def decisions(cost, thr):
    return cost <= thr


def test_precision_study_4096x250(haru):
    """Cost error of int16 (saturating), int16 with 32-bit accumulation (the
    paper's PE, at its scale 32 and at 64) and FP32 against FP64, end-column
    agreement, and accept/eject agreement at a threshold fixed on 1,024
    held-out queries (FP64 costs; fewest misclassified, midpoint of the gap)."""
    import bench
    w = synth.workload("sars_4096x250")
    held = synth.workload("sars_heldout_1024")
    ref = oracle.ref_levels(w.genome, w.model, w.k)
    q = w.queries
    hq = held.queries
    h64 = oracle.batch(oracle.PREC_F64, ref, hq.events, hq.offsets)
    thr = bench.pick_threshold(h64.cost, hq.on_target)
    o64 = oracle.batch(oracle.PREC_F64, ref, q.events, q.offsets)
    with haru.Context() as ctx:
        ctx.ref_load(ref, scale_log2=6)
        c16, j16 = ctx.sdtw_batch(haru.HARU_INT16, q.events, q.offsets)
        c32, j32 = ctx.sdtw_batch(haru.HARU_FP32, q.events, q.offsets)
        cw64, jw64 = ctx.sdtw_batch(haru.HARU_INT16_ACC32, q.events, q.offsets)
        sweep, wide = {}, {}
        for k in range(1, 8):
            ctx.ref_load(ref, scale_log2=k)
            ck, jk = ctx.sdtw_batch(haru.HARU_INT16, q.events, q.offsets)
            cw, jw = ctx.sdtw_batch(haru.HARU_INT16_ACC32, q.events, q.offsets)
            sweep[2 ** k] = {"position_agreement_vs_fp32": float(np.mean(np.abs(jk - j32) <= 0)),
                             "position_within_5_vs_fp32": float(np.mean(np.abs(jk - j32) <= 5)),
                             "capped": int(np.sum(ck * 2 ** k >= haru.HARU_INT16_CAP)),
                             "acc32_position_agreement_vs_fp32": float(np.mean(jw == j32)),
                             "acc32_decision_agreement_vs_fp64":
                                 float(np.mean(decisions(cw.astype(np.float64), np.floor(thr * 2 ** k) / 2 ** k)
                                               == decisions(o64.cost, thr)))}
            wide[2 ** k] = (cw, jw)
    rel32 = np.abs(c32 - o64.cost) / o64.cost
    rel16 = np.abs(c16 - o64.cost) / o64.cost
    # FP32 form: the 1e-5 relative bar, and the FP64 column where it is unique
    assert rel32.max() <= 1e-5
    uniq = (o64.runner_up - o64.cost) > 1e-5 * o64.cost
    np.testing.assert_array_equal(j32[uniq], o64.col[uniq])
    d64 = decisions(o64.cost, thr)
    d32 = decisions(c32.astype(np.float64), thr)
    d16 = decisions(c16.astype(np.float64), np.floor(thr * 64) / 64)
    agree16 = float(np.mean(d16 == d64))
    agree32 = float(np.mean(d32 == d64))
    assert agree32 >= 0.999
    assert agree16 >= 0.999
    # wide accumulation never saturates: equal to int16 below CAP, larger above
    below = c16 * 64 < haru.HARU_INT16_CAP
    np.testing.assert_array_equal(cw64[below], c16[below])
    assert (cw64[~below] * 64 >= haru.HARU_INT16_CAP).all()
    relw = {}
    for s_, (cw, jw) in wide.items():
        r = np.abs(cw - o64.cost) / o64.cost
        dw = decisions(cw.astype(np.float64), np.floor(thr * s_) / s_)
        relw[s_] = {"max_rel_err": float(r.max()), "p99_rel_err": float(np.percentile(r, 99)),
                    "col_agreement": float(np.mean(jw == o64.col)),
                    "col_within_5": float(np.mean(np.abs(jw - o64.col) <= 5)),
                    "decision_agreement": float(np.mean(dw == d64))}
    assert relw[64]["decision_agreement"] >= 0.999
    report = {
        "threshold_z": thr,
        "fp32": {"max_rel_err": float(rel32.max()), "p99_rel_err": float(np.percentile(rel32, 99)),
                 "col_agreement": float(np.mean(j32 == o64.col)), "decision_agreement": agree32},
        "int16_scale64": {"max_rel_err": float(rel16.max()), "p99_rel_err": float(np.percentile(rel16, 99)),
                          "col_agreement": float(np.mean(j16 == o64.col)),
                          "col_within_5": float(np.mean(np.abs(j16 - o64.col) <= 5)),
                          "decision_agreement": agree16},
        "int16_acc32_scale32": relw[32],
        "int16_acc32_scale64": relw[64],
        "truth_accuracy_fp64": float(np.mean(d64 == q.on_target)),
        "scale_sweep_int16_vs_fp32": sweep,
    }
    out = os.environ.get("HARU_PRECISION_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(report, f, indent=1)
    print(json.dumps(report))
