"""Helpers shared by the GPU tests: a context fixture and oracle comparisons."""
import numpy as np

import oracle


def compare_int16(cost, col, ref_levels, events, offsets, scale_log2=6, normalize_ref=True, idx=None,
                  normalize_q=True, prec=None):
    """Bit-exact check of an integer form (default the saturating int16 one;
    prec=oracle.PREC_I32 for wide accumulation) against the oracle on queries idx."""
    prec = oracle.PREC_I16 if prec is None else prec
    q = idx if idx is not None else np.arange(offsets.shape[0] - 1)
    sub_ev, sub_off = subset(events, offsets, q)
    o = oracle.batch(prec, ref_levels, sub_ev, sub_off, scale_log2=scale_log2,
                     normalize_ref=normalize_ref, normalize_q=normalize_q)
    np.testing.assert_array_equal(col[q], o.col, err_msg="integer form end column")
    np.testing.assert_array_equal(cost[q].astype(np.float64), o.cost, err_msg="integer form cost")
    return o


def compare_fp32(cost, col, ref_levels, events, offsets, normalize_ref=True, idx=None, bitwise=True,
                 normalize_q=True, f64_every=1):
    """FP32 form: bitwise equal to the FP32 oracle, and within 1e-5 relative
    of FP64 with the FP64 end column unless the FP64 runner-up is within
    that tolerance of the best. f64_every > 1 runs the FP64 check on every
    f64_every-th of the compared queries only (the bitwise check, which pins
    every result, still covers all of them)."""
    q = idx if idx is not None else np.arange(offsets.shape[0] - 1)
    sub_ev, sub_off = subset(events, offsets, q)
    o32 = oracle.batch(oracle.PREC_F32, ref_levels, sub_ev, sub_off, normalize_ref=normalize_ref,
                       normalize_q=normalize_q)
    q64 = q[::f64_every]
    ev64, off64 = (sub_ev, sub_off) if f64_every == 1 else subset(events, offsets, q64)
    o64 = oracle.batch(oracle.PREC_F64, ref_levels, ev64, off64, normalize_ref=normalize_ref,
                       normalize_q=normalize_q)
    if bitwise:
        np.testing.assert_array_equal(cost[q], o32.cost.astype(np.float32), err_msg="fp32 cost vs fp32 oracle")
        np.testing.assert_array_equal(col[q], o32.col, err_msg="fp32 column vs fp32 oracle")
    rel = np.abs(cost[q64].astype(np.float64) - o64.cost) / np.maximum(np.abs(o64.cost), 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    tol = 1e-5 * np.abs(o64.cost)
    must = (o64.runner_up - o64.cost) > tol
    np.testing.assert_array_equal(col[q64][must], o64.col[must], err_msg="fp32 column vs fp64")
    return o32, o64


def subset(events, offsets, q):
    """Events and offsets of queries q of a CSR batch."""
    parts = [events[offsets[i]:offsets[i + 1]] for i in q]
    off = np.zeros(len(parts) + 1, dtype=np.uint32)
    off[1:] = np.cumsum([p.shape[0] for p in parts])
    ev = np.concatenate(parts).astype(np.float32) if parts else np.zeros(0, np.float32)
    return ev, off
