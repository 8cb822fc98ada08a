"""Oracle for HARU's sDTW hot path: a plain CPU restatement of the paper.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline / reference leg may import this package. The CUDA
library never imports, links or calls it, and it shares no code with it.

The arithmetic lives in sdtw_oracle.cpp (plain C++17, compiled with
-ffp-contract=off): Eq. 1 and Algorithm 1 (full matrix), Algorithm 2 (one
rolling cost array), the Section 4.3 processing-element chain (oblique
order), the Section 4.1 reference synthesis, z-score and fixed-point
quantiser; and in event_oracle.cpp: the event detection and adaptor trimming
of the Section 4.1 pre-processing (two-window t-test). This module only
builds those files and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdtw_oracle.cpp")
_SRC_EVENTS = os.path.join(_HERE, "event_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PREC_F32, PREC_I16, PREC_F64, PREC_I32 = 0, 1, 2, 3  # PREC_I32: int16 inputs, 32-bit accumulation


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                              os.path.getmtime(_SRC_EVENTS)):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                                   "-fPIC", "-shared", "-pthread", _SRC, _SRC_EVENTS, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_zscore.argtypes = [P, ctypes.c_size_t, P]
        lib.oracle_zscore.restype = ctypes.c_int
        lib.oracle_quantise.argtypes = [P, ctypes.c_size_t, ctypes.c_int, P]
        lib.oracle_quantise.restype = None
        lib.oracle_ref_levels.argtypes = [P, ctypes.c_size_t, P, ctypes.c_int, P]
        lib.oracle_ref_levels.restype = ctypes.c_long
        for name in ("oracle_sdtw_full_f64", "oracle_sdtw_roll_f64"):
            getattr(lib, name).restype = None
        lib.oracle_sdtw_full_f64.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P]
        lib.oracle_sdtw_full_i16.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P]
        lib.oracle_sdtw_full_i16.restype = None
        lib.oracle_sdtw_lastrow_f64.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P]
        lib.oracle_sdtw_lastrow_f64.restype = None
        lib.oracle_sdtw_roll_f64.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P, P]
        lib.oracle_sdtw_roll_f32.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P]
        lib.oracle_sdtw_roll_f32.restype = None
        lib.oracle_sdtw_roll_i16.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P]
        lib.oracle_sdtw_roll_i16.restype = None
        lib.oracle_sdtw_roll_i32.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P]
        lib.oracle_sdtw_roll_i32.restype = None
        lib.oracle_batch.argtypes = [ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int, P, P, ctypes.c_uint32,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        lib.oracle_sdtw_span_f32.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P, P]
        lib.oracle_sdtw_span_f32.restype = None
        lib.oracle_sdtw_span_i32.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P, P]
        lib.oracle_sdtw_span_i32.restype = None
        lib.oracle_sdtw_wavefront_f64.argtypes = [P, ctypes.c_int, P, ctypes.c_long, P, P, P]
        lib.oracle_sdtw_wavefront_f64.restype = None
        lib.oracle_batch.restype = ctypes.c_int
        L = ctypes.c_long
        lib.oracle_event_tstat.argtypes = [P, L, ctypes.c_int, P, P]
        lib.oracle_event_tstat.restype = None
        lib.oracle_event_boundaries.argtypes = [P, L, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, L]
        lib.oracle_event_boundaries.restype = L
        lib.oracle_read_events.argtypes = [P, L, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, L, L, P]
        lib.oracle_read_events.restype = L
        lib.oracle_signal_batch.argtypes = [P, P, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, L, L, ctypes.c_int, P, P]
        lib.oracle_signal_batch.restype = None
        lib.oracle_cap.restype = ctypes.c_int
        lib.oracle_qmax.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def cap() -> int:
    return int(_load().oracle_cap())


def qmax() -> int:
    return int(_load().oracle_qmax())


def zscore(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    z = np.empty_like(x)
    if _load().oracle_zscore(_p(x), x.shape[0], _p(z)) != 0:
        raise ValueError("z-score undefined (empty input or zero spread)")
    return z


def quantise(z, scale_log2: int) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float32)
    q = np.empty(z.shape[0], dtype=np.int16)
    _load().oracle_quantise(_p(z), z.shape[0], int(scale_log2), _p(q))
    return q


def ref_levels(bases, model, k: int) -> np.ndarray:
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    model = np.ascontiguousarray(model, dtype=np.float32)
    n = bases.shape[0]
    out = np.empty(max(0, 2 * (n - k + 1)), dtype=np.float32)
    r = _load().oracle_ref_levels(_p(bases), n, _p(model), int(k), _p(out))
    if r < 0:
        raise ValueError("genome shorter than k")
    return out


def sdtw_full_f64(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c, j = ctypes.c_double(), ctypes.c_long()
    _load().oracle_sdtw_full_f64(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j))
    return c.value, j.value


def sdtw_full_i16(x, y):
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    c, j = ctypes.c_int32(), ctypes.c_long()
    _load().oracle_sdtw_full_i16(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j))
    return c.value, j.value


def sdtw_lastrow_f64(x, y) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    last = np.empty(y.shape[0], dtype=np.float64)
    _load().oracle_sdtw_lastrow_f64(_p(x), x.shape[0], _p(y), y.shape[0], _p(last))
    return last


def sdtw_roll_f64(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c, j, r = ctypes.c_double(), ctypes.c_long(), ctypes.c_double()
    _load().oracle_sdtw_roll_f64(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j),
                                 ctypes.byref(r))
    return c.value, j.value, r.value


def sdtw_wavefront_f64(x, y):
    """Eq. 1 in the processing-element chain's oblique order (Section 4.3,
    Fig. 5): (cost, end column, steps the chain ran)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c, j, t = ctypes.c_double(), ctypes.c_long(), ctypes.c_long()
    _load().oracle_sdtw_wavefront_f64(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j),
                                      ctypes.byref(t))
    return c.value, j.value, t.value


def sdtw_roll_f32(x, y):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    c, j = ctypes.c_float(), ctypes.c_long()
    _load().oracle_sdtw_roll_f32(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j))
    return c.value, j.value


def sdtw_roll_i32(x, y):
    """int16 inputs, wide (exact) accumulation: the unsaturated integer DP."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    c, j = ctypes.c_int64(), ctypes.c_long()
    _load().oracle_sdtw_roll_i32(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j))
    return c.value, j.value


def sdtw_roll_i16(x, y):
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    c, j = ctypes.c_int32(), ctypes.c_long()
    _load().oracle_sdtw_roll_i16(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j))
    return c.value, j.value


def sdtw_span_f32(x, y):
    """FP32 DP carrying each path's start column: (cost, end column, start column)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    c, j, s = ctypes.c_float(), ctypes.c_long(), ctypes.c_long()
    _load().oracle_sdtw_span_f32(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j),
                                 ctypes.byref(s))
    return c.value, j.value, s.value


def sdtw_span_i32(x, y):
    """Wide-accumulation integer DP carrying each path's start column."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    c, j, s = ctypes.c_int64(), ctypes.c_long(), ctypes.c_long()
    _load().oracle_sdtw_span_i32(_p(x), x.shape[0], _p(y), y.shape[0], ctypes.byref(c), ctypes.byref(j),
                                 ctypes.byref(s))
    return c.value, j.value, s.value


class BatchResult:
    def __init__(self, cost, col, runner_up, icost, start=None):
        self.cost, self.col, self.runner_up, self.icost, self.start = cost, col, runner_up, icost, start


def batch(prec: int, ref, events, offsets, scale_log2: int = 6, normalize_ref: bool = True,
          normalize_q: bool = True, threads: int = 0, start: bool = False) -> BatchResult:
    """The whole path on the CPU: z-score, quantise (integer forms), Algorithm 2 per query."""
    ref = np.ascontiguousarray(ref, dtype=np.float32)
    events = np.ascontiguousarray(events, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    nq = offsets.shape[0] - 1
    cost = np.empty(nq, dtype=np.float64)
    col = np.empty(nq, dtype=np.int64)
    ru = np.empty(nq, dtype=np.float64)
    ic = np.zeros(nq, dtype=np.int32)
    if start and prec not in (PREC_F32, PREC_I32):
        raise ValueError("start columns: FP32 and wide-accumulation forms only")
    st = np.full(nq, -1, dtype=np.int64) if start else None
    bad = ctypes.c_long(-1)
    ev = events if events.shape[0] else np.zeros(1, np.float32)
    r = _load().oracle_batch(int(prec), _p(ref), ref.shape[0], int(normalize_ref), _p(ev), _p(offsets), nq,
                             int(normalize_q), int(scale_log2), int(threads), _p(cost), _p(col), _p(ru), _p(ic),
                             _p(st) if start else None, ctypes.byref(bad))
    if r != 0:
        raise ValueError(f"invalid input (query {bad.value})")
    return BatchResult(cost, col, ru if prec == PREC_F64 else None, ic if prec in (PREC_I16, PREC_I32) else None,
                       st)


# --------------------------------------------------- event detection --
# Defaults read for R9.4 (see event_oracle.cpp): windows of 3 and 6 samples,
# t thresholds 1.40 and 9.00 (in hundredths), 50 adaptor events trimmed,
# 250 query events.
EVENT_DEFAULTS = {"w1": 3, "w2": 6, "tau1_centi": 140, "tau2_centi": 900, "trim": 50, "max_events": 250}


def event_tstat(x, w: int):
    """Two-window t statistic of every position 0..n as (num, den): t^2 =
    num / den; den = 0 where it is undefined (positions < w or > n - w)."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    n = x.shape[0]
    num = np.empty(n + 1, dtype=np.int64)
    den = np.empty(n + 1, dtype=np.int64)
    _load().oracle_event_tstat(_p(x), n, int(w), _p(num), _p(den))
    return num, den


def event_boundaries(x, w1=3, w2=6, tau1_centi=140, tau2_centi=900) -> np.ndarray:
    """Sample positions where a new event starts (0 excluded), ascending."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    n = x.shape[0]
    out = np.empty(n + 1, dtype=np.int64)
    nb = _load().oracle_event_boundaries(_p(x), n, int(w1), int(w2), int(tau1_centi), int(tau2_centi), _p(out),
                                         n + 1)
    return out[:nb].copy()


def read_events(x, w1=3, w2=6, tau1_centi=140, tau2_centi=900, trim=50, max_events=250) -> np.ndarray:
    """The query of one read: means of events [trim, trim + max_events) (float32)."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    out = np.empty(max(1, int(max_events)), dtype=np.float32)
    k = _load().oracle_read_events(_p(x), x.shape[0], int(w1), int(w2), int(tau1_centi), int(tau2_centi),
                                   int(trim), int(max_events), _p(out))
    return out[:k].copy()


def signal_events(samples, offsets, threads: int = 0, **params):
    """Every read of a raw-signal batch to its query events: (events float32
    CSR, offsets uint32[nreads + 1])."""
    p = dict(EVENT_DEFAULTS, **params)
    samples = np.ascontiguousarray(samples, dtype=np.int16)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    nr = offsets.shape[0] - 1
    cap = int(p["max_events"])
    out = np.empty(max(1, nr * cap), dtype=np.float32)
    counts = np.zeros(max(1, nr), dtype=np.uint32)
    smp = samples if samples.shape[0] else np.zeros(1, np.int16)
    _load().oracle_signal_batch(_p(smp), _p(offsets), nr, int(p["w1"]), int(p["w2"]), int(p["tau1_centi"]),
                                int(p["tau2_centi"]), int(p["trim"]), cap, int(threads), _p(out), _p(counts))
    counts = counts[:nr]
    off = np.zeros(nr + 1, dtype=np.uint32)
    off[1:] = np.cumsum(counts)
    ev = np.concatenate([out[r * cap:r * cap + int(counts[r])] for r in range(nr)]) if nr else np.zeros(0)
    return ev.astype(np.float32), off
