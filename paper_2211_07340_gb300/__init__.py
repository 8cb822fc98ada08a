"""Python binding of libharu (include/haru.h): argument marshalling only.

Every step of the sDTW path (reference synthesis, z-score, quantisation,
planning, the wavefront kernels) runs in the CUDA library; this module loads
it with ctypes and passes pointers. There is no CPU fallback: if the library
is missing the import of `lib()` raises.

Device buffers may be torch tensors (their data_ptr() is passed with
HARU_ON_DEVICE); host buffers are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libharu.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "haru.h")

HARU_OK = 0
HARU_EINVAL = -1
HARU_ENOREF = -2
HARU_ENOMEM = -3
HARU_EBUSY = -4
HARU_ETIMEDOUT = -5
HARU_ECUDA = -6
HARU_FP32 = 0
HARU_INT16 = 1
HARU_INT16_ACC32 = 2  # int16 inputs, wide (32-bit) accumulation: the exact integer cost
HARU_ON_DEVICE = 1
HARU_RAW = 2
HARU_ASYNC = 4
HARU_PROFILE = 8
HARU_INT16_QMAX = 2047
HARU_INT16_CAP = 28673
HARU_MAX_QUERY = 512
HARU_NOALLOC_MAX_QUERIES = 1024
HARU_MAX_READ_SAMPLES = 16384


class HaruError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        name = lib().haru_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {name} ({code})" if what else f"{name} ({code})")


class haru_event_params(ctypes.Structure):
    _fields_ = [("window_short", ctypes.c_int), ("window_long", ctypes.c_int),
                ("threshold_short_centi", ctypes.c_int), ("threshold_long_centi", ctypes.c_int),
                ("trim_events", ctypes.c_uint32), ("max_events", ctypes.c_uint32)]


class haru_config(ctypes.Structure):
    _fields_ = [
        ("warps_per_cta", ctypes.c_int),
        ("tile_cols", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("wait_limit", ctypes.c_uint32),
        ("threshold", ctypes.c_float),
        ("serve_precision", ctypes.c_int),
        ("serve_budget_bytes", ctypes.c_size_t),
        ("serve_max_batch", ctypes.c_uint32),
        ("serve_prefix", ctypes.c_uint32),
        ("units_target", ctypes.c_int),
        ("stack_short", ctypes.c_int),
        ("serve_spin_us", ctypes.c_int),
        ("serve_events", haru_event_params),
    ]


class haru_batch_stats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_uint32), ("groups", ctypes.c_uint32), ("fixups", ctypes.c_uint32),
                ("max_segments", ctypes.c_uint32)]


class haru_result(ctypes.Structure):
    _fields_ = [("read_id", ctypes.c_uint64), ("channel", ctypes.c_uint32), ("decision", ctypes.c_int32),
                ("cost", ctypes.c_float), ("status", ctypes.c_int32), ("end_col", ctypes.c_int64),
                ("events", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("t_arrival_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("t_received_ns", ctypes.c_uint64)]


class haru_stream_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("reads_submitted", "reads_decided", "reads_waiting",
                                               "reads_in_flight", "batches", "max_batch", "max_concurrent",
                                               "slots", "max_upload_ns", "max_queue_ns", "max_gpu_ns",
                                               "slow_upload", "slow_queue", "slow_gpu", "max_upload_sync_ns",
                                               "max_turn_gap_ns", "worst_turn_complete_ns", "worst_turn_upload_ns",
                                               "worst_turn_launch_ns", "worst_turn_wait_ns",
                                               "worst_turn_voluntary_switches",
                                               "worst_turn_involuntary_switches", "max_gpu_exec_ns",
                                               "max_notice_ns", "max_drain_ns", "max_upload_calls_ns",
                                               "max_launch_inputs_ns", "max_launch_path_ns",
                                               "max_launch_results_ns", "max_detect_calls_ns",
                                               "worst_turn_detect_ns", "worst_turn_minor_faults",
                                               "worst_turn_major_faults", "worst_turn_at_ns", "turns_over_5ms",
                                               "worker_minor_faults", "worker_voluntary_switches",
                                               "max_lock_wait_ns", "max_upload_host_ns")]


_lib = None

_SIGS = {
    "haru_config_default": (ctypes.c_int, [ctypes.POINTER(haru_config)]),
    "haru_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(haru_config)]),
    "haru_destroy": (None, [ctypes.c_void_p]),
    "haru_configure": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(haru_config)]),
    "haru_get_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(haru_config)]),
    "haru_ref_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
    "haru_ref_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int]),
    "haru_ref_length": (ctypes.c_size_t, [ctypes.c_void_p]),
    "haru_ref_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "haru_sdtw_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_uint32]),
    "haru_sdtw_batch_span": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_uint32]),
    "haru_last_status": (ctypes.c_int, [ctypes.c_void_p]),
    "haru_event_params_default": (ctypes.c_int, [ctypes.POINTER(haru_event_params)]),
    "haru_detect_events": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                          ctypes.POINTER(haru_event_params), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_uint32]),
    "haru_sdtw_batch_signal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_uint32, ctypes.POINTER(haru_event_params), ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32]),
    "haru_last_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(haru_batch_stats)]),
    "haru_stream_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]),
    "haru_stream_submit_signal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]),
    "haru_stream_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32]),
    "haru_stream_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(haru_stream_stats)]),
    "haru_last_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float)]),
    "haru_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "haru_probe_peak": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "haru_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.POINTER(haru_config)]),
    "haru_sdtw_batch_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                               ctypes.c_uint32]),
}


def build_library(force: bool = False) -> str:
    """Compile libharu.so in-tree (nvcc, sm_103a)."""
    import importlib
    return importlib.import_module(__name__ + ".build").build(force=force)


def lib():
    """Load libharu.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libharu.so not built ({LIB_PATH}); run paper_2211_07340_gb300.build_library()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols() -> list[str]:
    """Entry points declared in include/haru.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(haru_[a-z_0-9]+)\s*\(", txt, re.M)))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def check(code: int, what: str = ""):
    if code != HARU_OK:
        raise HaruError(code, what)
    return code


def default_config(**kw) -> haru_config:
    cfg = haru_config()
    check(lib().haru_config_default(ctypes.byref(cfg)))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


class Context:
    """One libharu context on one CUDA device."""

    def __init__(self, device: int = 0, config: haru_config | None = None, **kw):
        self._h = ctypes.c_void_p()
        cfg = config if config is not None else default_config(**kw)
        check(lib().haru_create(ctypes.byref(self._h), int(device), ctypes.byref(cfg)), "haru_create")
        self.config = cfg

    @property
    def handle(self):
        return self._h

    def configure(self, **kw):
        """Change configuration fields (launch shape, int16 mode, ...) for later batches."""
        cfg = haru_config()
        check(lib().haru_get_config(self._h, ctypes.byref(cfg)), "haru_get_config")
        for k, v in kw.items():
            setattr(cfg, k, v)
        check(lib().haru_configure(self._h, ctypes.byref(cfg)), "haru_configure")
        self.config = cfg
        return cfg

    def close(self):
        if self._h:
            lib().haru_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # reference -----------------------------------------------------------
    def ref_load(self, levels, normalize: bool = True, scale_log2: int = 6):
        levels = np.ascontiguousarray(levels, dtype=np.float32)
        return check(lib().haru_ref_load(self._h, _ptr(levels), levels.shape[0], int(normalize), int(scale_log2)),
                     "haru_ref_load")

    def ref_build(self, bases, kmer_levels, k: int = 6, scale_log2: int = 6):
        bases = np.ascontiguousarray(bases, dtype=np.uint8)
        kmer_levels = np.ascontiguousarray(kmer_levels, dtype=np.float32)
        return check(lib().haru_ref_build(self._h, _ptr(bases), bases.shape[0], _ptr(kmer_levels), int(k),
                                          int(scale_log2)), "haru_ref_build")

    @property
    def ref_length(self) -> int:
        return int(lib().haru_ref_length(self._h))

    def ref_read(self):
        n = self.ref_length
        z = np.empty(n, dtype=np.float32)
        q = np.empty(n, dtype=np.int16)
        check(lib().haru_ref_read(self._h, _ptr(z), _ptr(q), n), "haru_ref_read")
        return z, q

    # batch ----------------------------------------------------------------
    def sdtw_batch_raw(self, precision: int, events, offsets, nq: int, out_cost, out_col, stream: int = 0,
                       flags: int = 0) -> int:
        """Direct call of haru_sdtw_batch with caller-provided buffers; returns the status code."""
        return int(lib().haru_sdtw_batch(self._h, int(precision), _ptr(events), _ptr(offsets), int(nq),
                                         _ptr(out_cost), _ptr(out_col), int(stream), int(flags)))

    def sdtw_batch(self, precision: int, events, offsets, raw: bool = True):
        """Host arrays in, host arrays out: (cost float32[nq], col int64[nq])."""
        events = np.ascontiguousarray(events, dtype=np.float32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        nq = offsets.shape[0] - 1
        cost = np.empty(max(nq, 1), dtype=np.float32)
        col = np.empty(max(nq, 1), dtype=np.int64)
        ev = events if events.shape[0] else np.zeros(1, np.float32)
        check(self.sdtw_batch_raw(precision, ev, offsets, nq, cost, col, 0, HARU_RAW if raw else 0),
              "haru_sdtw_batch")
        return cost[:nq], col[:nq]

    def sdtw_batch_span(self, precision: int, events, offsets, raw: bool = True):
        """haru_sdtw_batch_span with host arrays: (cost float32[nq], end col int64[nq],
        start col int64[nq]); precision HARU_FP32 or HARU_INT16_ACC32."""
        events = np.ascontiguousarray(events, dtype=np.float32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        nq = offsets.shape[0] - 1
        cost = np.empty(max(nq, 1), dtype=np.float32)
        col = np.empty(max(nq, 1), dtype=np.int64)
        start = np.empty(max(nq, 1), dtype=np.int64)
        ev = events if events.shape[0] else np.zeros(1, np.float32)
        check(int(lib().haru_sdtw_batch_span(self._h, int(precision), _ptr(ev), _ptr(offsets), int(nq), _ptr(cost),
                                             _ptr(col), _ptr(start), 0, HARU_RAW if raw else 0)),
              "haru_sdtw_batch_span")
        return cost[:nq], col[:nq], start[:nq]

    def sdtw_batch_span_device(self, precision: int, events, offsets, out_cost, out_col, out_start,
                               stream: int = 0, raw: bool = True, asynchronous: bool = False):
        """haru_sdtw_batch_span on device tensors (torch), ordered on `stream`."""
        nq = int(offsets.shape[0]) - 1
        flags = HARU_ON_DEVICE | (HARU_RAW if raw else 0) | (HARU_ASYNC if asynchronous else 0)
        return check(int(lib().haru_sdtw_batch_span(self._h, int(precision), _ptr(events), _ptr(offsets), nq,
                                                    _ptr(out_cost), _ptr(out_col), _ptr(out_start), int(stream),
                                                    flags)), "haru_sdtw_batch_span")

    def sdtw_batch_device(self, precision: int, events, offsets, out_cost, out_col, stream: int = 0,
                          raw: bool = True, asynchronous: bool = False, profile: bool = False):
        """Device tensors in and out (torch), ordered on `stream` (a cudaStream_t as int)."""
        nq = int(offsets.shape[0]) - 1
        flags = (HARU_ON_DEVICE | (HARU_RAW if raw else 0) | (HARU_ASYNC if asynchronous else 0)
                 | (HARU_PROFILE if profile else 0))
        return check(self.sdtw_batch_raw(precision, events, offsets, nq, out_cost, out_col, stream, flags),
                     "haru_sdtw_batch")

    # raw signal ------------------------------------------------------------
    @staticmethod
    def event_params(**kw) -> haru_event_params:
        p = haru_event_params()
        check(lib().haru_event_params_default(ctypes.byref(p)))
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def detect_events(self, samples, offsets, params: haru_event_params | None = None):
        """Host int16 samples (CSR) in: (events float32 CSR, event offsets uint32)."""
        p = params if params is not None else self.event_params()
        samples = np.ascontiguousarray(samples, dtype=np.int16)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        nr = offsets.shape[0] - 1
        ev = np.empty(max(1, nr * p.max_events), dtype=np.float32)
        eoff = np.zeros(nr + 1, dtype=np.uint32)
        smp = samples if samples.shape[0] else np.zeros(1, np.int16)
        check(int(lib().haru_detect_events(self._h, _ptr(smp), _ptr(offsets), nr, ctypes.byref(p), _ptr(ev),
                                           _ptr(eoff), 0, 0)), "haru_detect_events")
        return ev[:int(eoff[-1])].copy(), eoff

    def detect_events_device(self, samples, offsets, events, event_offsets, params=None, stream: int = 0,
                             asynchronous: bool = False):
        """haru_detect_events on device tensors (torch), ordered on `stream`."""
        p = params if params is not None else self.event_params()
        nr = int(offsets.shape[0]) - 1
        flags = HARU_ON_DEVICE | (HARU_ASYNC if asynchronous else 0)
        return check(int(lib().haru_detect_events(self._h, _ptr(samples), _ptr(offsets), nr, ctypes.byref(p),
                                                  _ptr(events), _ptr(event_offsets), int(stream), flags)),
                     "haru_detect_events")

    def sdtw_batch_signal(self, precision: int, samples, offsets, params: haru_event_params | None = None):
        """Raw int16 samples (host CSR) to (cost float32[nr], col int64[nr], query events uint32[nr])."""
        p = params if params is not None else self.event_params()
        samples = np.ascontiguousarray(samples, dtype=np.int16)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        nr = offsets.shape[0] - 1
        cost = np.empty(max(nr, 1), dtype=np.float32)
        col = np.empty(max(nr, 1), dtype=np.int64)
        nev = np.zeros(max(nr, 1), dtype=np.uint32)
        smp = samples if samples.shape[0] else np.zeros(1, np.int16)
        check(self.sdtw_batch_signal_raw(precision, smp, offsets, nr, p, cost, col, nev, 0, 0),
              "haru_sdtw_batch_signal")
        return cost[:nr], col[:nr], nev[:nr]

    def sdtw_batch_signal_raw(self, precision: int, samples, offsets, nreads: int, params, out_cost, out_col,
                              out_events, stream: int = 0, flags: int = 0) -> int:
        """Direct call of haru_sdtw_batch_signal; returns the status code."""
        p = params if params is not None else self.event_params()
        return int(lib().haru_sdtw_batch_signal(self._h, int(precision), _ptr(samples), _ptr(offsets), int(nreads),
                                                ctypes.byref(p), _ptr(out_cost), _ptr(out_col), _ptr(out_events),
                                                int(stream), int(flags)))

    def sdtw_batch_signal_device(self, precision: int, samples, offsets, out_cost, out_col, out_events=None,
                                 params=None, stream: int = 0, asynchronous: bool = False, profile: bool = False):
        """haru_sdtw_batch_signal on device tensors (torch), ordered on `stream`."""
        nr = int(offsets.shape[0]) - 1
        flags = HARU_ON_DEVICE | (HARU_ASYNC if asynchronous else 0) | (HARU_PROFILE if profile else 0)
        return check(self.sdtw_batch_signal_raw(precision, samples, offsets, nr, params, out_cost, out_col,
                                                out_events, stream, flags), "haru_sdtw_batch_signal")

    def last_status(self) -> int:
        return int(lib().haru_last_status(self._h))

    def last_stats(self) -> dict:
        st = haru_batch_stats()
        check(lib().haru_last_stats(self._h, ctypes.byref(st)), "haru_last_stats")
        return {"items": st.items, "groups": st.groups, "fixups": st.fixups, "max_segments": st.max_segments}

    # serving -------------------------------------------------------------
    def stream_submit(self, read_id: int, channel: int, events, t_arrival_ns: int, last_chunk: bool = False) -> int:
        """Append a chunk of raw events (numpy float32) to a read; returns the status code."""
        ev = np.ascontiguousarray(events, dtype=np.float32)
        return int(lib().haru_stream_submit(self._h, int(read_id), int(channel), _ptr(ev) if ev.size else None,
                                            int(ev.shape[0]), int(t_arrival_ns), int(bool(last_chunk))))

    def stream_submit_signal(self, read_id: int, channel: int, samples, t_arrival_ns: int,
                             last_chunk: bool = False) -> int:
        """Append a chunk of raw int16 ADC samples to a read; returns the status code."""
        smp = np.ascontiguousarray(samples, dtype=np.int16)
        return int(lib().haru_stream_submit_signal(self._h, int(read_id), int(channel),
                                                   _ptr(smp) if smp.size else None, int(smp.shape[0]),
                                                   int(t_arrival_ns), int(bool(last_chunk))))

    def stream_poll(self, max_results: int = 4096, timeout_us: int = 1000):
        """Finished decisions as a list of haru_result (possibly empty). The
        receive buffer is kept between calls (no allocation per poll)."""
        buf = getattr(self, "_poll_buf", None)
        if buf is None or len(buf) < max_results:
            buf = self._poll_buf = (haru_result * max_results)()
        n = ctypes.c_uint32()
        check(lib().haru_stream_poll(self._h, buf, max_results, ctypes.byref(n), int(timeout_us)), "haru_stream_poll")
        return [haru_result.from_buffer_copy(buf[i]) for i in range(n.value)]

    def stream_stats(self) -> dict:
        st = haru_stream_stats()
        check(lib().haru_stream_get_stats(self._h, ctypes.byref(st)), "haru_stream_get_stats")
        return {f: int(getattr(st, f)) for f, _ in haru_stream_stats._fields_}

    def autotune(self, precision: int, events, offsets, raw: bool = True, on_device: bool = False) -> dict:
        """Pick warps per CTA, tile width and work-unit target on this batch;
        the choice stays in the context. Returns the chosen settings."""
        cfg = haru_config()
        nq = int(offsets.shape[0]) - 1
        flags = (HARU_RAW if raw else 0) | (HARU_ON_DEVICE if on_device else 0)
        if not on_device:
            events = np.ascontiguousarray(events, dtype=np.float32)
            offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        check(lib().haru_autotune(self._h, int(precision), _ptr(events), _ptr(offsets), nq, flags,
                                  ctypes.byref(cfg)), "haru_autotune")
        self.config = cfg
        return {"warps_per_cta": cfg.warps_per_cta, "tile_cols": cfg.tile_cols, "units_target": cfg.units_target,
                "stack_short": cfg.stack_short}

    def probe_peak(self, precision: int) -> float:
        """Measured cells/s ceiling of the form's cell update (no data movement)."""
        v = ctypes.c_double()
        check(lib().haru_probe_peak(self._h, int(precision), ctypes.byref(v)), "haru_probe_peak")
        return v.value

    def last_timing(self):
        """(ms_prep, ms_sweep) of the last HARU_PROFILE batch."""
        a, b = ctypes.c_float(), ctypes.c_float()
        check(lib().haru_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)), "haru_last_timing")
        return a.value, b.value


def shard_queries(offsets, world: int, rank: int):
    """Contiguous range [lo, hi) of queries for `rank` of `world` GPUs, cut so
    that every rank gets about the same number of events (the sweep's work
    grows with each query's length). Queries are independent, so ranks need
    no exchange beyond gathering their results."""
    off = np.asarray(offsets, dtype=np.int64)
    nq = off.shape[0] - 1
    if world <= 1 or nq == 0:
        return 0, nq
    total = int(off[-1])
    cuts = [0] + [int(np.searchsorted(off, total * r / world, side="left")) for r in range(1, world)] + [nq]
    cuts = [min(max(c, 0), nq) for c in cuts]
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return cuts[rank], cuts[rank + 1]
