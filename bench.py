"""Benchmark of the sDTW hot path (HARU Read Until) on GB300.

One step = one batch of the uneven SARS-CoV-2-shaped workload (8,192 raw
event queries, lengths uniform in [100, 500], 50% on-target) through the
whole device path: the planner, per-query z-score + quantisation + packing,
and the persistent sweep kernel, replayed from a CUDA graph with the inputs
already in HBM. The headline form is int16 (two queries per 32-bit lane,
DPX min-plus); the FP32 form is timed the same way beside it.

Prints ONE JSON line (rank 0). GCUPS = sum over queries of M * N / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the oracle (the plain CPU restatement of the paper,
multi-threaded over queries) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "sDTW GCUPS (int16 DPX vs FP32) at 1 GB300; p50/p99 Read Until decision latency"
WORKLOAD = "sars_uneven_8192"
WORKLOAD_DESC = ("8192 raw-event queries, M ~ U[100,500], 50% on-target, vs a 29,903-base genome's 6-mer "
                 "levels on both strands (N = 59,796)")
LONG_DESC = ("512 raw-event queries x 250 events, 50% on-target, vs a 5,000,000-base genome's 6-mer levels on "
             "both strands (N = 9,999,990)")
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def profiled_traffic(form: str):
    """DRAM bytes (read + write) of one batch's sweep kernels from the
    committed ncu summary, or None if the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "sdtw_sweep_sars_uneven_8192.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("    "):
                k, v = line.strip().split(":", 1)
                vals[k.strip()] = v.strip()
    csrc = os.path.join(ROOT, "paper_2211_07340_gb300", "csrc")
    src = (open(os.path.join(csrc, "sdtw_kernels.cuh"), "rb").read() +
           open(os.path.join(csrc, "haru_internal.h"), "rb").read())
    if vals.get("kernel_source_sha1") != hashlib.sha1(src).hexdigest():
        return None
    v = vals.get(f"traffic_bytes_per_step_{form}")
    return float(v) if v is not None else None


def dram_rate(traffic, cells: float, gcups: float) -> dict:
    """DRAM bytes per second of the sweep kernel (ncu traffic per batch over the
    batch's sweep time at the achieved rate), against the measured HBM copy peak:
    it shows the sweep is compute bound."""
    if traffic is None or not gcups:
        return {"dram_gbs": None}
    gbs = traffic / (cells / (gcups * 1e9)) / 1e9
    hbm = peaks_file().get("hbm_gbs")
    return {"dram_gbs": gbs, "hbm_peak_gbs": hbm, "dram_frac_of_hbm": gbs / hbm if hbm else None}


def alu_peak_gcups(sms: int, clock_mhz: float, form: str = "int16") -> float:
    """Peak cell rate of the sweep at the given SM clock, from pipe rates.

    int16: one packed cell pair takes 4 instructions, 2 on the half-rate
    min/DPX pipe (|q - r| by viaddmax_relu, vimin3) and 2 on the other
    half-rate integer pipe (vsub2, and vadd2 on rows that do not saturate;
    the saturating rows' viaddmin is charged to the first pipe and is left
    out of this minimum): 2 warp-instructions/clk/SM per pipe and 4
    issued/clk/SM both give 64 cells/clk/SM. FP32: 3 instructions per cell
    (the distance fma, 3-input min, add) at one warp-instruction per clock
    per scheduler:
    128 / 3 = 42.7 cells/clk/SM.
    """
    per_clk = 64.0 if form == "int16" else 128.0 / 3.0
    return sms * per_clk * clock_mhz * 1e6 / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 100):
        self.index = index
        self.period_ms = period_ms  # 0: no sampling
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        if self.period_ms <= 0:
            return self
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None,
                    "reasons": ["not sampled" if self.period_ms <= 0 else "nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "sm_min_mhz": min(sm) if sm else None,
                "below_1000_mhz": sum(1 for x in sm if x < 1000.0)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(ref, queries, target_s: float = 12.0, prec=None):
    """The oracle (as it stands) on the host cores over a bounded sample."""
    import oracle
    prec = oracle.PREC_I16 if prec is None else prec
    form = {oracle.PREC_I16: "int16", oracle.PREC_F64: "fp64", oracle.PREC_F32: "fp32",
            oracle.PREC_I32: "int16_acc32"}[prec]
    threads = os.cpu_count() or 1
    N = ref.shape[0]
    probe = queries.subset(np.arange(min(queries.nq, max(threads, 16))))
    t = time.perf_counter()
    oracle.batch(prec, ref, probe.events, probe.offsets, threads=threads)
    rate = probe.lengths.sum() * N / max(time.perf_counter() - t, 1e-6)
    lens = queries.lengths
    want = target_s * rate / N
    n = int(np.searchsorted(np.cumsum(lens), want)) + 1
    n = max(threads, min(queries.nq, n))
    sample = queries.subset(np.arange(n))
    t = time.perf_counter()
    oracle.batch(prec, ref, sample.events, sample.offsets, threads=threads)
    dt = time.perf_counter() - t
    cells = float(sample.lengths.sum()) * N
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "sample": f"first {n} of {queries.nq} queries ({cells / 1e9:.1f} G cells), {form} form, "
                      f"{dt:.1f} s"}


def cpu_baselines(ref, queries, target_s: float = 8.0):
    """The oracle's int16 form (the headline's) and its FP64 form, each on a
    bounded sample of the workload; value/sample are the int16 form's."""
    import oracle
    i16 = cpu_baseline(ref, queries, target_s, oracle.PREC_I16)
    f64 = cpu_baseline(ref, queries, target_s, oracle.PREC_F64)
    out = dict(i16)
    out["cpu_model"] = cpu_model()
    out["forms"] = {"int16": {k: i16[k] for k in ("value", "unit", "sample")},
                    "fp64": {k: f64[k] for k in ("value", "unit", "sample")}}
    return out


def ref_sweep(haru, args, dev):
    """Reference-length sweep: the same 512 x 250 query shape against the
    SARS-CoV-2-sized (59,796 columns), RFC1-sized (257,820) and 5 Mb (~10M)
    references, every form, with the oracle on the host cores beside each
    (the paper's speed-up-versus-reference-length experiment)."""
    import oracle
    import torch
    forms = [("int16", haru.HARU_INT16), ("fp32", haru.HARU_FP32), ("int16_acc32", haru.HARU_INT16_ACC32)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    rows = []
    for name, nq in (("sars_4096x250", 512), ("rfc1_512x250", None), ("long_512x250", None)):
        w = synth.workload(name, nq=nq)
        q = w.queries
        with haru.Context(dev.index) as ctx:
            ctx.ref_build(w.genome, w.model, w.k, scale_log2=6)
            N = ctx.ref_length
            cells = float(q.lengths.sum()) * N
            ev_d = torch.from_numpy(q.events).to(dev)
            off_d = torch.from_numpy(q.offsets.astype(np.int32)).to(dev)
            cost_d = torch.empty(q.nq, dtype=torch.float32, device=dev)
            col_d = torch.empty(q.nq, dtype=torch.int64, device=dev)
            row = {"workload": name, "reference_len": N, "queries": q.nq, "cells": cells}
            for fname, prec in forms:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                times = []
                for rep in range(args.warmup + args.sweep_reps):
                    with torch.cuda.stream(stream):
                        flush.zero_()
                        e0.record(stream)
                        ctx.sdtw_batch_device(prec, ev_d, off_d, cost_d, col_d, stream=stream.cuda_stream,
                                              asynchronous=True)
                        e1.record(stream)
                    stream.synchronize()
                    if ctx.last_status() != haru.HARU_OK:
                        raise haru.HaruError(ctx.last_status(), "batch")
                    if rep >= args.warmup:
                        times.append(e0.elapsed_time(e1))
                row[fname + "_gcups"] = cells / (statistics.median(times) / 1e3) / 1e9
                row[fname + "_segments"] = ctx.last_stats()["max_segments"]
        cpu = cpu_baseline(oracle.ref_levels(w.genome, w.model, w.k), q, target_s=args.sweep_cpu_s)
        row["cpu_int16_gcups"] = cpu["value"]
        row["cpu_sample"] = cpu["sample"]
        row["int16_over_cpu"] = row["int16_gcups"] / cpu["value"]
        rows.append(row)
    return {"metric": "sDTW GCUPS vs reference length, 512 x 250 raw-event queries, 1 GB300", "unit": "GCUPS",
            "data": "synthetic", "rows": rows, "reps": args.sweep_reps, "warmup": args.warmup,
            "l2": "flushed between batches (512 MiB write)", "cpu_cores": os.cpu_count()}


def run_signal(haru, args, ctx, dev, stream, flush, rank):
    """The raw-signal path: 8,192 reads of int16 ADC samples (adaptor, then
    pore-model levels under noise) through haru_sdtw_batch_signal (event
    detection, adaptor trim, 250-event queries, int16 sDTW), replayed from a
    CUDA graph; event detection alone is timed the same way, and its share of
    the step is reported."""
    import torch
    g, m, k, R = synth.signal_workload("sars_signal_uneven_8192", seed=111 + 1000 * rank)
    d_smp = torch.from_numpy(R.samples).to(dev)
    d_off = torch.from_numpy(R.offsets.astype(np.int32)).to(dev)
    cost = torch.empty(R.nreads, dtype=torch.float32, device=dev)
    col = torch.empty(R.nreads, dtype=torch.int64, device=dev)
    nev = torch.empty(R.nreads, dtype=torch.int32, device=dev)
    p = ctx.event_params()
    d_ev = torch.empty(R.nreads * p.max_events, dtype=torch.float32, device=dev)
    d_eoff = torch.empty(R.nreads + 1, dtype=torch.int32, device=dev)
    sh = stream.cuda_stream

    def full():
        ctx.sdtw_batch_signal_device(haru.HARU_INT16, d_smp, d_off, cost, col, nev, p, stream=sh, asynchronous=True)

    def detect():
        ctx.detect_events_device(d_smp, d_off, d_ev, d_eoff, p, stream=sh, asynchronous=True)

    tuned = None
    if not args.no_tune:  # the int16 launch shape, tuned on this batch's own queries
        with torch.cuda.stream(stream):
            detect()
        stream.synchronize()
        tuned = ctx.autotune(haru.HARU_INT16, d_ev, d_eoff, raw=True, on_device=True)
    out = {}
    for name, fn in (("step", full), ("detect", detect)):
        with torch.cuda.stream(stream):
            for _ in range(2):  # workspace growth outside capture
                fn()
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for rep in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                graph.replay()
                e1.record(stream)
            stream.synchronize()
            if rep >= args.warmup:
                times.append(e0.elapsed_time(e1))
        if ctx.last_status() != haru.HARU_OK:
            raise haru.HaruError(ctx.last_status(), "signal " + name)
        out[name] = float(np.mean(times))
    n_ev = nev.cpu().numpy().astype(np.int64)
    cells = float(n_ev.sum()) * ctx.ref_length
    return {"value": cells / (out["step"] / 1e3) / 1e9, "unit": "GCUPS", "ms_per_step": out["step"],
            "detect_ms": out["detect"], "detect_share": out["detect"] / out["step"],
            "reads": R.nreads, "samples_per_step": int(R.samples.shape[0]), "autotuned": tuned,
            "sample_bytes_per_step": int(R.samples.nbytes), "query_events_mean": float(n_ev.mean()),
            "form": "int16", "note": "raw int16 ADC samples -> two-window t-test events (windows 3/6, "
                                     "thresholds 1.40/9.00), 50 adaptor events trimmed, 250-event queries, "
                                     "z-score, int16 sDTW; CUDA graph, L2 flushed"}


def process_thp_off():
    """This process only: no transparent huge pages (PR_SET_THP_DISABLE, which
    its children inherit) and no MADV_HUGEPAGE on numpy's large arrays. On a
    kernel with 64 KB base pages a huge page is 512 MB, and faults on
    hugepage-advised memory compact (migrate) other pages of the process."""
    import ctypes
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        libc.prctl(41, 1, 0, 0, 0)  # PR_SET_THP_DISABLE
    except (OSError, AttributeError):
        pass
    try:
        from numpy._core import multiarray
        multiarray._set_madvise_hugepage(False)
    except (ImportError, AttributeError):
        pass


def pick_threshold(costs, on_target):
    """Decision threshold from a labelled held-out set: the cost cut with the
    fewest misclassified queries (accept iff cost <= T); among equally good
    cuts the first, placed midway between the two neighbouring costs."""
    order = np.argsort(costs, kind="stable")
    c, y = np.asarray(costs)[order], np.asarray(on_target)[order]
    n = c.shape[0]
    # accept the first k: errors = off-target among them + on-target after them
    off_before = np.concatenate([[0], np.cumsum(~y)])
    on_after = np.concatenate([[y.sum()], y.sum() - np.cumsum(y)])
    err = off_before + on_after
    k = int(np.argmin(err))
    if k == 0:
        return float(c[0]) - 1.0
    if k == n:
        return float(c[-1]) + 1.0
    return float(0.5 * (c[k - 1] + c[k]))


def run_serving(haru, args, local, w, threshold, channels, signal=False):
    """Serve a simulated flow cell in real time; latency from the delivery of
    the chunk that completes a read's 250-event prefix to its decision. With
    signal=True the flow cell delivers raw int16 samples (400 per 100 ms
    chunk) and the serving loop detects the events on the device; latency
    then starts at the chunk after which the prefix's 250 events were final."""
    span = args.serve_warm + args.serve_seconds
    if signal:
        chunks, q = synth.flowcell_signal_schedule(channels, span, seed=305)
    else:
        chunks, q = synth.flowcell_schedule(channels, span, seed=105)
    ctx = haru.Context(local, serve_precision=haru.HARU_INT16, threshold=threshold)
    ctx.ref_build(w.genome, w.model, w.k, scale_log2=6)
    results = []
    done = threading.Event()

    def poller():
        while not done.is_set():
            results.extend(ctx.stream_poll(8192, 2000))

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t_start = time.monotonic_ns()
    # The arrival time is read before the Python submit call: keep the
    # collector from pausing the replay thread between the two.
    import gc
    gc.collect()
    gc.disable()
    try:
        submit = ctx.stream_submit_signal if signal else ctx.stream_submit
        with ClockSampler(local, args.serve_clock_ms) as clk:
            late = synth.replay(chunks, lambda c, t: submit(c.read_id, c.channel, c.events, t, c.last))
    finally:
        gc.enable()
    nreads = q.nreads if signal else q.nq
    deadline = time.monotonic() + 30
    while len(results) < nreads and time.monotonic() < deadline:
        time.sleep(0.01)
    done.set()
    th.join()
    results.extend(ctx.stream_poll(8192, 0))
    st = ctx.stream_stats()
    ctx.close()
    warm_ns = t_start + int(args.serve_warm * 1e9)
    kept = [r for r in results if r.t_arrival_ns >= warm_ns]
    lat = np.array([(r.t_done_ns - r.t_arrival_ns) / 1e6 for r in kept])
    lib_lat = np.array([(r.t_done_ns - r.t_received_ns) / 1e6 for r in kept])
    dec = {r.read_id: r.decision for r in results}
    acc = float(np.mean([dec.get(i, 0) == int(q.on_target[i]) for i in range(nreads)])) if nreads else None
    N = 2 * (synth.SARS_COV_2_BASES - 5)
    cells = float(sum(r.events for r in results)) * N
    return {"channels": channels, "seconds": args.serve_seconds, "warmup_s": args.serve_warm, "reads": nreads,
            "input": "raw int16 samples, events detected on the device" if signal else "event chunks",
            "decided": len(results), "precision": "int16", "threshold_z": threshold,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "p999_ms": float(np.percentile(lat, 99.9)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None, "latency_samples": int(lat.size),
            "over_10ms": int(np.sum(lat > 10.0)),
            "library_p50_ms": float(np.percentile(lib_lat, 50)) if lib_lat.size else None,
            "library_p99_ms": float(np.percentile(lib_lat, 99)) if lib_lat.size else None,
            "library_max_ms": float(lib_lat.max()) if lib_lat.size else None,
            "decisions_per_s": len(results) / span, "gcups": cells / span / 1e9,
            "accept_eject_accuracy_vs_truth": acc, "batches": st["batches"], "max_batch": st["max_batch"],
            "max_concurrent_batches": st["max_concurrent"], "late_chunks": late, "clocks": clk.summary(),
            "stages": {"max_upload_ms": st["max_upload_ns"] / 1e6, "max_queue_ms": st["max_queue_ns"] / 1e6,
                       "max_gpu_ms": st["max_gpu_ns"] / 1e6, "max_gpu_exec_ms": st["max_gpu_exec_ns"] / 1e6,
                       "max_notice_ms": st["max_notice_ns"] / 1e6, "max_drain_ms": st["max_drain_ns"] / 1e6,
                       "max_cuda_calls_ms": {k: st["max_" + k + "_ns"] / 1e6 for k in
                                             ("upload_calls", "launch_inputs", "launch_path", "launch_results",
                                              "detect_calls")},
                       "over_10ms_upload": st["slow_upload"],
                       "over_10ms_queue": st["slow_queue"], "over_10ms_gpu": st["slow_gpu"],
                       "max_upload_sync_ms": st["max_upload_sync_ns"] / 1e6,
                       "max_worker_turn_gap_ms": st["max_turn_gap_ns"] / 1e6,
                       "worst_turn_ms": {k: st["worst_turn_" + k + "_ns"] / 1e6
                                         for k in ("complete", "upload", "detect", "launch", "wait")},
                       "worst_turn_switches": {"voluntary": st["worst_turn_voluntary_switches"],
                                               "involuntary": st["worst_turn_involuntary_switches"]},
                       "worst_turn_page_faults": {"minor": st["worst_turn_minor_faults"],
                                                  "major": st["worst_turn_major_faults"]},
                       "worst_turn_at_s": st["worst_turn_at_ns"] / 1e9, "turns_over_5ms": st["turns_over_5ms"],
                       "worker_minor_faults": st["worker_minor_faults"],
                       "worker_voluntary_switches": st["worker_voluntary_switches"],
                       "max_lock_wait_ms": st["max_lock_wait_ns"] / 1e6,
                       "max_upload_host_ms": st["max_upload_host_ns"] / 1e6},
            "latency_clock": "chunk delivery that completes the prefix -> decision available (CLOCK_MONOTONIC); "
                             "library_*: the library's receipt of that chunk -> decision available"}


def run_reference(args, rank: int):
    """The reference arm: the oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle
    w = synth.workload(WORKLOAD)
    ref = oracle.ref_levels(w.genome, w.model, w.k)
    q = w.queries
    threads = os.cpu_count() or 1
    N = ref.shape[0]
    # size each step so that the whole run takes about two minutes of CPU work
    per_step_s = max(0.5, min(8.0, 120.0 / max(1, args.steps + args.warmup)))
    probe = q.subset(np.arange(min(q.nq, max(threads, 16))))
    t = time.perf_counter()
    oracle.batch(oracle.PREC_I16, ref, probe.events, probe.offsets, threads=threads)
    rate = probe.lengths.sum() * N / max(time.perf_counter() - t, 1e-6)
    n = int(np.searchsorted(np.cumsum(q.lengths), per_step_s * rate / N)) + 1
    n = max(threads, min(q.nq, n))
    times, cells_per_step = [], 0.0
    for step in range(args.warmup + args.steps):
        sub = q.subset((np.arange(n) + step * n) % q.nq)
        t = time.perf_counter()
        oracle.batch(oracle.PREC_I16, ref, sub.events, sub.offsets, threads=threads)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            cells_per_step = float(sub.lengths.sum()) * N
    ms = 1e3 * sum(times) / len(times)
    value = cells_per_step / (ms / 1e3) / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i16", "data": "synthetic",
           "config": {"workload": WORKLOAD_DESC, "sample_queries_per_step": n, "form": "int16"},
           "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                            "sample": f"{n} of {q.nq} queries per step"},
           "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="haru", choices=["haru", "reference"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--nq", type=int, default=0, help="first nq queries only (profiling runs)")
    ap.add_argument("--units", type=int, default=0, help="work units target (0 = library default)")
    ap.add_argument("--fixed-len", type=int, default=0, help="profiling: every query this many events")
    ap.add_argument("--forms", default="int16,fp32,acc32,span,signal",
                    help="forms to time: int16, fp32, acc32 (int16 inputs, 32-bit accumulation), span (FP32 with "
                         "alignment start columns), signal (raw samples: event detection then int16 sDTW)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (use the library defaults)")
    ap.add_argument("--workload", default=WORKLOAD, help="sars_uneven_8192 (default) or long_512x250")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="measured seconds of the simulated flow-cell run, after the warm-up (0 = skip; N = 1 only)")
    ap.add_argument("--serve-warm", type=float, default=5.0, help="seconds of serving before the measured span")
    ap.add_argument("--serve-channels", type=int, default=512, help="event-chunk serving channels (0 = skip)")
    ap.add_argument("--serve-clock-ms", type=int, default=100,
                    help="nvidia-smi sampling period during the serving runs (0 = none)")
    ap.add_argument("--stress-channels", type=int, default=4096,
                    help="second serving run at this many channels, same length (0 = skip)")
    ap.add_argument("--signal-channels", type=int, default=512,
                    help="serving run on raw samples (event detection on the device) at this many channels, "
                         "same length (0 = skip)")
    ap.add_argument("--ref-sweep", action="store_true",
                    help="reference-length sweep (59,796 / 257,820 / 9,999,990 columns) instead of the benchmark")
    ap.add_argument("--sweep-reps", type=int, default=10)
    ap.add_argument("--sweep-cpu-s", type=float, default=3.0, help="oracle seconds per reference in --ref-sweep")
    ap.add_argument("--thp", choices=["on", "off"], default="on",
                    help="off: no transparent huge pages for this process (prctl) and none requested by numpy")
    args = ap.parse_args()
    if args.thp == "off":
        process_thp_off()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import paper_2211_07340_gb300 as haru

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    haru.build_library()
    if args.ref_sweep:
        if rank == 0:
            print(json.dumps(ref_sweep(haru, args, dev)), flush=True)
        return

    # Weak scaling: every rank aligns its own batch (independent seeds).
    w = synth.workload(args.workload, seed=(101 if args.workload == WORKLOAD else 104) + 1000 * rank)
    q = w.queries if not args.nq else w.queries.subset(np.arange(min(args.nq, w.queries.nq)))
    if args.fixed_len:
        g_off = synth.genome(synth.SARS_COV_2_BASES, synth.SEED_GENOME_OFF)
        q = synth.make_queries(np.full(q.nq, args.fixed_len), 0.5, 777, w.genome, g_off, w.model, w.k)
    cfg = haru.default_config()
    if args.tile:
        cfg.tile_cols = args.tile
    if args.warps:
        cfg.warps_per_cta = args.warps
    if args.units:
        cfg.units_target = args.units
    ctx = haru.Context(local, config=cfg)
    ctx.ref_build(w.genome, w.model, w.k, scale_log2=6)
    N = ctx.ref_length
    cells = float(q.lengths.sum()) * N
    ev_d = torch.from_numpy(q.events).to(dev)
    off_d = torch.from_numpy(q.offsets.astype(np.int32)).to(dev)
    cost_d = torch.empty(q.nq, dtype=torch.float32, device=dev)
    col_d = torch.empty(q.nq, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    launches = []  # own kernels per timed step of each form

    def kernels_per_step():
        # planner, query statistics (raw events), pack, the sweep and the
        # segment fix-up kernel
        return 5

    tuned = {}
    work = {}
    medians = {}

    def run_form(prec):
        sh = stream.cuda_stream
        if not args.no_tune:
            key = {haru.HARU_INT16: "int16", haru.HARU_FP32: "fp32", haru.HARU_INT16_ACC32: "int16_acc32"}[prec]
            tuned[key] = ctx.autotune(prec, ev_d, off_d, raw=True, on_device=True)
        with torch.cuda.stream(stream):
            for _ in range(2):  # allocate the context workspace outside capture
                ctx.sdtw_batch_device(prec, ev_d, off_d, cost_d, col_d, stream=sh, asynchronous=True,
                                      profile=True)
        stream.synchronize()
        graph = None
        if not args.no_graph:
            try:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=stream):
                    ctx.sdtw_batch_device(prec, ev_d, off_d, cost_d, col_d, stream=stream.cuda_stream,
                                          asynchronous=True, profile=True)
            except Exception as e:  # capture unsupported: direct launches
                print(f"graph capture failed ({e}); timing direct launches", file=sys.stderr)
                graph = None
        launches.append(kernels_per_step() * args.steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def step():
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                if graph is not None:
                    graph.replay()
                else:
                    ctx.sdtw_batch_device(prec, ev_d, off_d, cost_d, col_d, stream=stream.cuda_stream,
                                          asynchronous=True, profile=True)
                e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1), ctx.last_timing()[1]

        for _ in range(args.warmup):
            step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        step_ms, sweep_ms = [], []
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                a, b = step()
                step_ms.append(a)
                sweep_ms.append(b)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        st = ctx.last_status()
        if st != haru.HARU_OK:
            raise haru.HaruError(st, "batch")
        work[prec] = ctx.last_stats()  # items, groups, segments and fix-ups of the last replay
        medians[prec] = (float(np.median(step_ms)), float(np.median(sweep_ms)))
        return float(np.mean(step_ms)), float(np.mean(sweep_ms)), clk.summary(), graph is not None

    forms = args.forms.split(",")
    nan = float("nan")
    ms16 = sweep16 = ms32 = sweep32 = nan
    clocks = clocks32 = {}
    graphed = False
    msw = sweepw = nan
    capped16 = None
    if "int16" in forms:
        ms16, sweep16, clocks, graphed = run_form(haru.HARU_INT16)
        # queries whose int16 cost saturated at CAP (cost = integer cost / 2^6, exact)
        capped16 = int((np.rint(cost_d.cpu().numpy().astype(np.float64) * 64) >= haru.HARU_INT16_CAP).sum())
    if "fp32" in forms:
        ms32, sweep32, clocks32, _ = run_form(haru.HARU_FP32)
    if "acc32" in forms:
        msw, sweepw, _, _ = run_form(haru.HARU_INT16_ACC32)
    span_ms = nan
    if "span" in forms:  # FP32 with start columns, default launch shape, direct launches
        d = haru.default_config()
        ctx.configure(warps_per_cta=args.warps or d.warps_per_cta, tile_cols=args.tile or d.tile_cols,
                      units_target=args.units or d.units_target)
        start_d = torch.empty(q.nq, dtype=torch.int64, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        times = []
        for rep in range(args.warmup + max(3, args.steps // 4)):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                ctx.sdtw_batch_span_device(haru.HARU_FP32, ev_d, off_d, cost_d, col_d, start_d,
                                           stream=stream.cuda_stream, asynchronous=True)
                e1.record(stream)
            stream.synchronize()
            if rep >= args.warmup:
                times.append(e0.elapsed_time(e1))
        if ctx.last_status() != haru.HARU_OK:
            raise haru.HaruError(ctx.last_status(), "span batch")
        span_ms = float(np.mean(times))
        launches.append(5 * len(times))  # plan, statistics, pack, sweep, fix-up
    signal = None
    if "signal" in forms and args.workload == WORKLOAD:
        if "int16" in tuned:  # the starting shape; the leg tunes its own unless --no-tune
            ctx.configure(**tuned["int16"])
        signal = run_signal(haru, args, ctx, dev, stream, flush, rank)
        launches.append(8 * (args.steps + args.steps))  # detect, scan, compact + the batch path; detect-only graph
    if "int16" in tuned:  # the end-to-end leg runs the benchmark batch at its own tuned shape
        ctx.configure(**tuned["int16"])

    # End to end through the C ABI with host buffers: H2D of raw events and
    # offsets, the batch, D2H of costs and columns, every step.
    ev_h = torch.from_numpy(q.events).pin_memory()
    off_h = torch.from_numpy(q.offsets).pin_memory()
    cost_h = torch.empty(q.nq, dtype=torch.float32).pin_memory()
    col_h = torch.empty(q.nq, dtype=torch.int64).pin_memory()

    def e2e_step():
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t = time.perf_counter()
        rc = ctx.sdtw_batch_raw(haru.HARU_INT16, ev_h.data_ptr(), off_h.data_ptr(), q.nq, cost_h.data_ptr(),
                                col_h.data_ptr(), 0, haru.HARU_RAW)
        haru.check(rc, "e2e batch")
        return time.perf_counter() - t

    e2e_ms = nan
    if not args.no_e2e:
        for _ in range(args.warmup):
            e2e_step()
        e2e_s = [e2e_step() for _ in range(args.steps)]
        e2e_ms = 1e3 * float(np.mean(e2e_s))
        launches.append(kernels_per_step() * args.steps)

    if dist:
        t = torch.tensor([ms16, e2e_ms, ms32, msw, span_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms16, e2e_ms, ms32, msw, span_ms = (float(x) for x in t.tolist())
    total_cells = cells * world
    value = total_cells / (ms16 / 1e3) / 1e9
    value32 = total_cells / (ms32 / 1e3) / 1e9
    e2e_value = total_cells / (e2e_ms / 1e3) / 1e9

    probe16 = ctx.probe_peak(haru.HARU_INT16) / 1e9
    probe32 = ctx.probe_peak(haru.HARU_FP32) / 1e9
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    pk = peaks_file()
    max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = alu_peak_gcups(sms, max_mhz, "int16")
    peak32 = alu_peak_gcups(sms, max_mhz, "fp32")
    ach16 = cells / (sweep16 / 1e3) / 1e9
    ach32 = cells / (sweep32 / 1e3) / 1e9
    result = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms16,
        "median_ms_per_step": medians.get(haru.HARU_INT16, (None, None))[0],
        "median_sweep_ms": medians.get(haru.HARU_INT16, (None, None))[1],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if args.workload == WORKLOAD else LONG_DESC,
                   "global_batch": q.nq * world, "reference_len": N,
                   "cells_per_step": total_cells,
                   "form": "int16 (two queries per 32-bit lane, DPX min-plus)",
                   "cuda_graph": graphed, "l2": "flushed between steps (512 MiB write)",
                   "parallelism": f"dp{world} (independent batches per GPU)",
                   "autotuned": tuned},
        "roofline": {"bound": "alu", "kernel": "sdtw_kernel<INT16>", "achieved": ach16, "peak": peak,
                     "unit": "GCUPS", "frac": ach16 / peak, "traffic": profiled_traffic("int16"),
                     "traffic_unit": "bytes per batch (DRAM read+write, ncu at the default launch shape, "
                                     "profiles/sdtw_sweep_sars_uneven_8192.md)",
                     "peak_basis": f"{sms} SMs x 64 cells/clk/SM (4 instructions per packed cell pair, 2 on "
                                   f"each half-rate integer pipe) x {max_mhz:.0f} MHz max SM clock",
                     "frac_at_sampled_clock": (ach16 / alu_peak_gcups(sms, clocks["sm_mhz"], "int16"))
                     if clocks.get("sm_mhz") else None,
                     "peak_probe": probe16, "frac_of_probe": ach16 / probe16,
                     "peak_probe_basis": "haru_probe_peak: the int16 cell-pair instructions on independent "
                                         "chains, no shuffles/reference/tracking, same run",
                     "probe_ratio_int16_over_fp32": probe16 / probe32,
                     **dram_rate(profiled_traffic("int16"), cells, ach16)},
        "fp32": {"value": value32, "unit": "GCUPS", "ms_per_step": ms32,
                 "median_ms_per_step": medians.get(haru.HARU_FP32, (None, None))[0], "dtype": "f32",
                 "roofline": {"bound": "alu", "kernel": "sdtw_kernel<FP32>", "achieved": ach32, "peak": peak32,
                              "unit": "GCUPS", "frac": ach32 / peak32, "traffic": profiled_traffic("fp32"),
                              "peak_basis": f"{sms} SMs x 42.67 cells/clk/SM (3 issue slots per cell: distance fma, "
                                            f"3-input min, add at 4 warp-instr/clk/SM) x {max_mhz:.0f} MHz",
                              "peak_probe": probe32, "frac_of_probe": ach32 / probe32,
                              **dram_rate(profiled_traffic("fp32"), cells, ach32)},
                 "clocks": clocks32},
        "int16_acc32": ({"value": total_cells / (msw / 1e3) / 1e9, "unit": "GCUPS", "ms_per_step": msw,
                         "sweep_gcups": cells / (sweepw / 1e3) / 1e9,
                         "note": "int16 inputs with 32-bit accumulation (Section 4.3's PE): exact integer costs, "
                                 "computed exactly in FP32, one query per strip"}
                        if msw == msw else None),
        "fp32_start_columns": ({"value": total_cells / (span_ms / 1e3) / 1e9, "unit": "GCUPS", "ms_per_step": span_ms,
                                "note": "FP32 with each alignment's start column (haru_sdtw_batch_span): "
                                        "direct launches, default launch shape"}
                               if span_ms == span_ms else None),
        "signal": signal,
        "int16_over_fp32": value / value32 if value32 == value32 else None,
        "int16_capped_queries": capped16,
        "batch_work": {{haru.HARU_INT16: "int16", haru.HARU_FP32: "fp32", haru.HARU_INT16_ACC32: "int16_acc32"}[k]: v
                       for k, v in work.items()},
        "prep_ms_per_step": ms16 - sweep16,
        "e2e": {"value": e2e_value, "unit": "GCUPS", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(q.events.nbytes + q.offsets.nbytes),
                "d2h_bytes_per_step": int(q.nq * (4 + 8))},
        "clocks": clocks,
        "gpu_launches": int(sum(launches)),
    }
    # decision latency is a one-GPU property: the serving legs run at N = 1
    # only, so a scaling run holds its GPUs for the batch legs alone
    if args.serve_seconds > 0 and args.workload == WORKLOAD and world == 1:
        held = synth.workload("sars_heldout_1024", seed=103)
        hc, _ = ctx.sdtw_batch(haru.HARU_FP32, held.queries.events, held.queries.offsets)
        thr = pick_threshold(hc.astype(np.float64), held.queries.on_target)
        if args.serve_channels > 0:
            result["serving"] = run_serving(haru, args, local, w, thr, args.serve_channels)
        if args.stress_channels > 0:
            result["serving_stress"] = run_serving(haru, args, local, w, thr, args.stress_channels)
        if args.signal_channels > 0:
            # the threshold of raw-signal queries, fixed the same way on 1,024 held-out raw-signal reads
            _, _, _, hs = synth.signal_workload("sars_signal_heldout_1024")
            hsc, _, _ = ctx.sdtw_batch_signal(haru.HARU_FP32, hs.samples, hs.offsets)
            thr_sig = pick_threshold(hsc.astype(np.float64), hs.on_target)
            result["serving_signal"] = run_serving(haru, args, local, w, thr_sig, args.signal_channels, signal=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ref_levels = oracle.ref_levels(w.genome, w.model, w.k)
        result["cpu_baseline"] = cpu_baselines(ref_levels, q)
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
