"""Seeded synthetic inputs shaped like the paper's nanopore workloads.

The paper measures on real MinION/PromethION reads against the SARS-CoV-2 and
RFC1 references (Section 5.3, Table 2). Neither the reads nor the R9.4 pore
model exist here, so every workload is generated from fixed seeds:

* a genome of i.i.d. uniform bases (A=0, C=1, G=2, T=3);
* a 6-mer pore model of 4**k current levels drawn i.i.d. from N(90, 12) pA;
* reads that follow one strand of a genome through that pore model: every
  level is skipped with probability 0.1, otherwise emitted 1, 2 or 3 times
  (probabilities 4/7, 2/7, 1/7), and every emitted event gets N(0, 2) pA noise.

This module only simulates the sequencer. It holds none of the method's
arithmetic: no reference synthesis for the aligner, no z-score, no
quantisation and no dynamic programming. Both the CUDA path and the oracle
consume its raw outputs (bases, pore-model levels, raw event currents) and
apply the method themselves.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASES = "ACGT"

# Seeds of the workloads (one per independent random stream).
SEED_GENOME_ON = 1
SEED_GENOME_OFF = 2
SEED_PORE_MODEL = 3
SEED_GENOME_LONG = 4

SARS_COV_2_BASES = 29_903  # Table 2
RFC1_BASES = 128_915  # Table 2
LONG_BASES = 5_000_000


def genome(n_bases: int, seed: int) -> np.ndarray:
    """Uniform i.i.d. bases coded 0..3 (A, C, G, T)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 4, size=n_bases, dtype=np.uint8)


def pore_model(k: int = 6, seed: int = SEED_PORE_MODEL, mean: float = 90.0, sd: float = 12.0) -> np.ndarray:
    """A k-mer pore model: 4**k mean currents in pA, indexed by the base-4 code
    of the k-mer with its first base most significant."""
    rng = np.random.default_rng(seed)
    return rng.normal(mean, sd, size=4**k).astype(np.float32)


def _pore_currents(bases: np.ndarray, model: np.ndarray, k: int) -> np.ndarray:
    """Mean current while each k-mer of `bases` sits in the simulated pore."""
    n = bases.shape[0] - k + 1
    code = np.zeros(n, dtype=np.int64)
    for u in range(k):
        code = code * 4 + bases[u:u + n].astype(np.int64)
    return model[code]


def _reverse_complement(bases: np.ndarray) -> np.ndarray:
    return (3 - bases[::-1]).astype(np.uint8)


@dataclasses.dataclass
class Queries:
    """A batch of raw event queries in CSR form.

    events[offsets[q]:offsets[q+1]] are the raw currents (pA) of query q.
    truth_end is the index, in the forward-then-reverse strand concatenation
    of the source genome, of the level that produced the query's last event
    (meaningful for on-target queries only).
    """

    events: np.ndarray  # float32 [sum M]
    offsets: np.ndarray  # uint32 [nq + 1]
    on_target: np.ndarray  # bool [nq]
    truth_end: np.ndarray  # int64 [nq]

    @property
    def nq(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def query(self, q: int) -> np.ndarray:
        return self.events[self.offsets[q]:self.offsets[q + 1]]

    def subset(self, idx) -> "Queries":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.query(int(q)) for q in idx]
        lens = np.array([p.shape[0] for p in parts], dtype=np.int64)
        off = np.zeros(len(parts) + 1, dtype=np.uint32)
        off[1:] = np.cumsum(lens)
        ev = np.concatenate(parts).astype(np.float32) if parts else np.zeros(0, np.float32)
        return Queries(ev, off, self.on_target[idx].copy(), self.truth_end[idx].copy())


class _Strands:
    """Pore currents along both strands of one genome (the simulated molecule)."""

    def __init__(self, bases: np.ndarray, model: np.ndarray, k: int):
        self.fwd = _pore_currents(bases, model, k)
        self.rev = _pore_currents(_reverse_complement(bases), model, k)


def _emit(rng: np.random.Generator, levels: np.ndarray, start: int, m: int,
          p_skip: float, noise_sd: float) -> tuple[np.ndarray, int]:
    """Events of one read starting at level `start`; returns (events, index of
    the level that produced the last event)."""
    avail = levels.shape[0] - start
    span = min(avail, 4 * m + 64)
    lv = levels[start:start + span]
    skip = rng.random(span) < p_skip
    u = rng.random(span)
    dwell = np.where(u < 4.0 / 7.0, 1, np.where(u < 6.0 / 7.0, 2, 3))
    dwell[skip] = 0
    cum = np.cumsum(dwell)
    if cum[-1] < m:
        return np.zeros(0, np.float32), -1
    src = np.repeat(np.arange(span), dwell)[:m]
    ev = lv[src].astype(np.float64) + rng.normal(0.0, noise_sd, size=m)
    return ev.astype(np.float32), int(src[-1])


def make_queries(lengths, on_fraction: float, seed: int, genome_on: np.ndarray,
                 genome_off: np.ndarray, model: np.ndarray, k: int = 6,
                 p_skip: float = 0.1, noise_sd: float = 2.0, shuffle: bool = True) -> Queries:
    """Queries of the given event counts; the first round(on_fraction * nq)
    follow genome_on, the rest genome_off; order shuffled (seeded)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    nq = lengths.shape[0]
    rng = np.random.default_rng(seed)
    on = np.zeros(nq, dtype=bool)
    on[: int(round(on_fraction * nq))] = True
    if shuffle:
        on = on[rng.permutation(nq)]
    s_on = _Strands(genome_on, model, k)
    s_off = _Strands(genome_off, model, k) if (~on).any() else None
    parts, truth = [], np.full(nq, -1, dtype=np.int64)
    for q in range(nq):
        src = s_on if on[q] else s_off
        m = int(lengths[q])
        while True:
            strand = int(rng.integers(0, 2))
            levels = src.fwd if strand == 0 else src.rev
            hi = max(1, levels.shape[0] - 2 * m)
            start = int(rng.integers(0, hi))
            ev, last = _emit(rng, levels, start, m, p_skip, noise_sd)
            if ev.shape[0] == m:
                break
        parts.append(ev)
        if on[q]:
            truth[q] = strand * src.fwd.shape[0] + start + last
    off = np.zeros(nq + 1, dtype=np.uint32)
    off[1:] = np.cumsum(lengths)
    ev = np.concatenate(parts) if parts else np.zeros(0, np.float32)
    return Queries(ev.astype(np.float32), off, on, truth)


# --------------------------------------------------------- raw signal --
# The sequencer's raw output: integer ADC samples at 4 kHz. A level of the
# pore model holds for a dwell of several samples, each sample is the level
# plus Gaussian noise, and the current is digitised as
# adc = round(pA * ADC_DIGITISATION / ADC_RANGE_PA) - ADC_OFFSET (the R9.4
# MinION's digitisation and range; the offset is arbitrary). Before the
# genome, a read passes the sequencing adaptor: ADAPTOR_LEVELS levels drawn
# from their own distribution.
SAMPLE_RATE_HZ = 4000
ADC_DIGITISATION = 8192
ADC_RANGE_PA = 1402.1
ADC_OFFSET = 10
ADAPTOR_LEVELS = 50


@dataclasses.dataclass
class SignalReads:
    """A batch of raw-signal reads in CSR form.

    samples[offsets[r]:offsets[r+1]] are read r's int16 ADC samples.
    level_pos[i] is, for sample i, the index (in the forward-then-reverse
    strand concatenation of the read's source genome) of the pore-model level
    it was drawn from; -1 for adaptor samples and for off-target reads.
    """

    samples: np.ndarray  # int16 [sum n]
    offsets: np.ndarray  # uint32 [nreads + 1]
    on_target: np.ndarray  # bool [nreads]
    level_pos: np.ndarray  # int64 [sum n]

    @property
    def nreads(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def read(self, r: int) -> np.ndarray:
        return self.samples[self.offsets[r]:self.offsets[r + 1]]

    def subset(self, idx) -> "SignalReads":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.read(int(r)) for r in idx]
        pos = [self.level_pos[self.offsets[r]:self.offsets[r + 1]] for r in idx]
        off = np.zeros(len(parts) + 1, dtype=np.uint32)
        off[1:] = np.cumsum([p.shape[0] for p in parts])
        cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
        return SignalReads(cat(parts, np.int16), off, self.on_target[idx].copy(), cat(pos, np.int64))


def to_adc(pa: np.ndarray) -> np.ndarray:
    return (np.rint(pa * (ADC_DIGITISATION / ADC_RANGE_PA)) - ADC_OFFSET).astype(np.int16)


def _signal(rng: np.random.Generator, levels: np.ndarray, pos: np.ndarray, dwell_min: int, dwell_mean: float,
            noise_sd: float):
    """Samples of a run of levels: each level held for dwell_min + Geometric
    samples (mean dwell_mean), each sample the level plus N(0, noise_sd) pA."""
    p = 1.0 / max(1.0, dwell_mean - dwell_min + 1.0)
    dwell = dwell_min - 1 + rng.geometric(p, size=levels.shape[0])
    pa = np.repeat(levels.astype(np.float64), dwell) + rng.normal(0.0, noise_sd, size=int(dwell.sum()))
    return to_adc(pa), np.repeat(pos, dwell)


def make_signal_reads(n_levels, on_fraction: float, seed: int, genome_on: np.ndarray, genome_off: np.ndarray,
                      model: np.ndarray, k: int = 6, adaptor_levels: int = ADAPTOR_LEVELS, p_skip: float = 0.1,
                      dwell_min: int = 4, dwell_mean: float = 10.0, noise_sd: float = 2.5,
                      shuffle: bool = True) -> SignalReads:
    """Raw-signal reads: read r passes the adaptor (adaptor_levels levels
    ~ N(75, 8) pA), then follows a random strand and start of genome_on (the
    first round(on_fraction * n) reads, order shuffled) or genome_off through
    the pore model for n_levels[r] levels, each skipped with probability
    p_skip."""
    n_levels = np.asarray(n_levels, dtype=np.int64)
    nr = n_levels.shape[0]
    rng = np.random.default_rng(seed)
    on = np.zeros(nr, dtype=bool)
    on[: int(round(on_fraction * nr))] = True
    if shuffle:
        on = on[rng.permutation(nr)]
    s_on = _Strands(genome_on, model, k)
    s_off = _Strands(genome_off, model, k) if (~on).any() else None
    parts, poss = [], []
    for r in range(nr):
        src = s_on if on[r] else s_off
        m = int(n_levels[r])
        strand = int(rng.integers(0, 2))
        levels = src.fwd if strand == 0 else src.rev
        start = int(rng.integers(0, max(1, levels.shape[0] - m)))
        idx = np.arange(start, min(levels.shape[0], start + m))
        idx = idx[rng.random(idx.shape[0]) >= p_skip]
        ad = rng.normal(75.0, 8.0, size=adaptor_levels)
        a_smp, a_pos = _signal(rng, ad, np.full(adaptor_levels, -1, np.int64), dwell_min, dwell_mean, noise_sd)
        gpos = (strand * src.fwd.shape[0] + idx) if on[r] else np.full(idx.shape[0], -1, np.int64)
        g_smp, g_pos = _signal(rng, levels[idx], gpos.astype(np.int64), dwell_min, dwell_mean, noise_sd)
        parts.append(np.concatenate([a_smp, g_smp]))
        poss.append(np.concatenate([a_pos, g_pos]))
    off = np.zeros(nr + 1, dtype=np.uint32)
    off[1:] = np.cumsum([p.shape[0] for p in parts])
    smp = np.concatenate(parts).astype(np.int16) if parts else np.zeros(0, np.int16)
    pos = np.concatenate(poss).astype(np.int64) if poss else np.zeros(0, np.int64)
    return SignalReads(smp, off, on, pos)


def signal_workload(name: str, nreads: int | None = None, seed: int | None = None):
    """Raw-signal forms of the paper-shaped workloads: (genome, model, k, SignalReads).

    sars_signal_32x250      32 reads whose trimmed prefixes hold ~250 events
    sars_signal_uneven_8192 8,192 reads, genome levels uniform in [100, 500]
                            plus a margin, half on-target
    sars_signal_heldout_1024 1,024 reads as sars_signal_32x250 (threshold set)
    """
    model = pore_model(6)
    g_on = genome(SARS_COV_2_BASES, SEED_GENOME_ON)
    g_off = genome(SARS_COV_2_BASES, SEED_GENOME_OFF)
    table = {"sars_signal_32x250": (32, 110, None), "sars_signal_uneven_8192": (8192, 111, (100, 500)),
             "sars_signal_heldout_1024": (1024, 113, None)}
    n_default, s_default, span = table[name]
    n = n_default if nreads is None else nreads
    s = s_default if seed is None else seed
    if span is None:
        lv = np.full(n, 250, dtype=np.int64)
    else:
        lv = np.random.default_rng(s + 1000).integers(span[0], span[1] + 1, size=n)
    lv = lv + lv // 4 + 16  # levels beyond the prefix, so that skips and merges leave enough events
    return g_on, model, 6, make_signal_reads(lv, 0.5, s, g_on, g_off, model, 6)


def random_signal(n: int, seed: int, scale: float = 12.0, loc: float = 90.0) -> np.ndarray:
    """Generic Gaussian signal (pA) for small parity cases."""
    return np.random.default_rng(seed).normal(loc, scale, size=n).astype(np.float32)


def copy_query(signal: np.ndarray, start: int, m: int, seed: int, max_dwell: int = 1) -> np.ndarray:
    """A query copied exactly from signal[start:start+m]; with max_dwell > 1,
    every sample is repeated 1..max_dwell times (seeded) and the result cut
    back to length m. No noise is added."""
    seg = signal[start:start + m]
    if max_dwell <= 1:
        return seg.copy()
    rng = np.random.default_rng(seed)
    rep = rng.integers(1, max_dwell + 1, size=seg.shape[0])
    return np.repeat(seg, rep)[:m].copy()


@dataclasses.dataclass
class Workload:
    """A reference genome plus a query batch."""

    name: str
    genome: np.ndarray
    model: np.ndarray
    k: int
    queries: Queries


def reference_genome(n_bases: int = SARS_COV_2_BASES, seed: int = SEED_GENOME_ON) -> np.ndarray:
    return genome(n_bases, seed)


def workload(name: str, nq: int | None = None, seed: int | None = None) -> Workload:
    """The paper-shaped workloads, by name.

    sars_32x250      32 queries x 250 events, half on-target (SARS-CoV-2 size)
    sars_uneven_8192 8,192 queries, lengths uniform in [100, 500], half on-target
    sars_4096x250    4,096 queries x 250 events, half on-target
    sars_heldout_1024 1,024 queries x 250 events, half on-target (threshold set)
    long_512x250     512 queries x 250 events vs a 5,000,000-base genome
    rfc1_512x250     512 queries x 250 events vs a 128,915-base genome
    """
    model = pore_model(6)
    if name == "long_512x250":
        g_on = genome(LONG_BASES, SEED_GENOME_LONG)
    elif name == "rfc1_512x250":
        g_on = genome(RFC1_BASES, 5)
    else:
        g_on = genome(SARS_COV_2_BASES, SEED_GENOME_ON)
    g_off = genome(g_on.shape[0] if g_on.shape[0] <= RFC1_BASES else SARS_COV_2_BASES, SEED_GENOME_OFF)
    table = {
        "sars_32x250": (32, 100, None),
        "sars_uneven_8192": (8192, 101, (100, 500)),
        "sars_4096x250": (4096, 102, None),
        "sars_heldout_1024": (1024, 103, None),
        "long_512x250": (512, 104, None),
        "rfc1_512x250": (512, 106, None),
    }
    n_default, s_default, span = table[name]
    n = n_default if nq is None else nq
    s = s_default if seed is None else seed
    if span is None:
        lengths = np.full(n, 250, dtype=np.int64)
    else:
        lengths = np.random.default_rng(s + 1000).integers(span[0], span[1] + 1, size=n)
    q = make_queries(lengths, 0.5, s, g_on, g_off, model, 6)
    return Workload(name, g_on, model, 6, q)


@dataclasses.dataclass
class FlowCellChunk:
    t: float  # seconds since the start of the run
    read_id: int
    channel: int
    events: np.ndarray  # float32 raw event currents, or int16 ADC samples (raw-signal schedules)
    last: bool  # this chunk completes the decision prefix (raw-signal schedules: ends the read)


def flowcell_schedule(channels: int, duration_s: float, seed: int, prefix_events: int = 250,
                      events_per_s: float = 400.0, chunk_s: float = 0.1, idle_mean_s: float = 0.5,
                      accept_mean_s: float = 10.0, on_fraction: float = 0.2):
    """Open-loop arrival schedule of a simulated flow cell.

    Each channel idles for Exp(idle_mean_s), then a read starts and delivers
    its events in chunks every chunk_s seconds (events_per_s events per
    second). The chunk that holds event number `prefix_events` completes the
    decision prefix (flag `last`); later chunks of the read are not needed.
    A read on the target genome is assumed accepted and keeps the channel busy
    for Exp(accept_mean_s) more seconds; other reads are assumed ejected at
    once. Decisions are taken as instantaneous, so the schedule does not
    depend on the system under test.

    Returns (chunks sorted by time, Queries of every read's decision prefix
    indexed by read_id).
    """
    rng = np.random.default_rng(seed)
    model = pore_model(6)
    s_on = _Strands(genome(SARS_COV_2_BASES, SEED_GENOME_ON), model, 6)
    s_off = _Strands(genome(SARS_COV_2_BASES, SEED_GENOME_OFF), model, 6)
    per_chunk = int(round(events_per_s * chunk_s))
    n_chunks = -(-prefix_events // per_chunk)
    total = n_chunks * per_chunk
    chunks, prefixes, on_list, truth = [], [], [], []
    read_id = 0
    for ch in range(channels):
        t = rng.exponential(idle_mean_s)
        while t < duration_s:
            on = bool(rng.random() < on_fraction)
            src = s_on if on else s_off
            while True:
                strand = int(rng.integers(0, 2))
                levels = src.fwd if strand == 0 else src.rev
                start = int(rng.integers(0, levels.shape[0] - 2 * total))
                ev, last = _emit(rng, levels, start, total, 0.1, 2.0)
                if ev.shape[0] == total:
                    break
            for c in range(n_chunks):
                tc = t + (c + 1) * chunk_s
                chunks.append(FlowCellChunk(tc, read_id, ch, ev[c * per_chunk:(c + 1) * per_chunk],
                                            c == n_chunks - 1))
            prefixes.append(ev[:prefix_events])
            on_list.append(on)
            truth.append(-1)
            t_decide = t + n_chunks * chunk_s
            t = t_decide + (rng.exponential(accept_mean_s) if on else 0.0) + rng.exponential(idle_mean_s)
            read_id += 1
    chunks.sort(key=lambda c: (c.t, c.channel))
    off = np.arange(read_id + 1, dtype=np.uint32) * prefix_events
    ev = np.concatenate(prefixes).astype(np.float32) if prefixes else np.zeros(0, np.float32)
    q = Queries(ev, off, np.array(on_list, dtype=bool), np.array(truth, dtype=np.int64))
    return chunks, q


def flowcell_signal_schedule(channels: int, duration_s: float, seed: int, prefix_events: int = 250,
                             chunk_s: float = 0.1, idle_mean_s: float = 0.5, accept_mean_s: float = 10.0,
                             on_fraction: float = 0.2):
    """Open-loop arrival schedule of a simulated flow cell that delivers raw
    samples: as flowcell_schedule, but every read is a raw int16 ADC signal
    (the adaptor, then ~1.25 x prefix_events + 16 pore-model levels; see
    make_signal_reads) delivered in chunks of SAMPLE_RATE_HZ * chunk_s
    samples; the read's last chunk carries `last`. A read on the target
    genome keeps the channel busy for Exp(accept_mean_s) more seconds after
    its signal ends; other reads free it at once.

    Returns (chunks sorted by time, SignalReads of every read's whole
    signal indexed by read_id)."""
    rng = np.random.default_rng(seed)
    model = pore_model(6)
    g_on = genome(SARS_COV_2_BASES, SEED_GENOME_ON)
    g_off = genome(SARS_COV_2_BASES, SEED_GENOME_OFF)
    s_on, s_off = _Strands(g_on, model, 6), _Strands(g_off, model, 6)
    per_chunk = int(round(SAMPLE_RATE_HZ * chunk_s))
    n_levels = prefix_events + prefix_events // 4 + 16
    chunks, parts, poss, on_list = [], [], [], []
    read_id = 0
    for ch in range(channels):
        t = rng.exponential(idle_mean_s)
        while t < duration_s:
            on = bool(rng.random() < on_fraction)
            src = s_on if on else s_off
            strand = int(rng.integers(0, 2))
            levels = src.fwd if strand == 0 else src.rev
            start = int(rng.integers(0, levels.shape[0] - n_levels))
            idx = np.arange(start, start + n_levels)
            idx = idx[rng.random(idx.shape[0]) >= 0.1]
            ad = rng.normal(75.0, 8.0, size=ADAPTOR_LEVELS)
            a_smp, a_pos = _signal(rng, ad, np.full(ADAPTOR_LEVELS, -1, np.int64), 4, 10.0, 2.5)
            gpos = (strand * src.fwd.shape[0] + idx) if on else np.full(idx.shape[0], -1, np.int64)
            g_smp, g_pos = _signal(rng, levels[idx], gpos.astype(np.int64), 4, 10.0, 2.5)
            smp = np.concatenate([a_smp, g_smp])
            n_chunks = -(-smp.shape[0] // per_chunk)
            for c in range(n_chunks):
                chunks.append(FlowCellChunk(t + (c + 1) * chunk_s, read_id, ch, smp[c * per_chunk:(c + 1) * per_chunk],
                                            c == n_chunks - 1))
            parts.append(smp)
            poss.append(np.concatenate([a_pos, g_pos]))
            on_list.append(on)
            t = t + n_chunks * chunk_s + (rng.exponential(accept_mean_s) if on else 0.0) + rng.exponential(idle_mean_s)
            read_id += 1
    chunks.sort(key=lambda c: (c.t, c.channel))
    off = np.zeros(read_id + 1, dtype=np.uint32)
    off[1:] = np.cumsum([p.shape[0] for p in parts])
    smp = np.concatenate(parts).astype(np.int16) if parts else np.zeros(0, np.int16)
    pos = np.concatenate(poss).astype(np.int64) if poss else np.zeros(0, np.int64)
    return chunks, SignalReads(smp, off, np.array(on_list, dtype=bool), pos)


def replay(chunks, submit, speed: float = 1.0, stop=None):
    """Deliver a flow-cell schedule in (scaled) wall-clock time.

    submit(chunk, t_arrival_ns) is called for every chunk at start +
    chunk.t / speed, with the CLOCK_MONOTONIC time of delivery; it returns a
    status code, and a nonzero code other than busy (-4) stops the replay.
    Busy chunks are retried after 200 microseconds. Returns the number of
    chunks delivered late by more than 5 ms (a measure of replay fidelity).
    """
    import time
    t0 = time.monotonic_ns()
    late = 0
    for c in chunks:
        due = t0 + int(c.t / speed * 1e9)
        now = time.monotonic_ns()
        if due > now:
            time.sleep((due - now) / 1e9)
        elif now - due > 5_000_000:
            late += 1
        while True:
            rc = submit(c, time.monotonic_ns())
            if rc != -4:
                break
            time.sleep(0.0002)
        if rc != 0:
            raise RuntimeError(f"submit failed with {rc}")
        if stop is not None and stop():
            break
    return late
