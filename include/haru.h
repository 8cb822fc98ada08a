/* libharu: GB300-native subsequence DTW for signal-alignment Read Until.
 *
 * The method is HARU's (arXiv 2211.07340): a z-score-normalised query of
 * nanopore events is aligned against a reference signal built from a k-mer
 * pore model over both strands of a genome (Section 4.1); the alignment is
 * subsequence dynamic time warping, Eq. 1 of Section 2.3:
 *
 *   gamma(i, j) = |x_i - y_j| + min(gamma(i-1, j), gamma(i-1, j-1), gamma(i, j-1))
 *   gamma(i, 0) = inf for i >= 1,   gamma(0, j) = 0 for j >= 0 (free start)
 *
 * and the answer per query is the minimum of the last row and the first
 * column that reaches it (Algorithm 1's final scan, Algorithm 2's
 * per-column update; ties go to the smallest column). Columns are 0-based
 * indices into the reference as loaded (forward strand first when built by
 * haru_ref_build).
 *
 * Three arithmetic forms:
 *   HARU_FP32  plain float: delta = |x - y| rounded once, sums rounded once.
 *   HARU_INT16 the paper's fixed-point idea (Sections 4.1 and 4.3): samples
 *              are quantised to q = clamp(round_half_even(z * 2^k), -2047,
 *              2047) and costs saturate at HARU_INT16_CAP, which also stands
 *              for infinity; the reported cost is the integer cost / 2^k.
 *   HARU_INT16_ACC32 the same quantised samples with wide (32-bit)
 *              accumulation, the PE of Section 4.3: the exact integer cost,
 *              never saturated (every cost of a query of <= 512 events is
 *              below 2^31), reported as integer / 2^k. Batch calls only.
 *
 * Conventions for every entry point:
 *   - return 0 (HARU_OK) or a negative HARU_E* code; nothing aborts or traps;
 *   - the caller owns every buffer it passes; the library copies what it
 *     keeps (the reference) before returning and keeps no caller pointer;
 *   - a context is used by one host thread at a time (the serving calls are
 *     the exception: haru_stream_submit and haru_stream_poll may be called
 *     from different threads);
 *   - the first CUDA error seen by a context is sticky: later calls return
 *     HARU_ECUDA until the context is destroyed.
 */
#ifndef HARU_H_
#define HARU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HARU_OK 0
#define HARU_EINVAL (-1)    /* bad argument: empty/NaN/Inf input, M = 0, M > N, M too long, bad scale */
#define HARU_ENOREF (-2)    /* no reference loaded */
#define HARU_ENOMEM (-3)    /* device or host allocation failed, or admission budget exceeded */
#define HARU_EBUSY (-4)     /* serving queue full: poll, then retry; or a reference change on a serving context */
#define HARU_ETIMEDOUT (-5) /* a bounded wait (device or host) gave up */
#define HARU_ECUDA (-6)     /* a CUDA runtime error (sticky per context) */

#define HARU_FP32 0
#define HARU_INT16 1
#define HARU_INT16_ACC32 2

#define HARU_INT16_QMAX 2047
#define HARU_INT16_CAP 28673 /* 32767 - 2 * HARU_INT16_QMAX */
#define HARU_MAX_QUERY 512   /* longest query (events) one warp strip holds: 32 lanes x 16 rows */

/* haru_sdtw_batch flags */
#define HARU_ON_DEVICE 1u /* events/offsets/out_* are device pointers, ordered on `stream` */
#define HARU_RAW 2u       /* events are raw currents: z-score each query on the device first */
#define HARU_ASYNC 4u     /* HARU_ON_DEVICE only: return after enqueueing; read the status later
                             with haru_last_status() once the stream has been synchronised */
#define HARU_PROFILE 8u   /* record CUDA events around the preparation kernels and the sweep kernel of
                             this batch (also inside a captured CUDA graph); read with haru_last_timing() */

typedef struct haru_ctx haru_ctx;

/* Event detection on raw samples (see "Raw signal" below for the method). */
#define HARU_MAX_READ_SAMPLES 16384 /* samples of one read's signal, at most */

typedef struct {
  int window_short;          /* samples per window of the short t-test, 2..16 (default 3) */
  int window_long;           /* of the long t-test, window_short..16 (default 6) */
  int threshold_short_centi; /* t threshold of the short window in hundredths, 1..10000 (default 140) */
  int threshold_long_centi;  /* of the long window (default 900) */
  uint32_t trim_events;      /* leading events dropped: the read adaptor (default 50, Section 4.1) */
  uint32_t max_events;       /* events kept after the trim: the query prefix, 1..HARU_MAX_QUERY (default 250) */
} haru_event_params;

typedef struct {
  int warps_per_cta;        /* warps (queries or query pairs) sharing one reference tile stream: 2, 4, 8
                               or 12 (start-column batches run at most 8); other values = 8 */
  int tile_cols;            /* reference columns per shared-memory tile, 2048..16384; 0 = auto */
  int ctas_per_sm;          /* persistent CTAs per SM; 0 = as many as fit */
  uint32_t wait_limit;      /* longest single device wait, microseconds, before HARU_ETIMEDOUT; 0 = 2 s;
                               values below 1000 act as 1000 (a timed-out CTA's drain of its copies in
                               flight shares the limit and must outlast a tile copy) */
  /* serving */
  float threshold;          /* accept iff cost <= threshold (z units; int16 compares floor(threshold * 2^k)) */
  int serve_precision;      /* HARU_FP32 or HARU_INT16 */
  size_t serve_budget_bytes;/* device memory for in-flight serving requests; 0 = 64 MiB */
  uint32_t serve_max_batch; /* most requests launched together; 0 = 1024; at most the slots
                               serve_budget_bytes gives (a batch holds admitted reads only) */
  uint32_t serve_prefix;    /* events per decision prefix; 0 = 250 (Section 4.1) */
  int units_target;         /* work units (query x reference segment) a batch is cut into, at least;
                               0 = 4 x SMs x warps_per_cta; 1 = never split the reference */
  int stack_short;          /* queries of at most 256 events stacked two to a warp strip (lanes 0-15
                               and 16-31), doubling the rows each lane sweeps: more throughput, but
                               each strip takes longer. 0 (default) = in batches of at least
                               units_target queries (or 4 x SMs x warps_per_cta when that is 0),
                               or whose stacked items cut into reference segments still make that
                               many work units (long references); 1 = always; -1 = never */
  int serve_spin_us;        /* serving: microseconds the worker keeps polling after its last piece of
                               work before it sleeps (a sleeping thread can be woken late on a busy
                               host); 0 = 2000, negative = never poll idle */
  haru_event_params serve_events; /* serving raw samples (haru_stream_submit_signal): the event detector's
                               parameters; max_events is replaced by serve_prefix; all zero = defaults */
} haru_config;

/* Fill *cfg with defaults. Returns HARU_OK, or HARU_EINVAL if cfg is NULL. */
int haru_config_default(haru_config *cfg);

/* Create a context on CUDA device `device` (the device is made current for
 * every later call on this context). cfg may be NULL (defaults). */
int haru_create(haru_ctx **out, int device, const haru_config *cfg);

/* Replace the context's configuration for later batches. The serving fields
 * take effect only before the first haru_stream_submit. Errors: HARU_EINVAL. */
int haru_configure(haru_ctx *ctx, const haru_config *cfg);

/* Copy the context's current configuration (e.g. after haru_autotune). */
int haru_get_config(haru_ctx *ctx, haru_config *cfg);

/* Release the context, its device memory and its serving thread. NULL is a no-op. */
void haru_destroy(haru_ctx *ctx);

/* Load a reference signal of n levels (host pointer, float32).
 * normalize = 1: levels are raw currents; they are z-scored on the device
 *   (Section 4.1; population sigma, double-precision sums).
 * normalize = 0: levels are already z-scores.
 * scale_log2 = k in [1, 7]: int16 quantisation scale 2^k (Section 4.3 uses 2^5).
 * Replaces any previous reference; a failed call leaves the previous one in
 * place. A context that serves (after its first haru_stream_submit or
 * haru_stream_submit_signal) keeps the reference its serving loop started
 * with until haru_destroy: HARU_EBUSY (serve another reference from another
 * context). Errors: HARU_EINVAL (n = 0, non-finite value, zero spread, bad
 * k), HARU_ENOMEM, HARU_EBUSY, HARU_ECUDA. */
int haru_ref_load(haru_ctx *ctx, const float *levels, size_t n, int normalize, int scale_log2);

/* Build the reference on the device from a genome (Sections 2.2 and 4.1):
 * bases[0..n_bases) in {0,1,2,3} = A,C,G,T; kmer_levels[4^k] the pore model
 * indexed by the base-4 k-mer code (first base most significant). The signal
 * is the forward strand's k-mer levels followed by the reverse complement's,
 * 2 * (n_bases - k + 1) values, then z-scored and quantised as in
 * haru_ref_load (HARU_EBUSY on a serving context, as there). Host pointers.
 * Errors: HARU_EINVAL (k not in 1..12, genome shorter than k, base > 3),
 * HARU_ENOMEM, HARU_EBUSY, HARU_ECUDA. */
int haru_ref_build(haru_ctx *ctx, const uint8_t *bases, size_t n_bases, const float *kmer_levels, int k,
                   int scale_log2);

/* Length of the loaded reference (0 if none). */
size_t haru_ref_length(const haru_ctx *ctx);

/* Copy the loaded reference back: z-scores (float, n values) and/or the
 * int16 codes (n values). Either pointer may be NULL. Host pointers. */
int haru_ref_read(haru_ctx *ctx, float *z, int16_t *q, size_t n);

/* Align a batch of queries against the loaded reference (the hot path).
 * events[offsets[q] .. offsets[q+1]) are query q's events, float32;
 * offsets has nq + 1 entries, offsets[0] = 0, non-decreasing.
 * precision: HARU_FP32, HARU_INT16 or HARU_INT16_ACC32.
 * out_cost[q]: the minimum last-row cost (float; int16: integer cost / 2^k,
 *   exact). out_col[q]: its first (smallest) 0-based reference column.
 * flags: HARU_ON_DEVICE (device pointers, work ordered on `stream`, a
 *   cudaStream_t cast to uintptr_t, 0 = the context's stream), HARU_RAW (z-score
 *   each query on the device, Section 4.1), HARU_ASYNC.
 * Without HARU_ASYNC the call returns after the results are in out_*.
 * Every query needs 1 <= M <= min(N, HARU_MAX_QUERY). nq = 0 is a no-op.
 * Errors: HARU_EINVAL, HARU_ENOREF, HARU_ENOMEM, HARU_ETIMEDOUT, HARU_ECUDA. */
int haru_sdtw_batch(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
                    float *out_cost, int64_t *out_col, uintptr_t stream, uint32_t flags);

/* haru_sdtw_batch that also reports where each alignment starts: out_start[q]
 * (int64, nq) is the 0-based reference column at which the chosen warping
 * path of query q enters its first row, so the query maps to reference
 * columns [out_start[q], out_col[q]]. The paper drops backtracking
 * (Section 4.3); here the start column is carried forward through the DP:
 * every cell takes the start of its up neighbour if that is a minimum
 * predecessor, else of its diagonal one, else of its left one (a fixed
 * preference where costs tie). Costs and end columns equal haru_sdtw_batch's.
 * precision: HARU_FP32 or HARU_INT16_ACC32 (the packed int16 form has no room
 * for a start column per cell). Layout, flags, ownership and errors as in
 * haru_sdtw_batch; out_start is a host pointer, or a device pointer with
 * HARU_ON_DEVICE. About 2-2.5x the time of haru_sdtw_batch (more work per
 * cell); sweeps are cut into verified reference segments as there, a segment
 * being kept only if both its costs and its start columns match. */
int haru_sdtw_batch_span(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
                         float *out_cost, int64_t *out_col, int64_t *out_start, uintptr_t stream, uint32_t flags);

/* ---- Raw signal: event detection on the device ---------------------------
 * Section 4.1's pre-processing (Section 5.1: event detection, prefix
 * trimming, normalisation) on the GPU: raw ADC samples in, events out, and
 * the sDTW path run on them. The detector is the two-window t-test of the
 * R9.4 tool chain Section 5.2 names (its parameters are not printed in the
 * paper; the defaults below are this library's reading of them). At sample
 * position i, the w samples before i and the w samples from i on give
 *   t^2 = w (B - A)^2 / max(1, w (QA + QB) - A^2 - B^2)
 * for their sums A, B and sums of squares QA, QB: the squared difference of
 * the window means over (v1 + v2) / w with population variances; defined for
 * w <= i <= n - w. Statistics are compared exactly (as rationals). A peak of
 * a window is a position whose t exceeds the window's threshold, is strictly
 * greater than the defined t of the w positions before it and at least that
 * of the w positions after it. Events start at the long window's peaks and at
 * the short window's peaks that have no long-window peak within window_short
 * positions; event e spans samples [b_e, b_{e+1}) (b_0 = 0, the last b = n)
 * and its value is its mean, (float)((double) sum / length). A read's query is
 * events [trim_events, trim_events + max_events): the adaptor's events are
 * dropped and the decision prefix kept. The event values are in ADC units;
 * the sDTW path z-scores each query (HARU_RAW behaviour). */
/* Fill *p with the defaults. Returns HARU_OK, or HARU_EINVAL if p is NULL. */
int haru_event_params_default(haru_event_params *p);

/* Detect the events of nreads reads. samples[sample_offsets[r] ..
 * sample_offsets[r+1]) are read r's int16 ADC samples (at most
 * HARU_MAX_READ_SAMPLES each); sample_offsets has nreads + 1 entries,
 * non-decreasing from 0. params may be NULL (defaults). Output: read r's
 * query events in events[event_offsets[r] .. event_offsets[r+1]) (float, ADC
 * units); event_offsets has nreads + 1 entries; events must hold nreads *
 * max_events floats. A read with fewer than trim_events + 1 events gets an
 * empty query. flags: HARU_ON_DEVICE (all four arrays are device pointers,
 * ordered on `stream`), HARU_ASYNC (with HARU_ON_DEVICE). Errors: HARU_EINVAL
 * (bad parameters, offsets or read length), HARU_ENOMEM, HARU_ECUDA. */
int haru_detect_events(haru_ctx *ctx, const int16_t *samples, const uint32_t *sample_offsets, uint32_t nreads,
                       const haru_event_params *params, float *events, uint32_t *event_offsets, uintptr_t stream,
                       uint32_t flags);

/* The whole path from raw signal to alignment: haru_detect_events, then
 * haru_sdtw_batch on each read's query (z-scored on the device), in one
 * stream-ordered sequence. Layout of samples/sample_offsets and params as in
 * haru_detect_events; precision, out_cost, out_col, stream and flags
 * (HARU_ON_DEVICE, HARU_ASYNC, HARU_PROFILE) as in haru_sdtw_batch.
 * out_events (may be NULL): the query length used per read (uint32, nreads).
 * Every read must give a query of 2 or more events with a nonzero spread,
 * else the batch returns HARU_EINVAL. Errors: as haru_sdtw_batch. */
int haru_sdtw_batch_signal(haru_ctx *ctx, int precision, const int16_t *samples, const uint32_t *sample_offsets,
                           uint32_t nreads, const haru_event_params *params, float *out_cost, int64_t *out_col,
                           uint32_t *out_events, uintptr_t stream, uint32_t flags);

/* ---- Serving: continuous batching of Read Until decisions -----------------
 * A persistent request loop inside the context (a worker thread) takes the
 * event chunks of reads as a flow cell delivers them, keeps each admitted
 * read's events in a device slot, and once a read's decision prefix is
 * complete (serve_prefix events, Section 4.1 uses 250) batches it with the
 * other complete reads into the sDTW path. Batches launch while earlier ones
 * are still on the GPU (several in flight on separate streams). Reads are
 * admitted to device slots as the memory budget (serve_budget_bytes) allows;
 * the rest wait on the host in arrival order. Each result carries the
 * decision: accept (keep sequencing) iff cost <= threshold, else eject. */
typedef struct {
  uint64_t read_id;
  uint32_t channel;
  int32_t decision;       /* 1 accept, 0 eject */
  float cost;             /* z units (int16: integer cost / 2^k) */
  int32_t status;         /* HARU_OK, or why no alignment was made (HARU_EINVAL: prefix too short/flat) */
  int64_t end_col;        /* 0-based reference column of the alignment end */
  uint32_t events;        /* prefix length used */
  uint32_t pad;
  uint64_t t_arrival_ns;  /* as submitted with the chunk that completed the prefix */
  uint64_t t_done_ns;     /* when the decision was ready (CLOCK_MONOTONIC ns) */
  uint64_t t_received_ns; /* when the library received that chunk (CLOCK_MONOTONIC ns): t_done_ns -
                             t_received_ns is the library's own share of the latency */
} haru_result;

/* Append a chunk of raw event currents (host pointer, n floats) to read
 * read_id on channel. t_arrival_ns is the caller's CLOCK_MONOTONIC time of
 * delivery (it starts the decision-latency clock when this chunk completes
 * the prefix). last_chunk = 1 ends the read: a shorter prefix is decided as
 * is. Chunks after the prefix is complete are ignored, and so are the
 * events of a chunk beyond the first serve_prefix (no read can use more).
 * The call copies the events and hands them to the serving thread without
 * waiting on it (a
 * lock-free list), so a submitter is never held up by the serving loop and
 * vice versa. The first call starts the serving thread. Errors: HARU_EINVAL,
 * HARU_ENOREF, HARU_ENOMEM, HARU_EBUSY (too many events waiting on the host:
 * poll, then retry), HARU_ECUDA. */
int haru_stream_submit(haru_ctx *ctx, uint64_t read_id, uint32_t channel, const float *events, uint32_t n,
                       uint64_t t_arrival_ns, int last_chunk);

/* Append a chunk of raw int16 ADC samples (host pointer, n of them) to read
 * read_id on channel: haru_stream_submit for a flow cell that delivers its
 * raw signal. The read's samples go to a device slot (at most
 * HARU_MAX_READ_SAMPLES are kept; a read that reaches them counts as ended).
 * After each upload the serving loop runs the event detector (see "Raw
 * signal": adaptor trim, serve_events parameters) over every read with new
 * samples and counts its query events whose closing boundary is final: at
 * least window_short + 2 window_long samples before the newest sample, where
 * later samples can no longer move it. The decision prefix is complete once
 * serve_prefix such events exist, or when the read ends (last_chunk = 1; its
 * query is then every event after the trim). Either way the query equals
 * what haru_sdtw_batch_signal computes on the read's whole signal. The
 * latency clock starts at t_arrival_ns of the newest chunk the completing
 * detection covered. A context serves either events or samples: whichever
 * submit call comes first fixes it, and the other returns HARU_EINVAL.
 * Errors as haru_stream_submit. */
int haru_stream_submit_signal(haru_ctx *ctx, uint64_t read_id, uint32_t channel, const int16_t *samples, uint32_t n,
                              uint64_t t_arrival_ns, int last_chunk);

/* Collect up to max finished decisions into out (host array), waiting up to
 * timeout_us microseconds for the first. *n_out = how many were written
 * (0 on timeout, which returns HARU_OK). */
int haru_stream_poll(haru_ctx *ctx, haru_result *out, uint32_t max, uint32_t *n_out, uint32_t timeout_us);

typedef struct {
  uint64_t reads_submitted;   /* reads seen */
  uint64_t reads_decided;     /* results produced */
  uint64_t reads_waiting;     /* complete or partial reads not yet admitted to a device slot */
  uint64_t reads_in_flight;   /* admitted, not yet decided */
  uint64_t batches;           /* batches launched */
  uint64_t max_batch;         /* largest batch launched */
  uint64_t max_concurrent;    /* most batches on the GPU at once */
  uint64_t slots;             /* device slots the budget allows */
  /* where decided reads spent their time (for latency diagnosis), per stage
   * the longest time seen and how many reads took over 10 ms there:
   * upload = the completing chunk received -> all events on the device and
   * the read queued; queue = queued -> launched in a batch; gpu = launched
   * -> the batch's completion seen by the worker */
  uint64_t max_upload_ns, max_queue_ns, max_gpu_ns;
  uint64_t slow_upload, slow_queue, slow_gpu;
  /* the longest wait for an upload transfer to finish, and the longest gap
   * between two turns of the worker loop */
  uint64_t max_upload_sync_ns, max_turn_gap_ns;
  /* the slowest turn: time in its complete / upload / launch / idle-wait
   * parts, and the worker thread's voluntary and involuntary context
   * switches during it (Linux; 0 elsewhere); its detection part and page
   * faults follow at the end */
  uint64_t worst_turn_complete_ns, worst_turn_upload_ns, worst_turn_launch_ns, worst_turn_wait_ns;
  uint64_t worst_turn_voluntary_switches, worst_turn_involuntary_switches;
  /* the GPU stage split: the longest device execution of a batch (CUDA
   * events from its first operation to its last), and the longest remainder
   * of a read's GPU stage (queueing on the device and the worker noticing
   * completion) */
  uint64_t max_gpu_exec_ns, max_notice_ns;
  /* the longest time the worker spent taking submitted chunks into its reads
   * (part of the upload stage) */
  uint64_t max_drain_ns;
  /* the longest time spent inside one group of CUDA calls of the worker: the
   * upload (staged copy, scatter launch, event), and a batch launch's input
   * copies and gather, its device path (planner to fix-up) and its result
   * copies and completion event */
  uint64_t max_upload_calls_ns, max_launch_inputs_ns, max_launch_path_ns, max_launch_results_ns;
  /* raw-sample serving: the longest group of detection CUDA calls (inputs,
   * launch, count copy, event), and the slowest turn's detection part; then
   * the worker thread's minor and major page faults during that turn */
  uint64_t max_detect_calls_ns, worst_turn_detect_ns;
  uint64_t worst_turn_minor_faults, worst_turn_major_faults;
  /* when the slowest turn began (ns after the serving loop started), and
   * how many turns took over 5 ms */
  uint64_t worst_turn_at_ns, turns_over_5ms;
  /* the worker thread's minor page faults and voluntary context switches
   * over the whole run */
  uint64_t worker_minor_faults, worker_voluntary_switches;
  /* the longest wait of the worker for a lock another thread held, and the
   * longest locked host pass of an upload turn (staging the chunks) */
  uint64_t max_lock_wait_ns, max_upload_host_ns;
} haru_stream_stats;
int haru_stream_get_stats(haru_ctx *ctx, haru_stream_stats *out);

/* Work accounting of the last batch on this context (read after its stream
 * has been synchronised): items = warps of work (queries, or query pairs in
 * the int16 form), groups = CTA work units, segments = reference segments
 * per item (largest), fixups = segments recomputed because their
 * speculative start did not converge to the exact state. */
typedef struct {
  uint32_t items;
  uint32_t groups;
  uint32_t fixups;
  uint32_t max_segments;
} haru_batch_stats;
int haru_last_stats(haru_ctx *ctx, haru_batch_stats *out);

/* Status of the last HARU_ASYNC batch on this context (after the caller has
 * synchronised its stream): HARU_OK or the first error the device reported. */
int haru_last_status(haru_ctx *ctx);

/* Durations of the last HARU_PROFILE batch (after its stream has been
 * synchronised; for a captured graph, of its latest replay): ms_prep = the
 * planner and packing kernels, ms_sweep = the sweep kernel. Either pointer
 * may be NULL. Errors: HARU_EINVAL (no profiled batch yet), HARU_ECUDA. */
int haru_last_timing(haru_ctx *ctx, float *ms_prep, float *ms_sweep);

/* ---- Batch without allocation --------------------------------------------
 * No counterpart in the paper: an interface option of this library.
 *
 * haru_sdtw_batch_noalloc is haru_sdtw_batch for callers that cannot let the
 * library allocate device memory: a service that reserves its whole device
 * budget at start-up and must not grow afterwards, a host that forbids
 * run-time device allocation, or a latency-critical caller that cannot
 * accept cudaMalloc's implicit synchronisation stalling its other streams.
 * It calls no cudaMalloc, cudaFree or allocating library routine. Its
 * scratch memory (planner items and groups, packed query images, status and
 * work-queue counters) is one fixed array of 4,409,600 bytes (4.2 MiB)
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.
 *
 * events, offsets, out_cost and out_col are DEVICE pointers owned by the
 * caller, laid out as in haru_sdtw_batch; the reference is the context's.
 * precision: HARU_FP32 or HARU_INT16 (HARU_INT16_ACC32 returns HARU_EINVAL).
 * flags: 0 or HARU_RAW. The call is ordered on `stream` (0 = the context's)
 * and returns after the results are written. Sweeps are never cut into
 * reference segments and short queries are never stacked (both need more
 * scratch); results equal haru_sdtw_batch's.
 * Limits and errors: nq <= HARU_NOALLOC_MAX_QUERIES, else HARU_EINVAL (as for
 * any other flag or bad argument); per-query rules and the other codes as
 * for haru_sdtw_batch (a CUDA error is sticky on the context).
 * The first call on a device looks up the array's device address (which may
 * load the library's GPU code); make that first call before any stream
 * capture. Every call on every context of the process shares the one array
 * and it keeps the last call's contents: calls that overlap on the GPU (two
 * streams, two threads, two contexts on one device) race and must be
 * serialised by the caller. The call reads the context's reference without
 * holding the context for its whole run, so replacing the reference
 * (haru_ref_load, haru_ref_build) from another thread during it races as
 * well. */
#define HARU_NOALLOC_MAX_QUERIES 1024
int haru_sdtw_batch_noalloc(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets,
                            uint32_t nq, float *out_cost, int64_t *out_col, uintptr_t stream, uint32_t flags);

/* Autotuner: run the batch path on this batch (layout and flags as in
 * haru_sdtw_batch; HARU_ON_DEVICE and HARU_RAW are honoured) under every
 * combination of warps per CTA {4, 8, 12}, tile width {2048, 4096, 8192, 16384}
 * and work-unit target {1 (no reference segments), auto / 2, auto,
 * 2 x auto}, then, at the best of those, every stack_short rule (auto,
 * always, never: 32-lane strips or stacked 16-lane strips of twice the rows
 * per lane for queries of <= 256 events), keep the fastest (minimum of two
 * timed runs each) in the context's configuration
 * for later batches, and copy the resulting configuration to *chosen (may be
 * NULL). The strip height is fixed by each query's length. Results of the
 * trial runs are discarded. Errors: as haru_sdtw_batch. */
int haru_autotune(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
                  uint32_t flags, haru_config *chosen);

/* Measured ceiling of the cell update: the per-cell instructions of the
 * given form (int16: vsub2, viaddmax_relu, vimin3, viaddmin per two cells;
 * FP32: sub, 3-input min, fma per cell) issued on independent chains over
 * every SM, with none of the wavefront's data movement. *cells_per_s is the
 * best of three runs at the clock the GPU ran them. Errors: HARU_EINVAL,
 * HARU_ECUDA. */
int haru_probe_peak(haru_ctx *ctx, int precision, double *cells_per_s);

/* Human-readable name of a status code (static storage). */
const char *haru_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HARU_H_ */
