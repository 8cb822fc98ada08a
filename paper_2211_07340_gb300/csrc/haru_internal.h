// Internal declarations shared by the CUDA translation units of libharu.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/haru.h"

namespace haru {

// One warp's work: a query (FP32), a pair of queries packed into the two
// 16-bit halves of every register (INT16 pair), or one query whose int16
// codes are computed exactly in FP32 (wide accumulation). qb < 0 when a pair
// is short. Its steps are cut into nseg segments (work units).
constexpr int kItemF32 = 0, kItemPair = 1, kItemExact = 2;
// A stacked item holds two strips one above the other in the warp's PE
// chain: lanes 0..15 sweep qa (and qb, INT16), lanes 16..31 sweep qc (and
// qd), each 16 * S rows high; lane 16 starts its stack from the free-start
// row instead of lane 15's last row.
struct Item {
  int qa;
  int qb;
  int S;        // rows per lane of the warp strip: 32 * S (16 * S if stacked) >= longest query
  int nseg;     // segments of its sweep
  int kind;     // kItemF32, kItemPair or kItemExact
  int qc;       // stacked: lower stack's queries (-1: none)
  int qd;
  int stacked;  // 1: two stacks of 16 lanes
};

// Queries of at most this many events are stacked two to a warp strip in
// batches large enough to fill the machine:
// stacking doubles the rows per lane, which raises throughput but also the
// time one strip takes, so small (latency-bound) batches stay unstacked.
constexpr int kStackMax = 16 * 16;

// Consecutive items with the same S swept over the same segment by one CTA,
// sharing one stream of reference tiles.
struct Group {
  int S;
  int first;
  int count;
  int seg;
  int nseg;
  int pad[3];
};

// Last-row minimum of one unit (item, segment): int16 halves a and b, or fp32.
struct Best {
  int ia, ib;
  float f;
  int pad;
  int64_t ca, cb;
};

// Per-item register image: [2][S][32] 32-bit words (INT16: packed query
// codes q and their negations -q, both -4095 on pad rows; FP32: query
// samples (0 on pad rows) and row weights, -1 on real rows and 0 on pad rows).
constexpr int kImgStride = 2 * 16 * 32;
// A saved strip state: the last two oblique columns, [2][S][32] words (the
// start-column forms follow them with their start columns, as many words).
constexpr int kStateStride = 2 * 16 * 32;
constexpr int kMaxS = 16;
constexpr int kMaxSeg = 64;
constexpr int kQmax = HARU_INT16_QMAX;
constexpr int kCap = HARU_INT16_CAP;
// Extra reference columns past N that the tile stream may read: the lane
// skew of the tallest strip (32 * 16) plus one whole tile.
constexpr int kMaxTile = 16384;
constexpr long kRefPad = 32 * kMaxS + kMaxTile + 64;
// Zero columns in front of column 0 of the device reference images: lane l
// of a strip reads the reference at column t - l * S (up to 31 * kMaxS
// behind the warp's step), and a tile's copy starts this many columns before
// the tile.
constexpr long kRefFront = 512;
static_assert(kRefFront >= 31 * kMaxS && kRefFront % 16 == 0, "front pad: the largest lane lag, whole 64-byte lines");

// Internal precisions of the sweep kernels beyond the public HARU_FP32,
// HARU_INT16 and HARU_INT16_ACC32: the FP32 and wide forms that also carry
// each alignment's start column (haru_sdtw_batch_span).
constexpr int kPrecF32Span = 3, kPrecWideSpan = 4;
__host__ __device__ constexpr bool prec_span(int p) { return p == kPrecF32Span || p == kPrecWideSpan; }
// Tracking-ring words per warp: costs (and start columns, +128, for the span forms).
// Words of one flush buffer of a warp's last-row tracking ring: a whole
// strip's tracked lane fills all of it between two scans, each stack of a
// stacked strip half. A warp holds two buffers, and the forms with start
// columns keep two more for the starts. Measured per form on GB300: 64 words
// for the int16 strips, 128 for the FP32-unit ones (fewer scans; the int16
// kernel ran 0.5% slower with 128, FP32 2.9% faster).
__host__ __device__ constexpr int flush_words(int p) { return p == HARU_INT16 ? 64 : 128; }
__host__ __device__ constexpr int ring_words(int p) { return (prec_span(p) ? 4 : 2) * flush_words(p); }
// Words of one saved strip state: costs, and start columns for the span forms.
__host__ __device__ constexpr int state_words(int p) { return prec_span(p) ? 2 * kStateStride : kStateStride; }

// Opt a kernel in to `bytes` of dynamic shared memory on the current
// device, calling the driver only when the size grows past what was set
// before on that device (a serving loop launches every few hundred
// microseconds). One record per kernel: `set` per device, under `mu`.
constexpr int kMaxDevices = 64;
struct SmemOptIn {
  std::atomic<int> set[kMaxDevices] = {};
  std::mutex mu;
};
template <class K>
inline cudaError_t opt_in_smem(K kernel, SmemOptIn &rec, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int want = static_cast<int>(bytes);
  if (dev < 0 || dev >= kMaxDevices)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (rec.set[dev].load(std::memory_order_acquire) >= want) return cudaSuccess;
  std::lock_guard<std::mutex> lk(rec.mu);
  if (rec.set[dev].load(std::memory_order_relaxed) >= want) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess) rec.set[dev].store(want, std::memory_order_release);
  return e;
}

// Layout of the small integer block every batch uses: the status word, the
// planner's group and item counts, the fix-up count, the sweep kernel's work
// queue counter and the most segments any item was cut into.
constexpr int kIntStatus = 0, kIntGroups = 1, kIntItems = 2, kIntFixups = 3, kIntQueue = 4, kIntMaxSeg = 5,
              kIntWords = 6;

__host__ __device__ inline int steps_per_chunk(int S) { return (S % 2 == 0) ? S : 2 * S; }

// Tile width (columns) for strip height S: a multiple of lcm(U, 4) not above T.
__host__ __device__ inline int tile_width(int S, int T) {
  const int U = steps_per_chunk(S);
  const int g = U % 4 == 0 ? 4 : (U % 2 == 0 ? 2 : 1);
  const int L = U / g * 4;
  const int w = (T / L) * L;
  return w > 0 ? w : L;
}

// Steps a speculative segment runs before its own first step: three strip
// heights, so even the strip's last row has two heights of columns behind
// it (alignments span fewer columns than rows here; a segment whose start
// state still differs is recomputed by the fix-up kernel).
__host__ __device__ inline long warmup_steps(int S) {
  const int U = steps_per_chunk(S);
  return (3L * 32 * S + U - 1) / U * U;
}

// Whole-chunk step count of one sweep of strip height S over N columns.
__host__ __device__ inline long sweep_steps(int S, long N) {
  const int U = steps_per_chunk(S);
  return (N + 32L * S - 1 + U - 1) / U * U;
}

// Steps of segment `seg` of `nseg`: own steps [t_own, t_end), warm-up from t_start.
__host__ __device__ inline void seg_bounds(int S, int nseg, int seg, long N, long *t_start, long *t_own,
                                           long *t_end) {
  const int U = steps_per_chunk(S);
  const long chunks = sweep_steps(S, N) / U;
  *t_own = chunks * seg / nseg * U;
  *t_end = chunks * (seg + 1) / nseg * U;
  const long w = *t_own - warmup_steps(S);
  *t_start = seg == 0 ? 0 : (w > 0 ? w : 0);
}

struct SdtwArgs {
  const void *ref_img;     // INT16: uint32 (r | r << 16); FP32: float. Column 0 of N + kRefPad words,
                           // kRefFront zero words before it
  long N;                  // reference length (columns)
  const uint32_t *img;     // item images, kImgStride words each
  const Item *items;
  const Group *groups;
  int *ints;               // kIntWords status and counter words
  uint32_t *states;        // [item][nseg_cap][2] saved states (start, final), kStateStride words each
  Best *bests;             // [item][nseg_cap]: the strip's (upper stack's) last-row minimum
  Best *bests2;            // [item][nseg_cap]: the lower stack's, for stacked items
  int64_t *out_start;      // span forms: the alignment start column per query
  int nseg_cap;
  float *out_cost;
  int64_t *out_col;
  float inv_scale;         // INT16: 2^-k
  int tile_cols;           // requested tile width T (columns)
  int warps;               // warps per CTA = items per group
  unsigned long long wait_ns;
};

// Planner / prep arguments.
struct PlanArgs {
  const uint32_t *offsets;  // nq + 1
  uint32_t nq;
  long N;
  int pair;                 // 0: FP32 singles; 1: INT16 pairs; 3: exact-integer singles, unsaturated
                            // (HARU_INT16_ACC32)
  int warps;                // items per group
  int units_target;         // wanted work units (item x segment) in the batch
  int stack;                // 1: stack queries of <= kStackMax events two to a strip
  int nseg_cap;             // most segments per item (state storage is sized for it)
  Item *items;
  Group *groups;
  int *ints;                // kIntWords counters (status, counts, queues, class ranges)
};

struct PackArgs {
  const float *events;
  const uint32_t *offsets;
  const Item *items;
  const int *n_items;
  uint32_t *img;
  int raw;                  // z-score each query first
  const double *qstats;     // raw: (mean, sigma) of query q at 2q, 2q+1 (launch_qstats)
  int pair;
  int scale_log2;
  int *status;
};

// Kernel launchers (stream-ordered, no synchronisation).
cudaError_t launch_plan(const PlanArgs &a, cudaStream_t s);
cudaError_t launch_pack(const PackArgs &a, uint32_t max_items, cudaStream_t s);
// Mean and population sigma (FP64, sequential order) of each query of 1..512 events.
cudaError_t launch_qstats(const float *events, const uint32_t *offsets, uint32_t nq, double *qstats, int *status,
                          cudaStream_t s);
cudaError_t launch_sdtw(int precision, const SdtwArgs &a, int grid, int fix_items, cudaStream_t s,
                        cudaEvent_t ev_fix = nullptr);
// cudaEventRecord that also works inside a stream capture (batch.cu).
cudaError_t record_event(cudaEvent_t e, cudaStream_t s);
// Load kernels into the current context now instead of at their first
// launch (lazy module loading): the planner, statistics and packing kernels,
// and the sweep and fix-up kernels of a precision.
cudaError_t load_prep_kernels();
cudaError_t load_sdtw(int precision);
size_t sdtw_smem_bytes(int precision, int tile_cols, int warps);
int sdtw_max_ctas_per_sm(int precision, int tile_cols, int warps);

// Reference preparation.
cudaError_t launch_ref_levels(const uint8_t *bases, size_t n, const float *model, int k, float *out,
                              int *status, cudaStream_t s);
cudaError_t launch_zscore_stats(const float *x, size_t n, double *partials, double *stats, int *status,
                                cudaStream_t s);
cudaError_t launch_ref_finish(const float *x, size_t n, const double *stats, int normalize, int scale_log2,
                              float *z, uint32_t *img16, float *img32, size_t img_len, int *status,
                              cudaStream_t s);

// Set *status to code if it is still 0 (device side).
__device__ __forceinline__ void report(int *status, int code) { atomicCAS(status, 0, code); }

}  // namespace haru
