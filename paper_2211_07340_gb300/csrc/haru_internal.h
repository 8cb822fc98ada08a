// Internal declarations shared by the CUDA translation units of libharu.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/haru.h"

namespace haru {

// One warp's work: a query (FP32) or a pair of queries packed into the two
// 16-bit halves of every register (INT16). qb < 0 when the pair is short.
struct Item {
  int qa;
  int qb;
  int S;  // rows per lane of the warp strip: 32 * S >= longest query of the item
  int pad;
};

// Consecutive items with the same S, swept together by one CTA over one
// shared stream of reference tiles.
struct Group {
  int S;
  int first;
  int count;
  int pad;
};

// Per-item register image: [2][S][32] 32-bit words (INT16: packed query
// samples, packed caps; FP32: query samples, row weights).
constexpr int kImgStride = 2 * 16 * 32;
constexpr int kMaxS = 16;
constexpr int kQmax = HARU_INT16_QMAX;
constexpr int kCap = HARU_INT16_CAP;
// Extra reference columns past N that the tile stream may read: the lane
// skew of the tallest strip (32 * 16) plus one whole tile.
constexpr int kMaxTile = 16384;
constexpr long kRefPad = 32 * kMaxS + kMaxTile + 64;

struct SdtwArgs {
  const void *ref_img;     // INT16: uint32 (r | r << 16); FP32: float. >= N + kRefPad words
  long N;                  // reference length (columns)
  const uint32_t *img;     // item images, kImgStride words each
  const Item *items;
  const Group *groups;
  const int *n_groups;
  int *queue;              // work counter, zero before launch
  float *out_cost;
  int64_t *out_col;
  float inv_scale;         // INT16: 2^-k
  int tile_cols;           // requested tile width T (columns)
  int warps;               // warps per CTA = items per group
  unsigned long long wait_ns;
  int *status;             // first error code (0 = none)
};

// Planner / prep arguments.
struct PlanArgs {
  const uint32_t *offsets;  // nq + 1
  uint32_t nq;
  long N;
  int pair;                 // 1: INT16 (two queries per item)
  int warps;                // items per group
  Item *items;
  Group *groups;
  int *n_groups;
  int *n_items;
  int *queue;
  int *status;
};

struct PackArgs {
  const float *events;
  const uint32_t *offsets;
  const Item *items;
  const int *n_items;
  uint32_t *img;
  int raw;                  // z-score each query first
  int pair;
  int scale_log2;
  int *status;
};

// Kernel launchers (stream-ordered, no synchronisation).
cudaError_t launch_plan(const PlanArgs &a, cudaStream_t s);
cudaError_t launch_pack(const PackArgs &a, uint32_t max_items, cudaStream_t s);
cudaError_t launch_sdtw(int precision, const SdtwArgs &a, int grid, cudaStream_t s);
size_t sdtw_smem_bytes(int tile_cols, int warps);
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
