// Launch dispatch of the sweep and fix-up kernels. The kernels are defined
// in sdtw_kernels.cuh and instantiated one kernel precision per translation
// unit (sdtw_p<P>.cu: sweep; fixup_p<P>.cu: fix-up), so they compile in
// parallel.

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "haru_internal.h"

namespace haru {

#define HARU_SDTW_DECLARE(P)                                                        \
  cudaError_t sdtw_sweep_##P(const SdtwArgs &a, int grid, cudaStream_t s);          \
  cudaError_t sdtw_fixup_##P(const SdtwArgs &a, int fix_items, cudaStream_t s);     \
  int sdtw_occupancy_##P(int tile_cols, int warps);                                 \
  cudaError_t sdtw_sweep_load_##P();                                                \
  cudaError_t sdtw_fixup_load_##P();
HARU_SDTW_DECLARE(0)
HARU_SDTW_DECLARE(1)
HARU_SDTW_DECLARE(2)
HARU_SDTW_DECLARE(3)
HARU_SDTW_DECLARE(4)

size_t sdtw_smem_bytes(int precision, int tile_cols, int warps) {
  // Shared header, per-warp tracking rings, two tile slots (each with the
  // kRefFront columns before its tile)
  return 128 + static_cast<size_t>(warps) * ring_words(precision) * 4 +
         2 * static_cast<size_t>(tile_cols + kRefFront) * 4;
}

namespace {
int occupancy_query(int precision, int tile_cols, int warps) {
  switch (precision) {
    case HARU_INT16: return sdtw_occupancy_1(tile_cols, warps);
    case HARU_INT16_ACC32: return sdtw_occupancy_2(tile_cols, warps);
    case kPrecF32Span: return sdtw_occupancy_3(tile_cols, warps);
    case kPrecWideSpan: return sdtw_occupancy_4(tile_cols, warps);
    default: return sdtw_occupancy_0(tile_cols, warps);
  }
}
}  // namespace

// Resident CTAs per SM of a launch shape, asked of the runtime once per
// (device, precision, tile, warps): every batch launch needs it.
int sdtw_max_ctas_per_sm(int precision, int tile_cols, int warps) {
  struct Entry {
    int dev, precision, tile_cols, warps, ctas;
  };
  static std::mutex mu;
  static std::vector<Entry> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return occupancy_query(precision, tile_cols, warps);
  std::lock_guard<std::mutex> lk(mu);
  for (const Entry &x : memo)
    if (x.dev == dev && x.precision == precision && x.tile_cols == tile_cols && x.warps == warps) return x.ctas;
  const int n = occupancy_query(precision, tile_cols, warps);
  if (n > 0) memo.push_back(Entry{dev, precision, tile_cols, warps, n});
  return n;
}

// Load the sweep and fix-up kernels of a precision into the context now
// rather than at their first launch (lazy module loading), so a latency-bound
// caller does not pay the load inside its first request.
cudaError_t load_sdtw(int precision) {
  cudaError_t e;
#define HARU_SDTW_LOAD(P)                                        \
  if ((e = sdtw_sweep_load_##P()) != cudaSuccess) return e;      \
  return sdtw_fixup_load_##P();
  switch (precision) {
    case HARU_INT16: HARU_SDTW_LOAD(1)
    case HARU_INT16_ACC32: HARU_SDTW_LOAD(2)
    case kPrecF32Span: HARU_SDTW_LOAD(3)
    case kPrecWideSpan: HARU_SDTW_LOAD(4)
    default: HARU_SDTW_LOAD(0)
  }
#undef HARU_SDTW_LOAD
}

// The sweep kernel of the precision, then its segment fix-up kernel (which
// also writes the outputs), stream-ordered; ev_fix (if given) is recorded
// between the two.
cudaError_t launch_sdtw(int precision, const SdtwArgs &a, int grid, int fix_items, cudaStream_t s,
                        cudaEvent_t ev_fix) {
  cudaError_t e;
#define HARU_SDTW_BOTH(P)                                                       \
  if ((e = sdtw_sweep_##P(a, grid, s)) != cudaSuccess) return e;                \
  if (ev_fix && (e = record_event(ev_fix, s)) != cudaSuccess) return e;         \
  return sdtw_fixup_##P(a, fix_items, s);
  switch (precision) {
    case HARU_INT16: HARU_SDTW_BOTH(1)
    case HARU_INT16_ACC32: HARU_SDTW_BOTH(2)
    case kPrecF32Span: HARU_SDTW_BOTH(3)
    case kPrecWideSpan: HARU_SDTW_BOTH(4)
    default: HARU_SDTW_BOTH(0)
  }
#undef HARU_SDTW_BOTH
}

}  // namespace haru
