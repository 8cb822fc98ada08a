// Launch dispatch of the sweep and fix-up kernels. The kernels are defined
// in sdtw_kernels.cuh and instantiated one (precision, strip-height class)
// per translation unit (sdtw_p<P>_c<C>.cu: sweep; fixup_p<P>_c<C>.cu: fix-up).

#include <cuda_runtime.h>

#include "haru_internal.h"

namespace haru {

#define HARU_SDTW_DECLARE(P, C)                                                        \
  cudaError_t sdtw_sweep_##P##_##C(const SdtwArgs &a, int grid, cudaStream_t s);       \
  cudaError_t sdtw_fixup_##P##_##C(const SdtwArgs &a, int fix_items, cudaStream_t s);  \
  int sdtw_occupancy_##P##_##C(int tile_cols, int warps);
HARU_SDTW_DECLARE(0, 0)
HARU_SDTW_DECLARE(0, 1)
HARU_SDTW_DECLARE(0, 2)
HARU_SDTW_DECLARE(0, 3)
HARU_SDTW_DECLARE(0, 4)
HARU_SDTW_DECLARE(1, 0)
HARU_SDTW_DECLARE(1, 1)
HARU_SDTW_DECLARE(1, 2)
HARU_SDTW_DECLARE(1, 3)
HARU_SDTW_DECLARE(1, 4)
HARU_SDTW_DECLARE(2, 4)
HARU_SDTW_DECLARE(3, 4)
HARU_SDTW_DECLARE(4, 4)
HARU_SDTW_DECLARE(5, 4)

namespace {
#define HARU_SDTW_BOTH(P, C)                                                               \
  if ((e = sdtw_sweep_##P##_##C(a, grid, s)) != cudaSuccess) return e;                     \
  return sdtw_fixup_##P##_##C(a, fix_items, s);
cudaError_t launch_p1(int cls, const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  switch (cls) {
    case 0: HARU_SDTW_BOTH(1, 0)
    case 1: HARU_SDTW_BOTH(1, 1)
    case 2: HARU_SDTW_BOTH(1, 2)
    case 4: HARU_SDTW_BOTH(1, 4)
    default: HARU_SDTW_BOTH(1, 3)
  }
}
// The wide form, the start-column forms and the int16 form with an exact
// share have the single kernel only.
cudaError_t launch_p2(const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  HARU_SDTW_BOTH(2, 4)
}
cudaError_t launch_p3(const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  HARU_SDTW_BOTH(3, 4)
}
cudaError_t launch_p4(const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  HARU_SDTW_BOTH(4, 4)
}
cudaError_t launch_p5(const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  HARU_SDTW_BOTH(5, 4)
}
cudaError_t launch_p0(int cls, const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  cudaError_t e;
  switch (cls) {
    case 0: HARU_SDTW_BOTH(0, 0)
    case 1: HARU_SDTW_BOTH(0, 1)
    case 2: HARU_SDTW_BOTH(0, 2)
    case 4: HARU_SDTW_BOTH(0, 4)
    default: HARU_SDTW_BOTH(0, 3)
  }
}
}  // namespace

size_t sdtw_smem_bytes(int precision, int tile_cols, int warps) {
  // Shared header, per-warp tracking rings, 32 zero words, two tile slots
  return 128 + static_cast<size_t>(warps) * ring_words(precision) * 4 + 32 * 4 +
         2 * static_cast<size_t>(tile_cols) * 4;
}

int sdtw_max_ctas_per_sm(int precision, int cls, int tile_cols, int warps) {
  if (precision == HARU_INT16_ACC32) return sdtw_occupancy_2_4(tile_cols, warps);
  if (precision == kPrecF32Span) return sdtw_occupancy_3_4(tile_cols, warps);
  if (precision == kPrecWideSpan) return sdtw_occupancy_4_4(tile_cols, warps);
  if (precision == kPrecI16Mixed) return sdtw_occupancy_5_4(tile_cols, warps);
  if (precision == HARU_INT16) {
    switch (cls) {
      case 0: return sdtw_occupancy_1_0(tile_cols, warps);
      case 1: return sdtw_occupancy_1_1(tile_cols, warps);
      case 2: return sdtw_occupancy_1_2(tile_cols, warps);
      case 4: return sdtw_occupancy_1_4(tile_cols, warps);
      default: return sdtw_occupancy_1_3(tile_cols, warps);
    }
  }
  switch (cls) {
    case 0: return sdtw_occupancy_0_0(tile_cols, warps);
    case 1: return sdtw_occupancy_0_1(tile_cols, warps);
    case 2: return sdtw_occupancy_0_2(tile_cols, warps);
    case 4: return sdtw_occupancy_0_4(tile_cols, warps);
    default: return sdtw_occupancy_0_3(tile_cols, warps);
  }
}

// The sweep kernel of the class, then its segment fix-up kernel (which also
// writes the outputs), stream-ordered.
cudaError_t launch_sdtw(int precision, int cls, const SdtwArgs &a, int grid, int fix_items, cudaStream_t s) {
  if (precision == HARU_INT16_ACC32) return launch_p2(a, grid, fix_items, s);
  if (precision == kPrecF32Span) return launch_p3(a, grid, fix_items, s);
  if (precision == kPrecWideSpan) return launch_p4(a, grid, fix_items, s);
  if (precision == kPrecI16Mixed) return launch_p5(a, grid, fix_items, s);
  return precision == HARU_INT16 ? launch_p1(cls, a, grid, fix_items, s) : launch_p0(cls, a, grid, fix_items, s);
}

}  // namespace haru
