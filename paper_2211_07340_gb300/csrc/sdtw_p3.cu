// FP32 with start columns: the sweep kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(3)

// The saved-state size the batch engine allocates per work unit (state_words)
// is the one the kernels index, for every form.
namespace haru {
static_assert(state_rows_per_s<kFormF32>() * kMaxS * 32 == state_words(HARU_FP32), "FP32 state size");
static_assert(state_rows_per_s<kFormI16>() * kMaxS * 32 == state_words(HARU_INT16), "int16 state size");
static_assert(state_rows_per_s<kFormExactWide>() * kMaxS * 32 == state_words(HARU_INT16_ACC32), "wide state size");
static_assert(state_rows_per_s<kFormF32Span>() * kMaxS * 32 == state_words(kPrecF32Span), "span state size");
static_assert(state_rows_per_s<kFormWideSpan>() * kMaxS * 32 == state_words(kPrecWideSpan), "wide span state size");
}  // namespace haru
