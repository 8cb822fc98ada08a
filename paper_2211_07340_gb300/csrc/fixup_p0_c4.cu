// FP32 segment fix-up kernel, strip-height class 4 (every S, 1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(0, 4)
