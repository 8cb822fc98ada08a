// FP32 segment fix-up kernel, strip-height class 3 (S 1..4).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(0, 3)
