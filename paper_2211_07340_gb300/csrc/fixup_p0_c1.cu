// FP32 segment fix-up kernel, strip-height class 1 (S 9..12).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(0, 1)
