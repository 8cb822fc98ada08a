// FP32 sweep kernel, strip-height class 4 (every S, 1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(0, 4)
