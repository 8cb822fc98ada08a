// INT16 sweep kernel, strip-height class 1 (S 9..12).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(1, 1)
