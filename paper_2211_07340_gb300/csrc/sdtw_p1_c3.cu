// INT16 sweep kernel, strip-height class 3 (S 1..4).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(1, 3)
