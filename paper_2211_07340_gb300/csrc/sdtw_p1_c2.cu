// INT16 sweep kernel, strip-height class 2 (S 5..8).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(1, 2)
