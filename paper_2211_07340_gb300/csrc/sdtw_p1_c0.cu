// INT16 sweep kernel, strip-height class 0 (S 13..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(1, 0)
