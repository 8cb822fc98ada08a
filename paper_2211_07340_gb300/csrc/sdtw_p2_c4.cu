// INT16_ACC32 (int16 inputs, wide accumulation) sweep kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(2, 4)
