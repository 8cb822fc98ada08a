// Sweep kernel of the int16 form with an exact-integer share (int16 pairs and
// exact FP32 singles in one queue), every strip height.
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(5, 4)
