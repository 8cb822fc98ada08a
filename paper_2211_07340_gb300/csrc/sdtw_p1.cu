// int16 (packed DPX pairs): the sweep kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_SWEEP_INSTANCE(1)
