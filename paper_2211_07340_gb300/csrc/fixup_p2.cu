// int16 inputs with wide accumulation: the segment fix-up kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(2)
