// INT16_ACC32 (wide accumulation) with start columns: segment fix-up kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(4, 4)
