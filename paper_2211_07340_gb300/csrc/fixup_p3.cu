// FP32 with start columns: the segment fix-up kernel, every strip height (1..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(3)
