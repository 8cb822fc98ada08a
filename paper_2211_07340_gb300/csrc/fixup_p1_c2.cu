// INT16 segment fix-up kernel, strip-height class 2 (S 5..8).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(1, 2)
