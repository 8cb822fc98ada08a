// FP32 segment fix-up kernel, strip-height class 0 (S 13..16).
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(0, 0)
