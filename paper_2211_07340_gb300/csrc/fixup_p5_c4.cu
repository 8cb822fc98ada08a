// Segment fix-up kernel of the int16 form with an exact-integer share.
#include "sdtw_kernels.cuh"

HARU_SDTW_FIXUP_INSTANCE(5, 4)
