// sw_gcr_s16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the FP16 mixed policy, one warp per row,
// specialised for rows of 1024 and 2048 points.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_SPEC_UNIT(PolF16, s16)
} // namespace sw
