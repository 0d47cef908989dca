// sw_gcr_sbf16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the BF16 mixed policy, one warp per row,
// specialised for rows of 1024 and 2048 points.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_SPEC_UNIT(PolBF16, sbf16)
} // namespace sw
