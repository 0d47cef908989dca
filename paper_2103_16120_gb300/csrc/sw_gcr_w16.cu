// sw_gcr_w16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the FP16 mixed policy, one warp per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolF16, 1, w16)
} // namespace sw
