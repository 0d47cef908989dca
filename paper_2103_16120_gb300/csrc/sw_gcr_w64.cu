// sw_gcr_w64.cu -- the persistent GCR kernel (sw_gcr.cuh) for the FP64 policy, one warp per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolFP64, 1, w64)
} // namespace sw
