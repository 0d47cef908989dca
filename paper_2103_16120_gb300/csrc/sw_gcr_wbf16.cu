// sw_gcr_wbf16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the BF16 mixed policy, one warp per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolBF16, 1, wbf16)
} // namespace sw
