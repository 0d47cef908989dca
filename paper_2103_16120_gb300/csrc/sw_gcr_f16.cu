// sw_gcr_f16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the FP16 mixed policy, one block per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolF16, 0, f16)
} // namespace sw
