// sw_gcr_bf16.cu -- the persistent GCR kernel (sw_gcr.cuh) for the BF16 mixed policy, one block per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolBF16, 0, bf16)
} // namespace sw
