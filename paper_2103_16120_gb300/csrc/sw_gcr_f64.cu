// sw_gcr_f64.cu -- the persistent GCR kernel (sw_gcr.cuh) for the FP64 policy, one block per row.
#include "sw_gcr.cuh"

namespace sw {
SW_GCR_UNIT(PolFP64, 0, f64)
} // namespace sw
