// sw_static.cu -- the fixed device scratch of sw_gcr_solve_noalloc.  The array
// is part of this translation unit's device code, so it comes into being when
// the module is loaded, not through a runtime allocation.  It sits in a file
// of its own so that, with lazy module loading, only programs that use the
// no-allocation solve load it.
#include <mutex>

#include "../../include/sw_elliptic.h"
#include "sw_internal.h"

namespace sw {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;

cudaError_t noalloc_scratch(void **ptr, size_t *bytes)
{
    static std::mutex mu;
    static void *addr[NOALLOC_MAX_DEVICES] = {};
    *ptr = nullptr;
    *bytes = SW_NOALLOC_SCRATCH_BYTES;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        // once per device, with that device current
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

} // namespace sw
