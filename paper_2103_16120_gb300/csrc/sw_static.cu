// sw_static.cu -- the fixed device scratch of sw_gcr_solve_noalloc.  The array
// is part of this translation unit's device code, so it comes into being when
// the module is loaded, not through a runtime allocation.  It sits in a file
// of its own so that, with lazy module loading, only programs that use the
// no-allocation solve load it.
#include "../../include/sw_elliptic.h"
#include "sw_internal.h"

namespace sw {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

// The device address of the scratch in the current context.  Host code only
// holds a stand-in for the array, so the address is asked of the runtime on
// every call: a context that was torn down and created again (a device reset,
// a released and re-retained primary context) reloads the module, and the
// array may then sit elsewhere.  The lookup allocates nothing.
cudaError_t noalloc_scratch(void **ptr, size_t *bytes)
{
    *ptr = nullptr;
    *bytes = SW_NOALLOC_SCRATCH_BYTES;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *ptr = p;
    return cudaSuccess;
}

} // namespace sw
