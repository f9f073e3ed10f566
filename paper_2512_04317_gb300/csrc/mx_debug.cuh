// Bounds checks of the MXFFT_DEBUG_BOUNDS build (a stand-in for a memory
// checker): each kernel passes its computed global and shared-memory indices
// through MX_BND(i, n).  In the normal build the macro is the index itself, so
// the code is unchanged.  In the debug build an index outside [0, n) is
// counted in this translation unit's device counter and replaced by 0 (a
// valid index), so that the access stays inside its buffer instead of
// faulting; mxfft_debug_bounds reads and clears the counters.
#pragma once

#include <cuda_runtime.h>

namespace mxfft {

#ifdef MXFFT_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_bad;   // one per translation unit

__device__ __forceinline__ long long bound_index(long long i, long long n) {
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_bad, 1ull);
        return 0;
    }
    return i;
}
#define MX_BND(i, n) ((int64_t)::mxfft::bound_index((long long)(i), (long long)(n)))
// Host reader of this translation unit's counter (returns it and clears it).
#define MX_BOUNDS_COUNTER(name)                                                            \
    unsigned long long bounds_take_##name() {                                              \
        unsigned long long v = 0, z = 0;                                                   \
        if (cudaMemcpyFromSymbol(&v, g_bounds_bad, sizeof v) != cudaSuccess) return ~0ull;  \
        if (cudaMemcpyToSymbol(g_bounds_bad, &z, sizeof z) != cudaSuccess) return ~0ull;    \
        return v;                                                                          \
    }
#else
#define MX_BND(i, n) (i)
#define MX_BOUNDS_COUNTER(name)
#endif

}  // namespace mxfft
