// Allocation-free variant of the prescale statistics kernel.
//
// Some callers cannot allocate device memory when they call in: a host
// thread working inside another framework's fixed memory pool, a real-time
// reconstruction loop that is not allowed to reach the CUDA allocator between
// acquisitions, or code that has already committed every free byte of the GPU.
// mxfft_prescale_exponents_noalloc serves them: it computes the prescale
// exponent k of every slice (the same exponents mxfft_forward uses) with no
// cudaMalloc, cudaFree or allocating library call.  Its per-slice scratch
// (histogram, maxima, counters) lives in the file-scope array below, which
// every GPU that loads this library's device code holds until the process
// exits.
#include <cmath>
#include <mutex>

#include "mx_device.cuh"
#include "mxfft.h"

namespace mxfft {
namespace {

constexpr int kNoallocMaxSlices = MXFFT_NOALLOC_MAX_SLICES;
constexpr int kNoallocThreads = 256;
constexpr int kNoallocPtsPerCta = 4096;

// Scratch shared by every call (kNoallocMaxSlices records, about 1.2 MB).
static __device__ __align__(256) SliceStats g_noalloc_scratch[kNoallocMaxSlices];

// Same work as the statistics kernel of the transforms; the last CTA of a
// slice also stores the slice's exponent in the caller's output.
__global__ void __launch_bounds__(kNoallocThreads)
stats_noalloc_kernel(const float2* __restrict__ x, int npts, SliceStats* __restrict__ st,
                     KParams kp, uint32_t ctas_per_slice, int32_t* __restrict__ k_out) {
    __shared__ uint32_t sh_hist[kHistBins];
    __shared__ uint32_t sh_misc[4];
    const int tid = threadIdx.x;
    const int slice = blockIdx.y;
    for (int b = tid; b < kHistBins; b += blockDim.x) sh_hist[b] = 0;
    __syncthreads();
    const float4* xs = reinterpret_cast<const float4*>(x + (size_t)slice * npts);
    const int begin = blockIdx.x * kNoallocPtsPerCta;
    const int end = min(begin + kNoallocPtsPerCta, npts);
    StatAcc acc;
    for (int base = begin; base < end; base += 2 * blockDim.x) {
        const int p = base + 2 * tid;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < end) v = __ldg(xs + (p >> 1));
        acc.add(v.x, v.y, sh_hist);
        acc.add(v.z, v.w, sh_hist);
    }
    __syncthreads();
    stats_flush_and_select(acc, sh_hist, sh_misc, st + slice, ctas_per_slice, kp);
    if (sh_misc[3] && tid == 0) k_out[slice] = st[slice].k;
}

// Device address of the scratch array, looked up once per device and
// context.  The context's unique id (cuCtxGetId) is kept beside the address:
// after the caller resets the device (cudaDeviceReset) the next call runs in
// a new context, where the module and its array are loaded again, possibly
// elsewhere, so the address is looked up again.  The two driver entry points
// come through the runtime, so the library needs no link-time libcuda.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
SliceStats* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Unique id of the calling thread's current context (0 if unavailable).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

int scratch_for_current_device(SliceStats** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MXFFT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    // id 0: no context is current yet (the lookup below creates the primary one)
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        // the symbol's host-side name is not a device address; ask the runtime
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MXFFT_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<SliceStats*>(p);
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return MXFFT_OK;
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace
}  // namespace mxfft

extern "C" int mxfft_prescale_exponents_noalloc(const void* in, int batch, int n0, int n1,
                                                int format, float tau, float target,
                                                int32_t* k_out, void* stream) {
    using namespace mxfft;
    if (batch < 0 || batch > kNoallocMaxSlices) return MXFFT_ERR_INVALID;
    if (!pow2_in(n0, 2, 2048) || !pow2_in(n1, 2, 2048)) return MXFFT_ERR_INVALID;
    if (format < MXFFT_E4M3 || format > MXFFT_E2M1) return MXFFT_ERR_INVALID;
    if (!(tau > 0.0f && tau < 1.0f)) return MXFFT_ERR_INVALID;
    if (!(target > 0.0f) || target > 3.4e38f) return MXFFT_ERR_INVALID;
    int ex;
    if (std::frexp((double)target, &ex) != 0.5) return MXFFT_ERR_UNSUPPORTED;
    if (batch == 0) return MXFFT_OK;
    if (!in || !k_out || ((uintptr_t)in & 15u) || ((uintptr_t)k_out & 3u)) return MXFFT_ERR_INVALID;
    SliceStats* st = nullptr;
    int rc = scratch_for_current_device(&st);
    if (rc) return rc;
    KParams kp;
    kp.tau = tau;
    kp.t_exp = ex - 1;
    kp.taumin_exp = format == MXFFT_E5M2 ? -12 : -10;
    kp.kmin = -126;
    kp.kmax = 126;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear this call's records
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(SliceStats) * (size_t)batch, s);
    if (e != cudaSuccess) return MXFFT_ERR_CUDA;
    const int npts = n0 * n1;
    const uint32_t per = (uint32_t)((npts + kNoallocPtsPerCta - 1) / kNoallocPtsPerCta);
    dim3 grid(per, batch);
    stats_noalloc_kernel<<<grid, kNoallocThreads, 0, s>>>((const float2*)in, npts, st, kp, per,
                                                          k_out);
    return cudaGetLastError() == cudaSuccess ? MXFFT_OK : MXFFT_ERR_CUDA;
}
