// Root-sum-of-squares coil combine of Eq. (1): x_RSS = (sum_c |T_c|^2)^(1/2)
// per point of each image, where the coil images T_c are consecutive slices.
// Coils are added in order c = 0, 1, ... in FP32 (acc + (re^2 + im^2)), then
// one correctly rounded square root.  Bound by HBM: 8 B read per point and
// coil, 4 B written per point; each thread combines two points (one 16-byte
// load per coil).
#include "mx_plan.h"

namespace mxfft {

namespace {

constexpr int kRssThreads = 256;

__global__ void __launch_bounds__(kRssThreads)
rss_kernel(RssRef val, const RssRef* __restrict__ dev) {
    const RssRef r = dev ? *dev : val;
    const long long pairs = r.npts >> 1;                 // per image
    const long long total = pairs * r.images;
    const float4* __restrict__ z = reinterpret_cast<const float4*>(r.z);
    float2* __restrict__ out = reinterpret_cast<float2*>(r.out);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long img = q / pairs, pp = q - img * pairs;
        const float4* zi = z + img * r.coils * pairs + pp;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll 4
        for (int c = 0; c < r.coils; c++) {
            const float4 v = __ldg(zi + (long long)c * pairs);
            a0 = __fadd_rn(a0, __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
            a1 = __fadd_rn(a1, __fadd_rn(__fmul_rn(v.z, v.z), __fmul_rn(v.w, v.w)));
        }
        out[q] = make_float2(__fsqrt_rn(a0), __fsqrt_rn(a1));
    }
}

int rss_grid(long long images, long long npts) {
    const long long pairs = images * (npts >> 1);
    long long blocks = (pairs + kRssThreads - 1) / kRssThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;            // grid-stride beyond that
    return (int)(blocks > 0 ? blocks : 1);
}

}  // namespace

cudaError_t launch_rss(const RssRef& val, const RssRef* dev, long long images, long long npts,
                       cudaStream_t s) {
    if (images <= 0 || npts <= 0) return cudaSuccess;
    rss_kernel<<<rss_grid(images, npts), kRssThreads, 0, s>>>(val, dev);
    note_launch();
    return cudaGetLastError();
}

}  // namespace mxfft

extern "C" int mxfft_rss(const void* z, void* out, int images, int coils, int n0, int n1,
                         void* stream) {
    using namespace mxfft;
    if (images < 0 || coils < 1 || n0 < 1 || n1 < 1) return MXFFT_ERR_INVALID;
    if (images == 0) return MXFFT_OK;
    const long long npts = (long long)n0 * n1;
    if ((npts & 1) || !z || !out || ((uintptr_t)z & 15u) || ((uintptr_t)out & 15u))
        return MXFFT_ERR_INVALID;
    const char* cz = (const char*)z;
    const char* co = (const char*)out;
    const size_t zb = (size_t)images * coils * npts * sizeof(float2);
    const size_t ob = (size_t)images * npts * sizeof(float);
    if (cz < co + ob && co < cz + zb) return MXFFT_ERR_INVALID;
    RssRef r{(const float2*)z, (float*)out, coils, images, npts};
    return cuda_status(launch_rss(r, nullptr, images, npts, (cudaStream_t)stream));
}
