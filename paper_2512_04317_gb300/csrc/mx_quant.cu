// The element quantiser of Alg. 2 (the rounding Q inside EncodeBlockMX and
// EncodeFromMantBlock) applied to plain FP32 values, with the device code of
// the transforms: the register-resident pass's hardware conversions
// (cvt.rn.satfinite.<fmt>x2.f32, then back to exact f16 values) and the
// generic pass's FP32 add-and-subtract rounding (q_elem).  It exists so that
// both can be compared value by value with an independent implementation.
#include <cuda_fp16.h>

#include "mx_fast_impl.cuh"
#include "mxfft.h"

namespace mxfft {
namespace {

constexpr int kQuantThreads = 256;

template <int FMT>
__global__ void __launch_bounds__(kQuantThreads)
quant_cvt_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long npairs) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const float2 v = in[i];
        const uint32_t h = fast::Cvt<FMT>::q2(v.x, v.y);
        const __half2 hh = *reinterpret_cast<const __half2*>(&h);
        out[i] = make_float2(__low2float(hh), __high2float(hh));
    }
}

__global__ void __launch_bounds__(kQuantThreads)
quant_generic_kernel(const float* __restrict__ in, float* __restrict__ out, long long n,
                     FmtParams fp) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = q_elem(in[i], fp);
}

}  // namespace
}  // namespace mxfft

extern "C" int mxfft_quantize(const void* in, void* out, long long n, int format, int path,
                              void* stream) {
    using namespace mxfft;
    FmtParams fp;
    if (n < 0 || format < MXFFT_E4M3 || format > MXFFT_E2M1 || !fmt_params(format, &fp))
        return MXFFT_ERR_INVALID;
    if (path != 0 && path != 1) return MXFFT_ERR_INVALID;
    if (n == 0) return MXFFT_OK;
    if (!in || !out) return MXFFT_ERR_INVALID;
    if (path == 0 && ((n & 1) || ((uintptr_t)in & 7u) || ((uintptr_t)out & 7u))) return MXFFT_ERR_INVALID;
    if (path == 1 && (((uintptr_t)in & 3u) || ((uintptr_t)out & 3u))) return MXFFT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const long long items = path == 0 ? n / 2 : n;
    const long long want = (items + kQuantThreads - 1) / kQuantThreads;
    const unsigned blocks = (unsigned)(want < 8192 ? want : 8192);
    if (path == 1) {
        quant_generic_kernel<<<blocks, kQuantThreads, 0, s>>>((const float*)in, (float*)out, n, fp);
    } else {
        const float2* i2 = (const float2*)in;
        float2* o2 = (float2*)out;
        switch (format) {
            case MXFFT_E4M3: quant_cvt_kernel<0><<<blocks, kQuantThreads, 0, s>>>(i2, o2, items); break;
            case MXFFT_E5M2: quant_cvt_kernel<1><<<blocks, kQuantThreads, 0, s>>>(i2, o2, items); break;
            case MXFFT_E2M3: quant_cvt_kernel<2><<<blocks, kQuantThreads, 0, s>>>(i2, o2, items); break;
            case MXFFT_E3M2: quant_cvt_kernel<3><<<blocks, kQuantThreads, 0, s>>>(i2, o2, items); break;
            default: quant_cvt_kernel<4><<<blocks, kQuantThreads, 0, s>>>(i2, o2, items); break;
        }
    }
    note_launch();
    return cudaGetLastError() == cudaSuccess ? MXFFT_OK : MXFFT_ERR_CUDA;
}
