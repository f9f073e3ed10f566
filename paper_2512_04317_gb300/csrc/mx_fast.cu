// Dispatch of the register-resident MX pass by element format and block size.
#include "mx_fast_kernel.cuh"

namespace mxfft {
namespace fast {
template <int FMT>
cudaError_t launch_fast_fmt(const FastArgs&, int, int, cudaStream_t);
extern template cudaError_t launch_fast_fmt<0>(const FastArgs&, int, int, cudaStream_t);
extern template cudaError_t launch_fast_fmt<1>(const FastArgs&, int, int, cudaStream_t);
extern template cudaError_t launch_fast_fmt<2>(const FastArgs&, int, int, cudaStream_t);
extern template cudaError_t launch_fast_fmt<3>(const FastArgs&, int, int, cudaStream_t);
extern template cudaError_t launch_fast_fmt<4>(const FastArgs&, int, int, cudaStream_t);
}  // namespace fast

namespace {
int log2_exact(int m) {
    int l = 0;
    while ((1 << l) < m) l++;
    return (1 << l) == m ? l : -1;
}
}  // namespace

bool fast_pass_supported(const PassArgs& a) {
    int TG, S, NG, threads;
    const int other = a.dim == 1 ? a.n0 : a.n1;
    const int logm = log2_exact(a.m);
    return logm >= 0 && logm <= 4 && a.fp.mbits > 0 &&
           fast::fast_geometry(a.n, other, &TG, &S, &NG, &threads);
}

cudaError_t launch_fast_pass(const PassArgs& a, const uint32_t* twh, const TwA& twa, int batch,
                             cudaStream_t s) {
    if (!fast_pass_supported(a)) return cudaErrorNotSupported;
    fast::FastArgs fa;
    fa.a = a;
    fa.twa = twa;
    fa.twh = twh;
    int threads;
    const int other = a.dim == 1 ? a.n0 : a.n1;
    fast::fast_geometry(a.n, other, &fa.TG, &fa.S, &fa.NG, &threads);
    fa.lgTG = fa.TG == 16 ? 4 : 3;
    const int logm = log2_exact(a.m);
    switch (a.fmt) {
        case 0: return fast::launch_fast_fmt<0>(fa, logm, batch, s);
        case 1: return fast::launch_fast_fmt<1>(fa, logm, batch, s);
        case 2: return fast::launch_fast_fmt<2>(fa, logm, batch, s);
        case 3: return fast::launch_fast_fmt<3>(fa, logm, batch, s);
        case 4: return fast::launch_fast_fmt<4>(fa, logm, batch, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace mxfft
