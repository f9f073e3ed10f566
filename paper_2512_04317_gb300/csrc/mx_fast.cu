// Dispatch of the register-resident MX pass by element format and block size.
#include <algorithm>
#include <cstring>

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
cudaError_t launch_ragged(const RaggedGroups& groups, const int4* ctas, int nctas, int dim,
                          size_t smem, cudaStream_t s);
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
    return a.fmt <= 4 && logm >= 0 && logm <= 6 && a.fp.mbits > 0 &&
           fast::fast_geometry(a.n, other, a.m, &TG, &S, &NG, &threads);
}

int fast_ng_candidates(int n, int other, int m, int* out, int max) {
    int TG, S, NG, threads;
    if (!fast::fast_geometry(n, other, m, &TG, &S, &NG, &threads)) return 0;
    const int per_group = TG * (n / 32);
    int c = 0;
    for (int ng = 1; per_group * ng <= fast::kMaxThreads && c < max; ng <<= 1) {
        const size_t smem = (size_t)ng * n * S * sizeof(float2);
        if (per_group * ng < 32 || other % (TG * ng) != 0 || smem > 227 * 1024) continue;
        out[c++] = ng;
    }
    return c;
}

namespace {
cudaError_t launch_fast(const PassArgs& a, const uint32_t* twh, const TwA& twa,
                        const uint32_t* twh2, const TwA* twa2, int batch, int ng, cudaStream_t s) {
    if (!fast_pass_supported(a)) return cudaErrorNotSupported;
    fast::FastArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.a = a;
    fa.twa = twa;
    fa.twh = twh;
    if (twa2) {
        fa.fused = 1;
        fa.twa2 = *twa2;
        fa.twh2 = twh2;
    }
    int threads;
    const int other = a.dim == 1 ? a.n0 : a.n1;
    fast::fast_geometry(a.n, other, a.m, &fa.TG, &fa.S, &fa.NG, &threads);
    fa.lgTG = fa.TG == 16 ? 4 : (fa.TG == 8 ? 3 : 2);
    if (ng == 0) ng = fast_ng_tuned(a.n, other, a.dim, a.fmt, a.m, batch);
    if (ng > 0) {
        int cand[16];
        const int nc = fast_ng_candidates(a.n, other, a.m, cand, 16);
        if (std::find(cand, cand + nc, ng) == cand + nc) return cudaErrorInvalidValue;
        fa.NG = ng;
    }
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
}  // namespace

// ---- ragged pass (mx_fast_ragged.cu): 256 threads per CTA for every group --

bool fast_ragged_geometry(int n, int other, int m, int* TG, int* S, int* NG) {
    if (m != 16 || n < 64 || n > 1024) return false;
    *TG = n == 1024 ? 8 : 16;
    *S = *TG == 16 ? 16 : *TG + 1;
    const int per_group = *TG * (n / 32);
    if (per_group > 256 || 256 % per_group) return false;
    *NG = 256 / per_group;
    return other % (*TG * *NG) == 0;
}

bool fast_ragged_supported(const PassArgs& a) {
    int TG, S, NG;
    const int other = a.dim == 1 ? a.n0 : a.n1;
    return a.fmt <= 4 && a.fp.mbits > 0 && fast_ragged_geometry(a.n, other, a.m, &TG, &S, &NG);
}

size_t fast_ragged_arg_size() { return sizeof(fast::FastArgs); }

bool fast_ragged_fill(void* dst, const PassArgs& a, const uint32_t* twh, const TwA& twa,
                      const uint32_t* twh2, const TwA* twa2, int* tpc, size_t* smem) {
    fast::FastArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    const int other = a.dim == 1 ? a.n0 : a.n1;
    if (!fast_ragged_geometry(a.n, other, a.m, &fa.TG, &fa.S, &fa.NG)) return false;
    fa.a = a;
    fa.twa = twa;
    fa.twh = twh;
    if (twa2) {
        fa.fused = 1;
        fa.twa2 = *twa2;
        fa.twh2 = twh2;
    }
    fa.lgTG = fa.TG == 16 ? 4 : 3;
    std::memcpy(dst, &fa, sizeof(fa));
    *tpc = fa.TG * fa.NG;
    *smem = (size_t)fa.NG * a.n * fa.S * sizeof(float2);
    return true;
}

int fast_ragged_max_groups() { return fast::kMaxRaggedGroups; }

cudaError_t launch_fast_ragged(const void* groups, int ngroups, const int4* ctas, int nctas, int dim,
                               size_t smem, cudaStream_t s) {
    if (ngroups < 1 || ngroups > fast::kMaxRaggedGroups) return cudaErrorInvalidValue;
    static thread_local fast::RaggedGroups rg;   // 24 KB: not on the stack
    rg.n = ngroups;
    std::memcpy(rg.g, groups, sizeof(fast::FastArgs) * (size_t)ngroups);
    return fast::launch_ragged(rg, ctas, nctas, dim, smem, s);
}

cudaError_t launch_fast_pass_ng(const PassArgs& a, const uint32_t* twh, const TwA& twa, int batch,
                                int ng, cudaStream_t s) {
    return launch_fast(a, twh, twa, nullptr, nullptr, batch, ng, s);
}

cudaError_t launch_fast_pass(const PassArgs& a, const uint32_t* twh, const TwA& twa, int batch,
                             cudaStream_t s) {
    return launch_fast(a, twh, twa, nullptr, nullptr, batch, 0, s);
}

cudaError_t launch_fast_pass_fused(const PassArgs& a, const uint32_t* twh, const TwA& twa,
                                   const uint32_t* twh_inv, const TwA& twa_inv, int batch,
                                   cudaStream_t s) {
    if (a.dim != 0) return cudaErrorInvalidValue;
    return launch_fast(a, twh, twa, twh_inv, &twa_inv, batch, 0, s);
}

}  // namespace mxfft
