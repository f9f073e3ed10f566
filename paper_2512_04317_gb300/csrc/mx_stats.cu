// Alg. 1 statistics pass: per slice, max |x|, the count of nonzero |x| and the
// histogram of floor(log2 |x|), then (last CTA of the slice) the prescale
// exponent k.  Reads each complex64 input once with 16-byte loads.
#include "mx_device.cuh"

namespace mxfft {

namespace {

constexpr int kStatsThreads = 256;

// Two points (one 16-byte load) into the accumulator: the same result as
// StatAcc::add_plain on each point.  When both lie in the fast range (each
// component zero or of magnitude in [2^-62, 2^63)) their squared magnitudes
// s = fl(fl(re^2) + fl(im^2)) are zero or normal and the bin is
// floor(floor(log2 s) / 2) + 149 = ((e + 171) >> 1) for s's biased exponent
// e in [1, 254]; as a byte offset into the histogram that is
// ((bits(s) >> 22) + 342) & ~3 (bits >> 22 is 2e plus s's top significand
// bit, which the mask drops).  The count of nonzero points is not kept here:
// every counted point adds one to exactly one bin, so it is the histogram's
// total.  The squares stay scalar: a packed multiply-then-add pair may be
// contracted into a fused multiply-add, which rounds differently.
__device__ __forceinline__ void add_two(StatAcc& acc, const float4 v, uint32_t* wh) {
    const uint32_t u0 = __float_as_uint(v.x) & 0x7fffffffu, u1 = __float_as_uint(v.y) & 0x7fffffffu;
    const uint32_t u2 = __float_as_uint(v.z) & 0x7fffffffu, u3 = __float_as_uint(v.w) & 0x7fffffffu;
    const uint32_t lo = (uint32_t)(127 - 62) << 23, hi = (uint32_t)(127 + 63) << 23;
    // (u - 1 wraps zero to the top, so "u == 0 or u >= lo" is one compare)
    const uint32_t mn = __vimin3_u32(u0 - 1u, u1 - 1u, min(u2 - 1u, u3 - 1u));
    const uint32_t mx = __vimax3_u32(u0, u1, max(u2, u3));
    if (mn >= lo - 1u && mx < hi) {
        const uint32_t s0 = __float_as_uint(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
        const uint32_t s1 = __float_as_uint(__fadd_rn(__fmul_rn(v.z, v.z), __fmul_rn(v.w, v.w)));
        acc.smax_bits = __vimax3_u32(acc.smax_bits, s0, s1);
        char* base = reinterpret_cast<char*>(wh);
        if (s0) atomicAdd(reinterpret_cast<uint32_t*>(base + (((s0 >> 22) + 342u) & ~3u)), 1u);
        if (s1) atomicAdd(reinterpret_cast<uint32_t*>(base + (((s1 >> 22) + 342u) & ~3u)), 1u);
    } else {
        acc.add_plain(v.x, v.y, wh);
        acc.add_plain(v.z, v.w, wh);
    }
}

// One CTA's share: points [chunk * kStatsPtsPerCta, +kStatsPtsPerCta) of a
// slice of npts points, then the flush into the slice's record.
__device__ __forceinline__ void stats_cta(const float2* __restrict__ x, int npts, int chunk,
                                          SliceStats* st, const KParams& kp, uint32_t ctas) {
    // one histogram per warp, lanes adding 1 each (no match), summed at the end
    __shared__ uint32_t sh_whist[kStatsThreads / 32][kHistBins];
    __shared__ uint32_t sh_hist[kHistBins];
    __shared__ uint32_t sh_misc[4];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int b = tid; b < kHistBins * (kStatsThreads / 32); b += blockDim.x) (&sh_whist[0][0])[b] = 0;
    __syncthreads();
    uint32_t* wh = sh_whist[warp];
    const float4* xs = reinterpret_cast<const float4*>(x);
    const int begin = chunk * kStatsPtsPerCta;
    const int end = min(begin + kStatsPtsPerCta, npts);
    StatAcc acc;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);   // zeros do not count
    // four 16-byte loads in flight per thread before any of them is used
    for (int base = begin; base < end; base += 8 * kStatsThreads) {
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int p = base + 2 * tid + 2 * kStatsThreads * j;   // even; end is even
            v[j] = p < end ? __ldg(xs + (p >> 1)) : zero;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) add_two(acc, v[j], wh);
    }
    __syncthreads();
    uint32_t counted = 0;
    for (int b = tid; b < kHistBins; b += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kStatsThreads / 32; w++) c += sh_whist[w][b];
        sh_hist[b] = c;
        counted += c;
    }
    acc.nnz = counted;   // the flush sums it over the CTA
    __syncthreads();
    stats_flush_and_select(acc, sh_hist, sh_misc, st, ctas, kp);
}

__global__ void __launch_bounds__(kStatsThreads, 8)
stats_kernel(const float2* __restrict__ x, int npts, SliceStats* __restrict__ st,
             KParams kp, uint32_t ctas_per_slice) {
    const int slice = blockIdx.y;
    stats_cta(x + (size_t)slice * npts, npts, blockIdx.x, st + slice, kp, ctas_per_slice);
}

__global__ void __launch_bounds__(kStatsThreads, 8)
stats_ref_kernel(const StatsRef* __restrict__ refs, const int2* __restrict__ cta_tab) {
    const int2 w = cta_tab[blockIdx.x];
    const StatsRef r = refs[w.x];
    stats_cta(r.x, r.npts, w.y, r.st, r.kp, r.ctas);
}

}  // namespace

cudaError_t launch_stats(const float2* x, int batch, int n0, int n1, SliceStats* st,
                         KParams kp, cudaStream_t s) {
    const int npts = n0 * n1;
    const uint32_t per = (uint32_t)((npts + kStatsPtsPerCta - 1) / kStatsPtsPerCta);
    dim3 grid(per, batch);
    stats_kernel<<<grid, kStatsThreads, 0, s>>>(x, npts, st, kp, per);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stats_ref(const StatsRef* refs, const int2* cta_tab, int nctas, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    stats_ref_kernel<<<nctas, kStatsThreads, 0, s>>>(refs, cta_tab);
    note_launch();
    return cudaGetLastError();
}

}  // namespace mxfft
