// Alg. 1 statistics pass: per slice, max |x|, the count of nonzero |x| and the
// histogram of floor(log2 |x|), then (last CTA of the slice) the prescale
// exponent k.  Reads each complex64 input once with 16-byte loads.
#include "mx_device.cuh"

namespace mxfft {

namespace {

constexpr int kStatsThreads = 256;

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
    for (int base = begin; base < end; base += 4 * blockDim.x) {
        const int p0 = base + 2 * tid, p1 = p0 + 2 * blockDim.x;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);   // zeros do not count
        const float4 v0 = p0 < end ? __ldg(xs + (p0 >> 1)) : zero;
        const float4 v1 = p1 < end ? __ldg(xs + (p1 >> 1)) : zero;
        acc.add_plain(v0.x, v0.y, wh);
        acc.add_plain(v0.z, v0.w, wh);
        acc.add_plain(v1.x, v1.y, wh);
        acc.add_plain(v1.z, v1.w, wh);
    }
    __syncthreads();
    for (int b = tid; b < kHistBins; b += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kStatsThreads / 32; w++) c += sh_whist[w][b];
        sh_hist[b] = c;
    }
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
