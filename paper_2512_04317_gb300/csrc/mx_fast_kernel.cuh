// The register-resident MX pass kernel (see mx_fast_impl.cuh for the layout)
// and its launcher, instantiated once per element format in mx_fast_f*.cu.
#pragma once

#include "mx_debug.cuh"
#include "mx_fast_impl.cuh"

namespace mxfft {
namespace fast {

constexpr int kMaxThreads = 512;

__device__ __forceinline__ float2 epi_value(float2 v, int mode, float post) {
    if (mode != EPI_RAW) {
        v.x = __fmul_rn(v.x, post);
        v.y = __fmul_rn(v.y, post);
    }
    return v;
}

// All stages of one transform per thread slot: phase A on the 32 elements in
// r (bit-reversed chunk order), then phase B through shared memory.  Returns
// with the last stage's results in R, element e0[q] + i in R[q][i] (natural
// order), and the group's shared rows holding an earlier stage.
template <int FMT, int LOGM>
__device__ __forceinline__ void all_stages(float2 (&r)[32], float2 (&R)[4][8], int (&e0)[4],
                                           float2* __restrict__ Gs, const TwA& twa,
                                           const uint32_t* __restrict__ twh,
                                           const int8_t* __restrict__ tws, int L, int S, int TG,
                                           int sigma, int tau, int s, const FmtParams& fp) {
    // ---- phase A: stages h = 1..16 inside the chunk -------------------------
    stage_a<FMT, LOGM, 1>(r, twa, fp, (unsigned)TG);
    stage_a<FMT, LOGM, 2>(r, twa, fp, (unsigned)TG);
    stage_a<FMT, LOGM, 4>(r, twa, fp, (unsigned)TG);
    stage_a<FMT, LOGM, 8>(r, twa, fp, (unsigned)TG);
    stage_a<FMT, LOGM, 16>(r, twa, fp, (unsigned)TG);
    const int gs_slots = (1 << L) * S;   // the group's shared rows
    (void)gs_slots;
#pragma unroll
    for (int t = 0; t < 32; t++) Gs[MX_BND((32 * sigma + t) * S + tau, gs_slots)] = r[t];
    __syncthreads();

    // ---- phase B: stage pairs (h, 2h), an odd last stage alone ---------------
    const unsigned red = (unsigned)TG;           // lane offset of the partner run (slot ^ 1)
    int ast = 5;
    while (true) {
        const int h = 1 << ast;
        const bool two = ast + 1 < L;
        int jA, jB, jC, jD;
        if (two) {
            const int Gi = sigma >> (ast - 3), rr = sigma & ((h >> 3) - 1);
            const int base = 4 * h * Gi + 8 * rr;
#pragma unroll
            for (int q = 0; q < 4; q++) e0[q] = base + q * h;
            jA = jB = 8 * rr;
            jC = 8 * rr;
            jD = h + 8 * rr;
        } else {
            e0[0] = 8 * sigma;
            e0[1] = 8 * sigma + h;
            e0[2] = 8 * (sigma + s);
            e0[3] = 8 * (sigma + s) + h;
            jA = 8 * sigma;
            jB = 8 * (sigma + s);
            jC = jD = 0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int i = 0; i < 8; i++) R[q][i] = Gs[MX_BND((e0[q] + i) * S + tau, gs_slots)];
        if (LOGM == 6 && h == 32) {
            // m = 64 > h: a block of stage 32 is both groups of the slot's runs,
            // a block of stage 64 the whole group (always a stage pair: n >= 128)
            stage_b_dual<FMT>(R[0], R[1], R[2], R[3], twh + h, tws + h - 1, jA, jB, red, fp);
            stage_b_dual<FMT>(R[0], R[2], R[1], R[3], twh + 2 * h, tws + 2 * h - 1, jC, jD, red, fp);
        } else {
            stage_b8<FMT, LOGM>(R[0], R[1], twh + h, tws + h - 1, jA, red, fp);
            stage_b8<FMT, LOGM>(R[2], R[3], twh + h, tws + h - 1, jB, red, fp);
            if (two) {
                stage_b8<FMT, LOGM>(R[0], R[2], twh + 2 * h, tws + 2 * h - 1, jC, red, fp);
                stage_b8<FMT, LOGM>(R[1], R[3], twh + 2 * h, tws + 2 * h - 1, jD, red, fp);
            }
        }
        ast += two ? 2 : 1;
        if (ast >= L) break;
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int i = 0; i < 8; i++) Gs[MX_BND((e0[q] + i) * S + tau, gs_slots)] = R[q][i];
        __syncthreads();
    }
}

// One CTA's work: transforms t0 .. t0 + TG NG - 1 of slice `slice`, all
// stages.  FUSED (columns only): forward, then inverse columns of the fused
// round trip (reading C17).
template <int FMT, int LOGM, int DIM, bool FUSED>
__device__ __forceinline__ void fast_body(const FastArgs& fa, const int slice, const int t0) {
    extern __shared__ float2 sm[];
    const PassArgs& a = fa.a;
    const int n = a.n, L = a.logn, TG = fa.TG, S = fa.S;
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int lgTG = fa.lgTG;
    const int lg_pg = lgTG + L - 5;              // log2 of threads per group
    const int grp = tid >> lg_pg;
    const int w = tid & ((1 << lg_pg) - 1);
    const int tau = w & (TG - 1);
    const int sigma = w >> lgTG;
    const int tr = t0 + (grp << lgTG) + tau;     // row (dim 1) or column (dim 0)
    float2* __restrict__ Gs = sm + (size_t)grp * n * S;
    const size_t sbase = (size_t)slice * a.n0 * a.n1;
    const float2* __restrict__ in = a.ref ? a.ref[slice].in : a.in + sbase;
    float2* __restrict__ out = a.ref ? a.ref[slice].out : a.out + sbase;
    const SliceStats* stp = a.ref ? a.ref[slice].st : a.st + slice;
    const FmtParams fp = a.fp;
    const size_t slice_pts = (size_t)a.n0 * a.n1;      // bounds of the debug build
    const size_t sm_slots = (size_t)fa.NG * n * S;
    (void)slice_pts;
    (void)sm_slots;

    const float pre = a.prologue == PRO_PRESCALE ? exp2i(stp->k) : 1.0f;
    const int s = n >> 5;                        // chunk stride of the bit-reversed gather
    const int rc = L > 5 ? (int)(__brev((unsigned)sigma) >> (37 - L)) : 0;

    // ---- phase A input: x[rc + j s] -> r[rev5(j)] ---------------------------
    float2 r[32];
    if (DIM == 0) {
#pragma unroll
        for (int j = 0; j < 32; j++) {
            float2 v = in[MX_BND((size_t)(rc + j * s) * a.n1 + tr, slice_pts)];
            if (a.prologue == PRO_PRESCALE) { v.x = __fmul_rn(v.x, pre); v.y = __fmul_rn(v.y, pre); }
            r[rev5(j)] = v;
        }
    } else {
        // stage the CTA's rows as [e][tau]: lanes run over rows, two lanes per
        // 16-byte pair, so each row contributes a full 32-byte sector per load.
        // The CTA's rows are NG * TG * n / 2 = 16 * threads float4: 16 per
        // thread, all in flight before the first store; the row of a thread's
        // float4 is fixed (threads is a multiple of TG)
        const int tc = tid & (TG - 1);
        const int r0 = tid >> lgTG, dr = nthr >> lgTG;
        float4 v[16];
#pragma unroll
        for (int b = 0; b < 16; b++) {
            const int rest = r0 + b * dr;
            const int p = rest & ((n >> 1) - 1);
            const int g = rest >> (L - 1);
            v[b] = __ldg(reinterpret_cast<const float4*>(
                in + MX_BND((size_t)(t0 + g * TG + tc) * a.n1 + 2 * p, slice_pts - 1)));
        }
#pragma unroll
        for (int b = 0; b < 16; b++) {
            const int rest = r0 + b * dr;
            const int p = rest & ((n >> 1) - 1);
            const int g = rest >> (L - 1);
            sm[MX_BND((size_t)g * n * S + (2 * p) * S + tc, sm_slots)] =
                make_float2(__fmul_rn(v[b].x, pre), __fmul_rn(v[b].y, pre));
            sm[MX_BND((size_t)g * n * S + (2 * p + 1) * S + tc, sm_slots)] =
                make_float2(__fmul_rn(v[b].z, pre), __fmul_rn(v[b].w, pre));
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 32; j++) r[rev5(j)] = Gs[MX_BND((rc + j * s) * S + tau, n * S)];
        __syncthreads();
    }

    float2 R[4][8];
    int e0[4];
    all_stages<FMT, LOGM>(r, R, e0, Gs, fa.twa, fa.twh, a.tws, L, S, TG, sigma, tau, s, fp);
    if (FUSED) {
        // the fused round trip's inverse columns on the same tile: the forward
        // result back to shared memory, gathered in bit-reversed chunk order
        // (as the row load does), then every stage with the inverse twiddles
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int i = 0; i < 8; i++) Gs[MX_BND((e0[q] + i) * S + tau, n * S)] = R[q][i];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 32; j++) r[rev5(j)] = Gs[MX_BND((rc + j * s) * S + tau, n * S)];
        __syncthreads();
        all_stages<FMT, LOGM>(r, R, e0, Gs, fa.twa2, fa.twh2, a.tws, L, S, TG, sigma, tau, s, fp);
    }

    // ---- output in natural order ---------------------------------------------
    float post = 1.0f;
    if (a.epilogue == EPI_UNSCALE) post = exp2i(-stp->k);
    else if (a.epilogue == EPI_RT_FINAL) post = exp2i(-stp->k - a.lg_total);
    if (DIM == 0) {
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int i = 0; i < 8; i++)
                out[MX_BND((size_t)(e0[q] + i) * a.n1 + tr, slice_pts)] = epi_value(R[q][i], a.epilogue, post);
    } else {
        // each run R[q] is 8 consecutive elements of this thread's own row:
        // four 16-byte stores per run, straight from registers
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                const float2 v0 = epi_value(R[q][i], a.epilogue, post);
                const float2 v1 = epi_value(R[q][i + 1], a.epilogue, post);
                *reinterpret_cast<float4*>(out + MX_BND((size_t)tr * a.n1 + e0[q] + i, slice_pts - 1)) =
                    make_float4(v0.x, v0.y, v1.x, v1.y);
            }
    }
}

// One launch of one plan's pass: CTA b takes the b-th run of TG NG
// transforms, slice by slice.
template <int FMT, int LOGM, int DIM, bool FUSED>
__global__ void __launch_bounds__(kMaxThreads)
fast_pass_kernel(const FastArgs fa) {
    const int other = DIM == 1 ? fa.a.n0 : fa.a.n1;
    const int tpc = fa.TG * fa.NG;
    const int per_slice = other / tpc;
    const int slice = blockIdx.x / per_slice;
    fast_body<FMT, LOGM, DIM, FUSED>(fa, slice, (blockIdx.x - slice * per_slice) * tpc);
}

// Launch geometry: TG transforms per group (8 for n = 2048 so a group fits in
// shared memory, and for m = 32 so that the four lanes of a block share a
// warp; 4 for m = 64, eight lanes; a padded stride then), NG groups per CTA so
// that a CTA has at least 128 threads (a group of n = 512 has 256, of n >=
// 1024 has 512, with TG = 16).  Small CTAs let four of them share an SM and
// drift apart, so one CTA's loads overlap another's arithmetic.  m = 32 needs
// n >= 128 (for n = 64 the last stage's block spans both of a lane's run
// pairs).
inline bool fast_geometry(int n, int other, int m, int* TG, int* S, int* NG, int* threads) {
    if (n < 64 || n > 2048 || m > 64 || (m == 32 && n < 128)) return false;
    *TG = m == 64 ? 4 : ((n == 2048 || m == 32) ? 8 : 16);
    *S = *TG == 16 ? 16 : *TG + 1;
    const int per_group = *TG * (n / 32);
    int ng = per_group >= 128 ? 1 : 128 / per_group;
    while (ng > 1 && (*TG * ng > other || other % (*TG * ng) != 0)) ng >>= 1;
    if (*TG > other || other % *TG != 0) return false;
    *NG = ng;
    *threads = per_group * ng;
    return *threads <= kMaxThreads;
}

template <int FMT, int DIM, bool FUSED>
cudaError_t launch_fast_dim(const FastArgs& fa, int logm, int blocks, int threads, size_t smem,
                            cudaStream_t s) {
    void (*k)(const FastArgs) = nullptr;
    switch (logm) {
        case 0: k = fast_pass_kernel<FMT, 0, DIM, FUSED>; break;
        case 1: k = fast_pass_kernel<FMT, 1, DIM, FUSED>; break;
        case 2: k = fast_pass_kernel<FMT, 2, DIM, FUSED>; break;
        case 3: k = fast_pass_kernel<FMT, 3, DIM, FUSED>; break;
        case 4: k = fast_pass_kernel<FMT, 4, DIM, FUSED>; break;
        case 5: k = fast_pass_kernel<FMT, 5, DIM, FUSED>; break;
        case 6: k = fast_pass_kernel<FMT, 6, DIM, FUSED>; break;
        default: return cudaErrorNotSupported;
    }
    // raise the opt-in limit only (never lower it): launches captured earlier
    // in a graph may need more than this one
    static size_t smem_limit[7] = {0, 0, 0, 0, 0, 0, 0};
    if (smem > smem_limit[logm]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_limit[logm] = smem;
    }
    k<<<blocks, threads, smem, s>>>(fa);
    note_launch();
    return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_fast_fmt(const FastArgs& fa, int logm, int batch, cudaStream_t s) {
    const PassArgs& a = fa.a;
    const int other = a.dim == 1 ? a.n0 : a.n1;
    const int threads = fa.TG * (a.n / 32) * fa.NG;
    const int blocks = batch * (other / (fa.TG * fa.NG));
    const size_t smem = (size_t)fa.NG * a.n * fa.S * sizeof(float2);
    if (fa.fused) {
        if (a.dim != 0) return cudaErrorInvalidValue;
        return launch_fast_dim<FMT, 0, true>(fa, logm, blocks, threads, smem, s);
    }
    return a.dim == 1 ? launch_fast_dim<FMT, 1, false>(fa, logm, blocks, threads, smem, s)
                      : launch_fast_dim<FMT, 0, false>(fa, logm, blocks, threads, smem, s);
}

}  // namespace fast
}  // namespace mxfft
