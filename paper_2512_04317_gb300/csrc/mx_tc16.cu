// Tensor-core variant of the MX pass: radix-16 sub-DFTs as MXFP8 matrix
// products on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulation
// in tensor memory), for transform lengths n = 256 r, r in {1, 2}.
//
// Decomposition (four-step, rows of a transform viewed as 16 x M, M = 16 r):
//   j = M j1 + j2, k = k1 + 16 k2
//   A : Y[k1][j2] = W_n^(j2 k1) * DFT16_j1(x[M j1 + j2])[k1]
//   C1: for each k1, 16-point DFTs over j21 of Y[k1][r j21 + j22] (j22 < r),
//       times W_M^(j22 k21) when r > 1
//   C2: r-point DFT over j22 (r = 2: a sum and a difference, FP32)
//   X[k1 + 16 (k21 + 16 k22)]
// Every 16-point input vector (32 reals) is one MX block: shared power-of-two
// scale 2^s from its largest component, elements rounded to the 8-bit format
// (cvt.rn.satfinite).  The real 32 x 32 DFT matrix is prequantised with one
// shared scale per output row.  One tcgen05.mma (M = 128 vectors, N = 32, K =
// 32, kind::f8f6f4) multiplies 128 vectors; because K is one block, the two
// power-of-two scales factor out of the dot product and are applied exactly
// to the FP32 result when it is read back (tcgen05.ld).  Twiddles are MX
// element values (one block per 16 twiddles) multiplied in FP32.
//
// A CTA (128 threads) owns T = 8 transforms in shared memory; thread i owns
// row i of the MMA (one vector) in every round.  The only wait is on the MMA
// completion mbarrier, with an iteration limit: on time-out the kernel sets
// the plan's error flag, waits once more (bounded) for its own MMA, frees its
// tensor memory and finishes without using the result.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mx_device.cuh"

namespace mxfft {
namespace tc16 {

constexpr int kThreads = 128;
constexpr int kT = 8;                 // transforms per CTA
constexpr uint32_t kTmemCols = 32;
constexpr int kWaitLimit = 1 << 22;

using Args = Tc16Args;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major without swizzle: an 8-row x 16-byte
// core matrix is contiguous; K-adjacent core matrices are LBO bytes apart,
// row-group-adjacent ones SBO bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

template <int FMT> __device__ __forceinline__ uint16_t enc2(float lo, float hi);
template <> __device__ __forceinline__ uint16_t enc2<0>(float lo, float hi) {
    unsigned short p;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(p) : "f"(hi), "f"(lo));
    return p;
}
template <> __device__ __forceinline__ uint16_t enc2<1>(float lo, float hi) {
    unsigned short p;
    asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(p) : "f"(hi), "f"(lo));
    return p;
}

__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Padded shared index of element e: 16-element groups are 17 slots apart and
// transforms TS = n + n/16 + 2 slots apart (TS = 2 mod 16).  With 8-byte slots
// and 32 four-byte banks, every access pattern of the kernel (16 lanes on
// consecutive elements; 16 lanes on one element of 16 consecutive groups;
// 8 transforms x 2 groups; 4 transforms x 4 consecutive elements) then touches
// 16 distinct slots modulo 16, i.e. no bank conflicts.
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
__host__ __device__ constexpr int tstride(int n) { return n + n / 16 + 2; }

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitLimit && !done; it++) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
                     " selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(mbar), "r"(phase));
    }
    return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&d)[32]) {
    uint32_t v[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                   "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                   "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int c = 0; c < 32; c++) d[c] = __uint_as_float(v[c]);
}

// One MMA round: every thread MX-encodes its 16-element vector into row tid of
// the A operand, one thread issues the product, all read back their row.
// Returns the 16 complex DFT outputs (scales applied) in y.
template <int FMT>
__device__ __forceinline__ void dft16_round(const float2 (&x)[16], float2 (&y)[16], uint8_t* sA,
                                            uint32_t sa_u32, uint32_t sb_u32, uint32_t mbar,
                                            uint32_t tbase, uint32_t& phase, bool& ok,
                                            const Args& a, const FmtParams& fp) {
    const int tid = threadIdx.x, warp = tid >> 5;
    float m[16];
#pragma unroll
    for (int j = 0; j < 16; j++) m[j] = fmax_nan(fabsf(x[j].x), fabsf(x[j].y));
#pragma unroll
    for (int w = 1; w < 16; w <<= 1)
#pragma unroll
        for (int j = 0; j + w < 16; j += 2 * w) m[j] = fmax_nan(m[j], m[j + w]);
    const float A = m[0];
    const bool bad = !(A <= 3.402823466e38f);
    const int sv = mx_scale_exp(__float_as_uint(A), fp.emax);
    const float inv = exp2i(-sv);
    uint32_t w32[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t lo = enc2<FMT>(__fmul_rn(x[2 * j].x, inv), __fmul_rn(x[2 * j].y, inv));
        const uint32_t hi = enc2<FMT>(__fmul_rn(x[2 * j + 1].x, inv), __fmul_rn(x[2 * j + 1].y, inv));
        w32[j] = lo | (hi << 16);
    }
    // row tid: K bytes 0..15 in core matrix (tid / 8, 0), 16..31 in (tid / 8, 1)
    uint4* r0 = reinterpret_cast<uint4*>(sA + (tid >> 3) * 256 + (tid & 7) * 16);
    uint4* r1 = reinterpret_cast<uint4*>(sA + (tid >> 3) * 256 + 128 + (tid & 7) * 16);
    *r0 = make_uint4(w32[0], w32[1], w32[2], w32[3]);
    *r1 = make_uint4(w32[4], w32[5], w32[6], w32[7]);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
        const uint64_t ad = smem_desc(sa_u32, 128, 256);
        const uint64_t bd = smem_desc(sb_u32, 128, 256);
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;"
                     " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                     :: "r"(tbase), "l"(ad), "l"(bd), "r"(a.idesc), "r"(0));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mbar));
    }
    // tcgen05.ld below is warp-collective: the warp reads only if every lane saw
    // the product complete
    const bool done = __all_sync(0xffffffffu, wait_phase(mbar, phase));
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float d[32];
    if (done) {
        tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16), d);
    } else {
#pragma unroll
        for (int c = 0; c < 32; c++) d[c] = 0.f;
        ok = false;
    }
    // D is exact-scaled by the vector's scale and the matrix rows' scale, which
    // is 2^-emax for every row (each row holds an entry of magnitude 1)
    const float sc = bad ? __int_as_float(0x7fffffff) : exp2i(sv - fp.emax);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        y[k].x = __fmul_rn(d[2 * k], sc);
        y[k].y = __fmul_rn(d[2 * k + 1], sc);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();   // A and D may be reused once every row has been read
}

__device__ __forceinline__ float2 cmul(float2 w, float2 y) {
    return make_float2(__fsub_rn(__fmul_rn(w.x, y.x), __fmul_rn(w.y, y.y)),
                       __fadd_rn(__fmul_rn(w.x, y.y), __fmul_rn(w.y, y.x)));
}

__device__ __forceinline__ float2 scale2(float2 v, float s) {
    return make_float2(__fmul_rn(v.x, s), __fmul_rn(v.y, s));
}

template <int FMT, int DIM, int LOGN>
__global__ void __launch_bounds__(kThreads)
tc16_pass_kernel(const Args a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t* sA = smem;                                   // 4 KB A operand
    uint8_t* sB = smem + 4096;                            // 1 KB B operand
    float2* data = reinterpret_cast<float2*>(smem + 5120);
    constexpr int n = 1 << LOGN, r = n / 256, M = 16 * r;
    constexpr int TS = tstride(n);                        // padded transform stride (slots)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int other = DIM == 1 ? a.n0 : a.n1;
    const int per_slice = other / kT;
    const int slice = blockIdx.x / per_slice;
    const int t0 = (blockIdx.x - slice * per_slice) * kT;
    const size_t sbase = (size_t)slice * a.n0 * a.n1;
    const float2* __restrict__ in = a.in + sbase;
    float2* __restrict__ out = a.out + sbase;
    FmtParams fp;
    fp.emax = FMT == 0 ? 8 : 15;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 64) reinterpret_cast<uint4*>(sB)[tid] = __ldg(reinterpret_cast<const uint4*>(a.bmat) + tid);

    // ---- tile in: kT transforms, padded [t][e] layout, prescale on the first pass
    const float pre = a.prologue == PRO_PRESCALE ? exp2i(a.st[slice].k) : 1.0f;
    // (kT n / 2 = 1024 n / 256 float4 per CTA: a multiple of 8 x 128 threads)
    const int quads = kT * (n >> 1);
    for (int u0 = tid; u0 < quads; u0 += 8 * kThreads) {
        float4 v[8];
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const int u = u0 + b * kThreads;
            const float4* src;
            if (DIM == 1) {
                const int t = u / (n >> 1), e = 2 * (u - t * (n >> 1));
                src = reinterpret_cast<const float4*>(in + (size_t)(t0 + t) * a.n1 + e);
            } else {
                const int e = u / (kT >> 1), t = 2 * (u - e * (kT >> 1));
                src = reinterpret_cast<const float4*>(in + (size_t)e * a.n1 + t0 + t);
            }
            v[b] = __ldg(src);
        }
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const int u = u0 + b * kThreads;
            const float2 lo = make_float2(__fmul_rn(v[b].x, pre), __fmul_rn(v[b].y, pre));
            const float2 hi = make_float2(__fmul_rn(v[b].z, pre), __fmul_rn(v[b].w, pre));
            if (DIM == 1) {
                const int t = u / (n >> 1), e = 2 * (u - t * (n >> 1));
                data[t * TS + pidx(e)] = lo;
                data[t * TS + pidx(e + 1)] = hi;
            } else {
                const int e = u / (kT >> 1), t = 2 * (u - e * (kT >> 1));
                data[t * TS + pidx(e)] = lo;
                data[(t + 1) * TS + pidx(e)] = hi;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    const uint32_t sa_u32 = smem_u32(sA), sb_u32 = smem_u32(sB), mb = smem_u32(&mbar);
    uint32_t phase = 0;
    bool ok = true;

    // ---- round A: vectors (t, j2), 16 elements x[M j1 + j2] ------------------
    const int nvec = kT * M;
    for (int v0 = 0; v0 < nvec; v0 += kThreads) {
        const int v = v0 + tid;
        int t, j2;
        if (DIM == 1) { t = v / M; j2 = v - t * M; } else { j2 = v / kT; t = v - j2 * kT; }
        float2* d = data + t * TS;
        float2 x[16], y[16];
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = d[pidx(M * j + j2)];
        dft16_round<FMT>(x, y, sA, sa_u32, sb_u32, mb, tbase, phase, ok, a, fp);
        const float4* tw = reinterpret_cast<const float4*>(a.twA + j2 * 16);
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            const float4 w = __ldg(tw + (k >> 1));
            d[pidx(M * k + j2)] = cmul(make_float2(w.x, w.y), y[k]);
            d[pidx(M * (k + 1) + j2)] = cmul(make_float2(w.z, w.w), y[k + 1]);
        }
    }
    __syncthreads();

    // ---- round C1: vectors (t, k1, j22), 16 elements Y[M k1 + r j21 + j22] ---
    float post = 1.0f;
    if (a.epilogue == EPI_UNSCALE) post = exp2i(-a.st[slice].k);
    else if (a.epilogue == EPI_RT_FINAL) post = exp2i(-a.st[slice].k - a.lg_total);
    const bool scale_out = a.epilogue != EPI_RAW;
    for (int v0 = 0; v0 < nvec; v0 += kThreads) {
        const int v = v0 + tid;
        int t, k1, j22;
        if (DIM == 1) {
            t = v / M;
            const int rem = v - t * M;
            k1 = rem / r;
            j22 = rem - k1 * r;
        } else {
            t = v % kT;
            const int rem = v / kT;
            k1 = rem / r;
            j22 = rem - k1 * r;
        }
        float2* d = data + t * TS;
        float2 x[16], y[16];
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = d[pidx(M * k1 + r * j + j22)];
        dft16_round<FMT>(x, y, sA, sa_u32, sb_u32, mb, tbase, phase, ok, a, fp);
        if (r == 1) {
            // X[k1 + 16 k2]
#pragma unroll
            for (int k = 0; k < 16; k++) {
                float2 val = scale_out ? scale2(y[k], post) : y[k];
                const int e = k1 + 16 * k;
                if (DIM == 1) out[(size_t)(t0 + t) * a.n1 + e] = val;
                else out[(size_t)e * a.n1 + t0 + t] = val;
            }
        } else {
            const float4* tw = reinterpret_cast<const float4*>(a.twC + j22 * 16);
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float4 w = __ldg(tw + (k >> 1));
                d[pidx(M * k1 + r * k + j22)] = cmul(make_float2(w.x, w.y), y[k]);
                d[pidx(M * k1 + r * (k + 1) + j22)] = cmul(make_float2(w.z, w.w), y[k + 1]);
            }
        }
    }
    if (r == 2) {
        __syncthreads();
        // ---- C2: radix-2 over j22: X[k1 + 16 (k21 + 16 k22)] ---------------
        const int items = kT * 256;   // (t, k1, k21)
        for (int u = tid; u < items; u += kThreads) {
            int t, k1, k21;
            if (DIM == 1) { t = u >> 8; k21 = (u >> 4) & 15; k1 = u & 15; }
            else { t = u & (kT - 1); k1 = (u >> 3) & 15; k21 = u >> 7; }
            const float2* d = data + t * TS;
            const float2 p = d[pidx(M * k1 + 2 * k21)], q = d[pidx(M * k1 + 2 * k21 + 1)];
            float2 s0 = make_float2(__fadd_rn(p.x, q.x), __fadd_rn(p.y, q.y));
            float2 s1 = make_float2(__fsub_rn(p.x, q.x), __fsub_rn(p.y, q.y));
            if (scale_out) { s0 = scale2(s0, post); s1 = scale2(s1, post); }
            const int e0 = k1 + 16 * k21, e1 = e0 + 256;
            if (DIM == 1) {
                out[(size_t)(t0 + t) * a.n1 + e0] = s0;
                out[(size_t)(t0 + t) * a.n1 + e1] = s1;
            } else {
                out[(size_t)e0 * a.n1 + t0 + t] = s0;
                out[(size_t)e1 * a.n1 + t0 + t] = s1;
            }
        }
    }

    // ---- teardown: an abandoned product is waited for once more, then the
    // tensor memory is returned
    if (!ok) {
        wait_phase(mb, phase ^ 1u);
        if ((tid & 31) == 0) atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols));
}

template <int FMT>
cudaError_t launch_fmt(const Args& a, int batch, cudaStream_t s) {
    const int other = a.dim == 1 ? a.n0 : a.n1;
    const int blocks = batch * (other / kT);
    const size_t smem = 5120 + (size_t)kT * tstride(a.n) * sizeof(float2);
    void (*k)(const Args);
    if (a.n == 256) k = a.dim == 1 ? tc16_pass_kernel<FMT, 1, 8> : tc16_pass_kernel<FMT, 0, 8>;
    else k = a.dim == 1 ? tc16_pass_kernel<FMT, 1, 9> : tc16_pass_kernel<FMT, 0, 9>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tc16

bool tc16_supported(int n, int other, int fmt) {
    // n = 256 r (r = 1, 2), 8-bit element formats, whole CTAs of kT transforms
    return (n == 256 || n == 512) && other >= tc16::kT && other % tc16::kT == 0 && (fmt == 0 || fmt == 1);
}

cudaError_t launch_tc16_pass(const Tc16Args& a, int fmt, int batch, cudaStream_t s) {
    if (fmt == 0) return tc16::launch_fmt<0>(a, batch, s);
    if (fmt == 1) return tc16::launch_fmt<1>(a, batch, s);
    return cudaErrorNotSupported;
}

}  // namespace mxfft
