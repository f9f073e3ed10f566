// Fused 2D transform of the tensor-core variant for n0, n1 in {256, 512}: the
// whole slice stays on chip, spread over one thread-block cluster, from the
// statistics of Alg. 1 through the row and column passes, so every point
// crosses HBM once in and once out per transform (16 B per point).
//
// Per slice (a cluster of C = n0 n1 / 16384 CTAs walks slices cl, cl + ncl, ...):
//   1. CTA c loads its slab, rows [R c, R c + R) (R = 16384 / n1, 128 KB),
//      with bulk copies into a padded row layout.
//   2. Alg. 1 statistics: each CTA accumulates |x| maxima, the nonzero count
//      and the exponent histogram of its slab (StatAcc, the statistics
//      kernel's arithmetic), the cluster adds the records through distributed
//      shared memory and every CTA selects the same k (the exact integer
//      selection of the statistics kernel).
//   3. Rows: four tiles of 4096 points per CTA, each the radix-16 rounds of
//      the tensor-core pass (A, C1 and for n1 = 512 the radix-2 step C2) on
//      the prescaled slab, results back into the slab in natural order.
//   4. Columns: CTA c owns columns [Cc c, Cc c + Cc) (Cc = n1 / C) as four
//      tiles of 4096 / n0 columns; each tile is gathered from the slabs of
//      all C CTAs (distributed shared memory, 16-byte loads) into a staging
//      tile, transformed by the same rounds, and stored to HBM with the
//      epilogue scaling.  The slabs are free after the last gather, so the
//      next slice's bulk copies start before the last column tile is done.
// Arithmetic per element is that of the tensor-core pass kernel (mx_tc16.cu)
// rewritten with packed FP32 pairs: the block scale, the 8-bit encode, FP32
// accumulation of 32 exact products in tensor memory, the scales applied to
// the result, twiddles multiplied in FP32 with separately rounded products.
// A twiddle multiply is packed: the products w.re (re, im) and (-w.im, w.im)
// (im, re) of the unscaled accumulator pair, each times the exact power-of-
// two scale, then one add; in the normal range that gives the bits of the
// pass kernel's scale-then-multiply order.  The scale is applied to each
// product before the add on purpose: the code generator may merge a multiply
// into the add that follows it (a fused multiply-add rounds once), and only
// a product by a power of two is exact, so that merge cannot change a bit.
// (The (im, re) pair is taken from the same accumulator registers: a second
// set of B columns with re and im swapped would recompute each dot product,
// and the tensor core need not round the two computations alike.)
//
// Waits: the MMA completion and the slab copies are bounded (100 ms each by
// the global timer); after a time-out the CTA records the error, issues no
// further products, skips the remaining waits and still takes part in every
// cluster barrier, so the cluster finishes; outputs of such a call are
// undefined.  Before it exits a CTA waits once more (bounded) for anything of
// its own still in flight and frees its tensor memory.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mx_debug.cuh"
#include "mx_device.cuh"
#include "mx_tcgen05.cuh"

namespace mxfft {
namespace tc2d {

using namespace tcg;

constexpr int kThreads = 256;
constexpr int kTilePts = 4096;        // points per tile = 256 vectors x 16
constexpr int kSlabPts = 16384;       // points per CTA
constexpr uint32_t kTmemCols = 64;    // two 128 x 32 FP32 accumulators
constexpr int kTwRow = 17;            // float4 slots per twiddle row (16 + 1 pad)

// One axis of length n = 2^LOGN in {256, 512}.
template <int LOGN>
struct Ax {
    static constexpr int n = 1 << LOGN;
    static constexpr int r = n / 256;          // 1 or 2
    static constexpr int LGR = r == 1 ? 0 : 1;
    static constexpr int M = 16 * r;
    static constexpr int LGM = 4 + LGR;
    static constexpr int T = kTilePts / n;     // transforms per tile: 16 or 8
    static constexpr int LGT = T == 16 ? 4 : 3;
    static constexpr int PADR = 2;             // pad slots after every M elements of a row
    static constexpr int TS = n + PADR * (n / M);
};

constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

template <int LOGN0, int LOGN1>
struct Geo {
    using A0 = Ax<LOGN0>;   // columns: transforms of length n0
    using A1 = Ax<LOGN1>;   // rows: transforms of length n1
    static constexpr int n0 = A0::n, n1 = A1::n;
    static constexpr int C = n0 * n1 / kSlabPts;     // CTAs per cluster: 4, 8 or 16
    static constexpr int R = kSlabPts / n1;          // slab rows
    static constexpr int Cc = n1 / C;                // columns per CTA
    static constexpr int ROW_TILES = R / A1::T;
    static constexpr int COL_TILES = Cc / A0::T;
    static constexpr int SLAB_SLOTS = R * A1::TS;
    static constexpr int STG_SLOTS = n0 * A0::T + (A0::T < 16 ? A0::T * (n0 / 16) : 0);
    // dynamic shared memory (bytes)
    static constexpr int OFF_A = 0;                                   // A operand, 2 x 4 KB
    static constexpr int OFF_B = 8192;                                // B operand, 32 x 32 B
    static constexpr int OFF_TWA1 = OFF_B + 1024;
    static constexpr int OFF_TWC1 = OFF_TWA1 + A1::M * kTwRow * 16;
    static constexpr int OFF_TWA0 = OFF_TWC1 + A1::r * kTwRow * 16;
    static constexpr int OFF_TWC0 = OFF_TWA0 + A0::M * kTwRow * 16;
    static constexpr int OFF_REC = OFF_TWC0 + A0::r * kTwRow * 16;    // statistics record
    static constexpr int REC_WORDS = 4 + 280;
    static constexpr int OFF_SLAB = align_up(OFF_REC + REC_WORDS * 4, 128);
    static constexpr int OFF_STG = OFF_SLAB + SLAB_SLOTS * 8;
    static constexpr int SMEM = OFF_STG + STG_SLOTS * 8;
    static_assert(ROW_TILES == 4 && COL_TILES == 4, "four row and four column tiles per CTA");
    static_assert(C * R == n0 && C * Cc == n1, "slabs cover the slice");
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert(STG_SLOTS * 8 >= REC_WORDS * 4, "the staging tile holds the cluster totals");
};

// Slot (8 bytes) of element e of row t in the slab's row layout; the row
// pass's rounds and the natural-order results use it (see mx_tc16.cu for the
// bank analysis of each access pattern).
template <class A>
__device__ __forceinline__ int slot_row(int t, int e) {
    return t * A::TS + e + A::PADR * (e >> A::LGM);
}
// Slot of element e of column t in a staging tile of A::T columns.
template <class A>
__device__ __forceinline__ int slot_col(int t, int e) {
    return e * A::T + (A::T < 16 ? A::T * (e >> 4) : 0) + t;
}

// MMA state of a CTA.
struct Mma {
    uint8_t* sA;
    uint32_t sa, sb, mbar, tbase, phase;
    bool ok;         // no wait has timed out
    bool pending;    // a product was issued and its completion not seen
};

// One radix-16 round on 256 vectors (thread i: vector i, operand half i / 128,
// row i % 128): MX-encode x (shared scale 2^sv from the largest component,
// elements rounded by cvt.rn.satfinite), one thread issues both products
// against the DFT operand, every thread reads its row back.  d gets the 32
// outputs (re, im interleaved), unscaled; returns the exact scale 2^(sv -
// emax) (NaN for a block holding Inf/NaN).  A CTA barrier inside orders every
// thread's reads of its round inputs before any thread's writes of the
// results.
template <int FMT>
__device__ __forceinline__ float round_mma(const float2 (&x)[16], float (&d)[32], Mma& mm,
                                           uint32_t idesc, int emax, bool issue) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const float A = vec_max_abs(x);
    const bool bad = !(A <= 3.402823466e38f);
    const int sv = mx_scale_exp(__float_as_uint(A), emax);
    const float inv = exp2i(-sv);
    const float2 inv2 = make_float2(inv, inv);
    uint32_t w32[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float2 a = mul2_rn(x[2 * j], inv2);
        const float2 b = mul2_rn(x[2 * j + 1], inv2);
        w32[j] = (uint32_t)enc2<FMT>(a.x, a.y) | ((uint32_t)enc2<FMT>(b.x, b.y) << 16);
    }
    // row rr of half h: K bytes 0..15 in core matrix (rr / 8, 0), 16..31 in (rr / 8, 1)
    const int h = tid >> 7, rr = tid & 127;
    uint8_t* row = mm.sA + h * 4096 + (rr >> 3) * 256 + (rr & 7) * 16;
    *reinterpret_cast<uint4*>(row) = make_uint4(w32[0], w32[1], w32[2], w32[3]);
    *reinterpret_cast<uint4*>(row + 128) = make_uint4(w32[4], w32[5], w32[6], w32[7]);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool go = issue && mm.ok;
    if (tid == 0 && go) {
        const uint64_t bd = smem_desc(mm.sb, 128, 256);
        const uint64_t a0 = smem_desc(mm.sa, 128, 256);
        const uint64_t a1 = smem_desc(mm.sa + 4096, 128, 256);
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;"
                     " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                     :: "r"(mm.tbase), "l"(a0), "l"(bd), "r"(idesc), "r"(0));
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;"
                     " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                     :: "r"(mm.tbase + 32u), "l"(a1), "l"(bd), "r"(idesc), "r"(0));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mm.mbar));
    }
    bool done = false;
    if (mm.ok) {
        // warp 0 waits, the others sleep on the CTA barrier; with the test
        // hook nothing was issued, so the bounded wait runs out
        done = wait_phase_cta(mm.mbar, mm.phase);
        if (go) {
            mm.phase ^= 1u;
            mm.pending = !done;
        }
    }
    if (!done) mm.ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
        // warp w reads lanes 32 (w % 4) .. of accumulator w / 4
        tmem_ld32(mm.tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * 32), d);
    } else {
#pragma unroll
        for (int c = 0; c < 32; c++) d[c] = 0.f;
    }
    // D is exact-scaled by the vector's scale and the matrix rows' scale 2^-emax
    return bad ? __int_as_float(0x7fffffff) : exp2i(sv - emax);
}

// Output k of a round times twiddle w = (w.re, w.re, -w.im, w.im), with the
// exact scale: (w.re re - w.im im, w.re im + w.im re) sc, each product
// rounded, scaled exactly, then added (see above).
__device__ __forceinline__ float2 tw_out(const float (&d)[32], int k, float4 w, float2 sc2) {
    const float2 p1 = mul2_rn(mul2_rn(make_float2(d[2 * k], d[2 * k + 1]), make_float2(w.x, w.y)), sc2);
    const float2 p2 = mul2_rn(mul2_rn(make_float2(d[2 * k + 1], d[2 * k]), make_float2(w.z, w.w)), sc2);
    return add2_rn(p1, p2);
}
__device__ __forceinline__ float2 plain_out(const float (&d)[32], int k, float2 sc2) {
    return mul2_rn(make_float2(d[2 * k], d[2 * k + 1]), sc2);
}

// Slice buffers.
__device__ __forceinline__ void resolve(const Tc2dArgs& a, int slice, const float2** in, float2** out,
                                        SliceStats** st) {
    if (a.ref) {
        const SliceRef r = a.ref[slice];
        *in = r.in;
        *out = r.out;
        *st = r.st;
    } else {
        const size_t b = (size_t)slice * a.n0 * a.n1;
        *in = a.in + b;
        *out = a.out + b;
        *st = a.st + slice;
    }
}

// Bulk copies of this CTA's slab of a slice (rows R rank .. + R) into the
// padded row layout: one copy per run of M elements.  Thread 0 arms the
// barrier with the slab's bytes first.
template <class G>
__device__ __forceinline__ void load_slab(const float2* in, uint32_t rank, uint32_t slab_u32,
                                          uint32_t mbar) {
    using A1 = typename G::A1;
    constexpr int RUNS = G::R * (A1::n / A1::M);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(mbar, (uint32_t)(kSlabPts * 8));
    __syncthreads();
    // earlier generic-proxy accesses of the slab before the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const float2* src = in + (size_t)rank * G::R * A1::n;
    for (int q = threadIdx.x; q < RUNS; q += kThreads) {
        const int row = q / (A1::n / A1::M), run = q % (A1::n / A1::M);
        bulk_g2s(slab_u32 + 8u * (uint32_t)MX_BND(slot_row<A1>(row, run * A1::M), G::SLAB_SLOTS - A1::M + 1),
                 src + (size_t)row * A1::n + run * A1::M, (uint32_t)(A1::M * 8), mbar);
    }
}

template <int FMT, int LOGN0, int LOGN1>
__global__ void __launch_bounds__(kThreads, 1)
tc2d_kernel(const Tc2dArgs a) {
    using G = Geo<LOGN0, LOGN1>;
    using A0 = typename G::A0;
    using A1 = typename G::A1;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar_mma;
    __shared__ __align__(8) uint64_t mbar_ld;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_k;

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t rank = cluster_ctarank();
    const int clus = (int)cluster_idx(), nclus = (int)cluster_count();
    const int emax = FMT == 0 ? 8 : 15;
    float2* slab = reinterpret_cast<float2*>(smem + G::OFF_SLAB);
    float2* stg = reinterpret_cast<float2*>(smem + G::OFF_STG);
    uint32_t* rec = reinterpret_cast<uint32_t*>(smem + G::OFF_REC);
    const float4* twA1 = reinterpret_cast<const float4*>(smem + G::OFF_TWA1);
    const float4* twC1 = reinterpret_cast<const float4*>(smem + G::OFF_TWC1);
    const float4* twA0 = reinterpret_cast<const float4*>(smem + G::OFF_TWA0);
    const float4* twC0 = reinterpret_cast<const float4*>(smem + G::OFF_TWC0);
    // slab and staging slots, checked in the debug build
    auto srow = [](int t, int e) { return (int)MX_BND(slot_row<A1>(t, e), G::SLAB_SLOTS); };
    auto scol = [](int t, int e) { return (int)MX_BND(slot_col<A0>(t, e), G::STG_SLOTS); };
    const size_t slice_pts = (size_t)G::n0 * G::n1;
    (void)slice_pts;
    const uint32_t slab_u32 = smem_u32(slab);
    const uint32_t rec_u32 = smem_u32(rec);
    const uint32_t ldb = smem_u32(&mbar_ld);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar_mma), 1);
        mbar_init(ldb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // operand B and the twiddle tables
    if (tid < 64)
        reinterpret_cast<uint4*>(smem + G::OFF_B)[tid] = __ldg(reinterpret_cast<const uint4*>(a.bmat) + tid);
    {
        float4* t = reinterpret_cast<float4*>(smem + G::OFF_TWA1);
        for (int i = tid; i < A1::M * 16; i += kThreads) t[(i >> 4) * kTwRow + (i & 15)] = __ldg(a.twA1 + i);
        t = reinterpret_cast<float4*>(smem + G::OFF_TWC1);
        for (int i = tid; i < A1::r * 16; i += kThreads) t[(i >> 4) * kTwRow + (i & 15)] = __ldg(a.twC1 + i);
        t = reinterpret_cast<float4*>(smem + G::OFF_TWA0);
        for (int i = tid; i < A0::M * 16; i += kThreads) t[(i >> 4) * kTwRow + (i & 15)] = __ldg(a.twA0 + i);
        t = reinterpret_cast<float4*>(smem + G::OFF_TWC0);
        for (int i = tid; i < A0::r * 16; i += kThreads) t[(i >> 4) * kTwRow + (i & 15)] = __ldg(a.twC0 + i);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    Mma mm;
    mm.sA = smem + G::OFF_A;
    mm.sa = smem_u32(smem + G::OFF_A);
    mm.sb = smem_u32(smem + G::OFF_B);
    mm.mbar = smem_u32(&mbar_mma);
    mm.tbase = tmem_base;
    mm.phase = 0;
    mm.ok = true;
    mm.pending = false;
    uint32_t ld_phase = 0;
    bool ld_ok = true, ld_pending = false;
    const bool issue = !a.stall;

    // every CTA of a cluster walks the same slices: cluster cl takes cl, cl + ncl, ...
    if (clus < a.batch) {
        const float2* in0;
        float2* out0;
        SliceStats* st0;
        resolve(a, clus, &in0, &out0, &st0);
        load_slab<G>(in0, rank, slab_u32, ldb);
        ld_pending = true;
    }
    for (int sl = clus; sl < a.batch; sl += nclus) {
        const float2* in;
        float2* out;
        SliceStats* st;
        resolve(a, sl, &in, &out, &st);
        for (int i = tid; i < G::REC_WORDS; i += kThreads) rec[i] = 0u;
        // ---- 1. the slab ---------------------------------------------------
        if (ld_ok) {
            if (!wait_phase_cta(ldb, ld_phase)) {
                ld_ok = false;           // the copies stay pending on phase ld_phase
            } else {
                ld_pending = false;
                ld_phase ^= 1u;
            }
        } else {
            __syncthreads();
        }

        // ---- 2. Alg. 1 statistics over the cluster -------------------------
        {
            StatAcc acc;
#pragma unroll 4
            for (int i = 0; i < kSlabPts / 2 / kThreads; i++) {
                const int c = tid + i * kThreads;              // pair of points
                const int row = c / (A1::n / 2), col = 2 * (c % (A1::n / 2));
                const float4 v = *reinterpret_cast<const float4*>(slab + srow(row, col));
                acc.add<true>(v.x, v.y, rec + 4);
                acc.add<true>(v.z, v.w, rec + 4);
            }
            uint32_t am = acc.amax(), nz = acc.nnz, nf = acc.nonfinite;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
                nz += __shfl_xor_sync(0xffffffffu, nz, o);
                nf |= __shfl_xor_sync(0xffffffffu, nf, o);
            }
            if ((tid & 31) == 0) {
                atomicMax(&rec[0], am);
                atomicAdd(&rec[1], nz);
                atomicOr(&rec[2], nf);
            }
        }
        cluster_sync();                          // every CTA's record is complete
        {
            uint32_t* tot = reinterpret_cast<uint32_t*>(stg);   // free until the column phase
            for (int b = tid; b < G::REC_WORDS; b += kThreads) {
                if (b == 3) continue;
                uint32_t v = 0;
#pragma unroll 4
                for (int j = 0; j < G::C; j++) {
                    const uint32_t x = ld_cluster_u32(mapa_shared(rec_u32 + 4u * (uint32_t)b, (uint32_t)j));
                    v = b == 0 ? max(v, x) : (b == 2 ? (v | x) : v + x);
                }
                tot[b] = v;
            }
            __syncthreads();
            if (warp == 0) {
                const int kk = select_k_core(tot[2], tot[0], tot[1],
                                             [tot](int bin) { return tot[4 + bin]; }, a.kp);
                if (tid == 0) {
                    sh_k = kk;
                    if (rank == 0) {
                        st->amax_bits = tot[0];
                        st->nnz = tot[1];
                        st->nonfinite = tot[2];
                        st->k = kk;
                    }
                }
            }
            __syncthreads();
        }
        const int k = sh_k;
        const float pre = exp2i(k);
        const float2 pre2 = make_float2(pre, pre);

        // ---- 3. rows -------------------------------------------------------
#pragma unroll 1
        for (int rt = 0; rt < G::ROW_TILES; rt++) {
            float2* d = slab + rt * A1::T * A1::TS;
            {   // round A: vector (t, j2), elements x[M j1 + j2]
                const int t = tid >> A1::LGM, j2 = tid & (A1::M - 1);
                float2 x[16];
                float D[32];
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = mul2_rn(d[srow(t, A1::M * j + j2)], pre2);
                const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                const float2 sc2 = make_float2(sc, sc);
                const float4* tw = twA1 + j2 * kTwRow;
#pragma unroll
                for (int kk = 0; kk < 16; kk++) d[srow(t, A1::M * kk + j2)] = tw_out(D, kk, tw[kk], sc2);
                __syncthreads();
            }
            {   // round C1: vector (t, k1, j22), elements Y[M k1 + r j21 + j22]
                const int t = tid >> A1::LGM, rem = tid & (A1::M - 1);
                const int k1 = rem >> A1::LGR, j22 = rem & (A1::r - 1);
                float2 x[16];
                float D[32];
                if (A1::r == 1) {
                    const float4* g = reinterpret_cast<const float4*>(d + srow(t, A1::M * k1));
#pragma unroll
                    for (int c = 0; c < 8; c++) {
                        const float4 q = g[c];
                        x[2 * c] = make_float2(q.x, q.y);
                        x[2 * c + 1] = make_float2(q.z, q.w);
                    }
                    const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                    const float2 sc2 = make_float2(sc, sc);
                    // X[k1 + 16 k2], natural order (every input was read before the round's barrier)
#pragma unroll
                    for (int kk = 0; kk < 16; kk++) d[srow(t, k1 + 16 * kk)] = plain_out(D, kk, sc2);
                    __syncthreads();
                } else {
#pragma unroll
                    for (int j = 0; j < 16; j++) x[j] = d[srow(t, A1::M * k1 + 2 * j + j22)];
                    const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                    const float2 sc2 = make_float2(sc, sc);
                    const float4* tw = twC1 + j22 * kTwRow;
#pragma unroll
                    for (int kk = 0; kk < 16; kk++)
                        d[srow(t, A1::M * k1 + 2 * kk + j22)] = tw_out(D, kk, tw[kk], sc2);
                    __syncthreads();
                    // C2: radix 2 over j22, X[k1 + 16 (k21 + 16 k22)]; every
                    // pair is read before any result is written
                    float2 s0[8], s1[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int u = tid + i * kThreads;      // (t, k1, k21), T x 16 x 16
                        const int c1 = u & 15, k21 = (u >> 4) & 15, tt = u >> 8;
                        const float4 pq = *reinterpret_cast<const float4*>(d + srow(tt, A1::M * c1 + 2 * k21));
                        const float2 p = make_float2(pq.x, pq.y), q = make_float2(pq.z, pq.w);
                        s0[i] = add2_rn(p, q);
                        s1[i] = sub2_rn(p, q);
                    }
                    __syncthreads();
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int u = tid + i * kThreads;
                        const int c1 = u & 15, k21 = (u >> 4) & 15, tt = u >> 8;
                        d[srow(tt, c1 + 16 * k21)] = s0[i];
                        d[srow(tt, c1 + 16 * k21 + 256)] = s1[i];
                    }
                    __syncthreads();
                }
            }
        }
        cluster_sync();                          // every slab holds its rows' results

        // ---- 4. columns ----------------------------------------------------
        float post = exp2i(-k);
        if (a.epilogue == EPI_RT_FINAL) post = exp2i(-k - a.lg_total);
        else if (a.epilogue == EPI_RAW) post = 1.0f;
        const float2 post2 = make_float2(post, post);
        const bool next = sl + nclus < a.batch;
#pragma unroll 1
        for (int q = 0; q < G::COL_TILES; q++) {
            const int col0 = G::Cc * (int)rank + A0::T * q;
            {   // gather columns col0 .. col0 + T0 - 1 of every slab (16-byte pieces)
                constexpr int CPR = A0::T / 2;               // pieces per slab row
                float4 v[8];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int g = tid + i * kThreads;
                    const int j = g / (G::R * CPR), rem = g % (G::R * CPR);
                    const int rho = rem / CPR, c2 = rem % CPR;
                    const int src = srow(rho, col0 + 2 * c2);
                    v[i] = ld_cluster_f4(mapa_shared(slab_u32 + 8u * (uint32_t)src, (uint32_t)j));
                }
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int g = tid + i * kThreads;
                    const int j = g / (G::R * CPR), rem = g % (G::R * CPR);
                    const int rho = rem / CPR, c2 = rem % CPR;
                    *reinterpret_cast<float4*>(stg + scol(2 * c2, G::R * j + rho)) = v[i];
                }
            }
            __syncthreads();
            if (q == G::COL_TILES - 1) {
                cluster_sync();                  // every gather from every slab is done
                if (next) {
                    const float2* nin;
                    float2* nout;
                    SliceStats* nst;
                    resolve(a, sl + nclus, &nin, &nout, &nst);
                    if (ld_ok) {
                        load_slab<G>(nin, rank, slab_u32, ldb);
                        ld_pending = true;
                    }
                }
            }
            {   // round A: vector (t, j2), elements x[M j1 + j2] of column t
                const int t = tid & (A0::T - 1), j2 = tid >> A0::LGT;
                float2 x[16];
                float D[32];
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = stg[scol(t, A0::M * j + j2)];
                const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                const float2 sc2 = make_float2(sc, sc);
                const float4* tw = twA0 + j2 * kTwRow;
#pragma unroll
                for (int kk = 0; kk < 16; kk++) stg[scol(t, A0::M * kk + j2)] = tw_out(D, kk, tw[kk], sc2);
                __syncthreads();
            }
            {   // round C1 (and C2 for n0 = 512), results to HBM
                const int t = tid & (A0::T - 1), rem = tid >> A0::LGT;
                const int k1 = rem >> A0::LGR, j22 = rem & (A0::r - 1);
                float2 x[16];
                float D[32];
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = stg[scol(t, A0::M * k1 + A0::r * j + j22)];
                if (A0::r == 1) {
                    const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                    const float2 sc2 = make_float2(sc, sc);
#pragma unroll
                    for (int kk = 0; kk < 16; kk++)
                        out[MX_BND((size_t)(k1 + 16 * kk) * A1::n + col0 + t, slice_pts)] = mul2_rn(plain_out(D, kk, sc2), post2);
                    __syncthreads();
                } else {
                    const float sc = round_mma<FMT>(x, D, mm, a.idesc, emax, issue);
                    const float2 sc2 = make_float2(sc, sc);
                    const float4* tw = twC0 + j22 * kTwRow;
#pragma unroll
                    for (int kk = 0; kk < 16; kk++)
                        stg[scol(t, A0::M * k1 + 2 * kk + j22)] = tw_out(D, kk, tw[kk], sc2);
                    __syncthreads();
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int u = tid + i * kThreads;      // (t, k1, k21), T x 16 x 16
                        const int tt = u & 7, k21 = 8 * ((u >> 3) & 1) + (u >> 8), c1 = (u >> 4) & 15;
                        const int e = A0::M * c1 + 2 * k21;
                        const float2 p = stg[scol(tt, e)], qv = stg[scol(tt, e + 1)];
                        const float2 s0 = mul2_rn(add2_rn(p, qv), post2);
                        const float2 s1 = mul2_rn(sub2_rn(p, qv), post2);
                        const int e0 = c1 + 16 * k21;
                        out[MX_BND((size_t)e0 * A1::n + col0 + tt, slice_pts)] = s0;
                        out[MX_BND((size_t)(e0 + 256) * A1::n + col0 + tt, slice_pts)] = s1;
                    }
                    __syncthreads();
                }
            }
        }
    }

    // ---- teardown: anything of this CTA still in flight is waited for once
    // more, then the tensor memory is returned
    if (ld_pending) wait_phase(ldb, ld_phase);
    if (mm.pending) wait_phase(mm.mbar, mm.phase ^ 1u);
    if ((!mm.ok || !ld_ok) && tid == 0) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(mm.tbase), "r"(kTmemCols));
}

// Clusters of one kernel instance that the device holds at once (0: none;
// the attributes are set on the first call).
template <int FMT, int LOGN0, int LOGN1>
int resident_clusters() {
    using G = Geo<LOGN0, LOGN1>;
    void (*k)(const Tc2dArgs) = tc2d_kernel<FMT, LOGN0, LOGN1>;
    static int max_clusters = -1;
    if (max_clusters >= 0) return max_clusters;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G::C, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e == cudaSuccess && G::C > 8)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // a refusal here only means "not available"
        n = 0;
    }
    max_clusters = n;
    return n;
}

template <int FMT, int LOGN0, int LOGN1>
cudaError_t launch_one(const Tc2dArgs& a, cudaStream_t s) {
    using G = Geo<LOGN0, LOGN1>;
    void (*k)(const Tc2dArgs) = tc2d_kernel<FMT, LOGN0, LOGN1>;
    const int max_clusters = resident_clusters<FMT, LOGN0, LOGN1>();
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters <= 0) return cudaErrorNotSupported;
    const int clusters = a.batch < max_clusters ? a.batch : max_clusters;
    cfg.gridDim = dim3((unsigned)(clusters * G::C), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e == cudaSuccess) note_launch();
    return e;
}

template <int FMT>
int resident_fmt(int n0, int n1) {
    if (n0 == 256 && n1 == 256) return resident_clusters<FMT, 8, 8>();
    if (n0 == 256 && n1 == 512) return resident_clusters<FMT, 8, 9>();
    if (n0 == 512 && n1 == 256) return resident_clusters<FMT, 9, 8>();
    return resident_clusters<FMT, 9, 9>();
}

template <int FMT>
cudaError_t launch_fmt(const Tc2dArgs& a, cudaStream_t s) {
    if (a.n0 == 256 && a.n1 == 256) return launch_one<FMT, 8, 8>(a, s);
    if (a.n0 == 256 && a.n1 == 512) return launch_one<FMT, 8, 9>(a, s);
    if (a.n0 == 512 && a.n1 == 256) return launch_one<FMT, 9, 8>(a, s);
    return launch_one<FMT, 9, 9>(a, s);
}

}  // namespace tc2d

bool tc2d_supported(int n0, int n1, int fmt, int kblk) {
    return (n0 == 256 || n0 == 512) && (n1 == 256 || n1 == 512) && (fmt == 0 || fmt == 1) &&
           kblk == 32;
}

int tc2d_resident_clusters(int n0, int n1, int fmt) {
    if (!tc2d_supported(n0, n1, fmt, 32)) return 0;
    return fmt == 0 ? tc2d::resident_fmt<0>(n0, n1) : tc2d::resident_fmt<1>(n0, n1);
}

cudaError_t launch_tc2d(const Tc2dArgs& a, int fmt, cudaStream_t s) {
    if (a.batch <= 0) return cudaSuccess;
    if (!tc2d_supported(a.n0, a.n1, fmt, 32)) return cudaErrorNotSupported;
    return fmt == 0 ? tc2d::launch_fmt<0>(a, s) : tc2d::launch_fmt<1>(a, s);
}

MX_BOUNDS_COUNTER(tc2d)

}  // namespace mxfft
