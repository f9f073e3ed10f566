// Tensor-core variant of the MX pass: radix-16 sub-DFTs as MXFP8 matrix
// products on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulation
// in tensor memory), for transform lengths n = 256 r, r in {1, 2, 4, 8}.
//
// Decomposition (four-step, rows of a transform viewed as 16 x M, M = 16 r):
//   j = M j1 + j2, k = k1 + 16 k2
//   A : Y[k1][j2] = W_n^(j2 k1) * DFT16_j1(x[M j1 + j2])[k1]
//   C1: for each k1, 16-point DFTs over j21 of Y[k1][r j21 + j22] (j22 < r),
//       times W_M^(j22 k21) when r > 1
//   C2: r-point DFT over j22 in FP32 (r = 2: a sum and a difference; r = 4:
//       radix 4 with W_4 = -+i, exact; r = 8: radix 2 x radix 4, the odd
//       half times W_8^k, whose (1 -+ i) / sqrt(2) factors use sqrt(1/2)
//       rounded to FP32)
//   X[k1 + 16 (k21 + 16 k22)]
// Every 16-point input vector (32 reals) is one MX block for k = 32 (for k =
// 64 / 128 a block is 2 / 4 consecutive vectors of a transform): shared
// power-of-two scale 2^s from its largest component, elements rounded to the
// 8-bit format (cvt.rn.satfinite).  The real 32 x 32 DFT matrix is prequantised with one
// shared scale per output row.  One tcgen05.mma (M = 128 vectors, N = 32, K =
// 32, kind::f8f6f4) multiplies 128 vectors; because K is one block, the two
// power-of-two scales factor out of the dot product and are applied exactly
// to the FP32 result when it is read back (tcgen05.ld).  Twiddles are MX
// element values (one block per 16 twiddles) multiplied in FP32.
//
// Work unit: a tile of 4096 points (T = 4096 / n whole transforms of one
// slice), which is exactly 256 vectors per radix-16 stage, so a CTA of 256
// threads runs each stage as one round of two MMAs (rows 0-127 and 128-255,
// accumulators in tensor-memory columns 0-31 and 32-63); thread i owns
// vector i (the autotuner may pick, for n <= 1024, CTAs of 128 threads on
// tiles of 2048 points, one MMA per round: see Cta).  CTAs are persistent:
// each walks a contiguous range of tiles (mostly of one slice, whose buffers
// and exponent it resolves once; a columns pass with tiles two columns wide
// walks every grid-th tile instead) and
// copies the next tile into its second shared buffer (cp.async, 16 B per
// thread and copy) while it transforms the current one, so that HBM reads
// overlap the MMA rounds.  The shared layouts are padded so that every
// access pattern below is free of bank conflicts (see slot_row / slot_col).
//
// The only spin wait is on the MMA completion mbarrier, bounded to 100 ms by
// the global timer: on time-out the kernel sets the plan's error flag, waits
// once more (bounded) for its own MMA, frees its tensor memory and finishes.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mx_debug.cuh"
#include "mx_device.cuh"
#include "mx_tcgen05.cuh"

namespace mxfft {
namespace tc16 {

using namespace tcg;

// Two CTA shapes, NT threads on tiles of 16 NT points (NT vectors of 16, one
// per thread and round): NT = 256, two MMAs of 128 rows per round with
// accumulators in 64 tensor-memory columns, 2 CTAs per SM; NT = 128 (n <=
// 1024), one MMA per round, 32 columns, and up to 6 CTAs per SM, so that
// more independent tile pipelines share an SM.  Both compute the same bits.
template <int NT>
struct Cta {
    static constexpr int tile = 16 * NT;
    static constexpr uint32_t tmem_cols = NT == 256 ? 64 : 32;
    static constexpr int off_b = NT * 32;       // after the A operand: NT rows x 32 B
    static constexpr int min_blocks = NT == 256 ? 2 : 4;
};
// Twiddle rows of 16 padded to 18 values, so that a quarter-warp's 16-byte
// reads of 8 consecutive rows hit distinct banks.
constexpr int kTwRow = 18;

using Args = Tc16Args;

// Geometry of one transform length n = 2^LOGN.  n = 128 (R8): round A as
// for the other lengths with M = 8, then one round of 8-point DFTs (see the
// kernel), no C2.
template <int LOGN, int NT>
struct Geo {
    static constexpr int n = 1 << LOGN;
    static constexpr bool R8 = n == 128;
    static constexpr int r = n / 256;               // 1, 2, 4, 8 (0 for n = 128)
    static constexpr int LGR = r == 1 ? 0 : (r == 2 ? 1 : (r == 4 ? 2 : 3));
    static constexpr int M = R8 ? 8 : 16 * r;       // n / 16
    static constexpr int LGM = R8 ? 3 : 4 + LGR;
    static constexpr int T = Cta<NT>::tile / n;     // transforms per tile (32 .. 1)
    static constexpr int LGT = T == 32 ? 5 : (T == 16 ? 4 : (T == 8 ? 3 : (T == 4 ? 2 : (T == 2 ? 1 : 0))));
    // rows pass: [t][e], PADR pad slots after every 2^LGP elements (M; 16
    // for n = 128, whose rows also get 8 more slots so that the 4 transforms
    // a warp spans fall on alternate halves of the banks)
    static constexpr int PADR = r == 8 ? 8 : (r == 4 ? 4 : 2);
    static constexpr int LGP = R8 ? 4 : LGM;
    static constexpr int TS = n + PADR * (n >> LGP) + (R8 ? 8 : 0);
    static constexpr int ROW_SLOTS = T * TS;
    // columns pass: [e][t]; with T < 16, T pad slots after every 16 elements
    static constexpr int COL_SLOTS = n * T + (T < 16 ? T * (n / 16) : 0);
    static constexpr int BUF_SLOTS = ROW_SLOTS > COL_SLOTS ? ROW_SLOTS : COL_SLOTS;
    static_assert(T * M == NT, "one vector per thread per stage");
    static_assert(T >= 2, "columns tiles of at least two columns (16-byte copies)");
    // dynamic shared memory: A operand, B operand (32 x 32 B), twiddles of
    // round A (M rows), of C1 (up to 8 rows; for n = 128 the 8-point pair
    // matrix), then the two tile buffers
    static constexpr int OFF_B = Cta<NT>::off_b;
    static constexpr int OFF_TWA = OFF_B + 1024;
    static constexpr int OFF_TWC = OFF_TWA + M * kTwRow * 8;
    static constexpr int OFF_BUF = (OFF_TWC + 8 * kTwRow * 8 + 127) / 128 * 128;
    static constexpr int SMEM = OFF_BUF + 2 * BUF_SLOTS * 8;
    static_assert(OFF_TWC % 16 == 0, "16-byte aligned matrix and twiddle rows");
};

// Slot (8 bytes) of element e of transform t.  Rows pass: round A reads 16
// consecutive elements per half-warp; round C1 reads each thread's own group
// of M elements as 16-byte pairs (r = 1: chunks 9 k1 + c, distinct mod 8 over
// a quarter-warp) or 8-byte elements (r = 2: slots 34 k1 + 2 j + j22; r = 4:
// 68 k1 + 4 j + j22; r = 8: 136 k1 + 8 j + j22; distinct mod 16 over a
// half-warp); n = 128: round A's half-warp spans 8 elements of two
// transforms 152 slots apart, and the 8-point round reads 16 elements per
// thread as 16-byte pairs (chunks 9 p + c, distinct mod 8 over a
// quarter-warp).  Columns pass: a half-warp spans 16 transforms (T = 16, 32)
// or T transforms x 16 / T elements whose pads put them in distinct bank
// groups (T = 8, 4, 2).  Every pattern was checked for bank conflicts by
// enumerating its addresses.
template <int LOGN, int NT>
__device__ __forceinline__ int slot_row(int t, int e) {
    using G = Geo<LOGN, NT>;
    return (int)MX_BND(t * G::TS + e + G::PADR * (e >> G::LGP), G::BUF_SLOTS);
}
template <int LOGN, int NT>
__device__ __forceinline__ int slot_col(int t, int e) {
    using G = Geo<LOGN, NT>;
    return (int)MX_BND(e * G::T + (G::T < 16 ? G::T * (e >> 4) : 0) + t, G::BUF_SLOTS);
}
template <int LOGN, int DIM, int NT>
__device__ __forceinline__ int slot(int t, int e) {
    return DIM == 1 ? slot_row<LOGN, NT>(t, e) : slot_col<LOGN, NT>(t, e);
}

// Shared state of one CTA's MMA rounds.
struct Mma {
    uint8_t* sA;
    uint32_t sa, sb, sb8, mbar, tbase, phase;   // sb8: the 8-point pair matrix (n = 128)
    bool ok;
};

// One MMA round: every thread MX-encodes its 16-element vector into its row
// of the A operand (thread i: operand half i / 128, row i % 128), one thread
// issues both products, all read back their row.  Returns the 16 complex
// DFT outputs (scales applied) in y.  Ends with a CTA barrier, after which the
// A operand, the accumulators and the caller's shared-memory writes made
// before the call may be reused / are visible.
// Vector v of a round belongs to transform t and has index q in the round's
// order (round A: j2; round C1: r k1 + j22): v = t M + q on the rows pass, v =
// q T + t on the columns pass.  With k = 32 g an MX block is g consecutive q of
// one transform; member i of v's block:
template <int DIM>
__device__ __forceinline__ int block_member(int v, int g, int lgt, int i) {
    if (DIM == 1) return (v & ~(g - 1)) + i;
    const int t = v & ((1 << lgt) - 1);
    const int q = (v >> lgt) & ~(g - 1);
    return ((q + i) << lgt) | t;
}

// sb: the B operand (the 16-point DFT matrix, or for n = 128's second round
// two 8-point DFTs on the diagonal, so that the row's two halves transform
// two 8-point vectors).
template <int FMT, int DIM, int NT>
__device__ __forceinline__ void dft16_round(const float2 (&x)[16], float2 (&y)[16], Mma& mm,
                                            uint32_t sb, uint32_t idesc, int emax, bool issue,
                                            int g, int lgt, uint32_t* sAm) {
    const int tid = threadIdx.x, warp = tid >> 5;
    float A = vec_max_abs(x);
    if (g > 1) {
        // one shared scale for the g vectors of the block (members may sit in
        // other warps: exchanged through shared memory; the previous round's
        // reads of sAm finished before its product was issued)
        sAm[tid] = __float_as_uint(A);
        __syncthreads();
        for (int i = 0; i < g; i++) A = fmax_nan(A, __uint_as_float(sAm[block_member<DIM>(tid, g, lgt, i)]));
    }
    const bool bad = !(A <= 3.402823466e38f);
    const int sv = mx_scale_exp(__float_as_uint(A), emax);
    const float inv = exp2i(-sv);
    const float2 inv2 = make_float2(inv, inv);
    uint32_t w32[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float2 a = mul2_rn(x[2 * j], inv2), b = mul2_rn(x[2 * j + 1], inv2);
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
    if (tid == 0 && issue) {
        const uint64_t bd = smem_desc(sb, 128, 256);
        const uint64_t a0 = smem_desc(mm.sa, 128, 256);
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;"
                     " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                     :: "r"(mm.tbase), "l"(a0), "l"(bd), "r"(idesc), "r"(0));
        if (NT == 256) {
            const uint64_t a1 = smem_desc(mm.sa + 4096, 128, 256);
            asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;"
                         " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                         :: "r"(mm.tbase + 32u), "l"(a1), "l"(bd), "r"(idesc), "r"(0));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mm.mbar));
    }
    // warp 0 waits (sleeping between checks), the other warps on the CTA
    // barrier, so that they take no issue slots from the SM's other CTA
    const bool done = wait_phase_cta(mm.mbar, mm.phase);
    mm.phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float d[32];
    if (done) {
        // warp w reads lanes 32 (w % 4) .. of accumulator w / 4
        tmem_ld32(mm.tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * 32), d);
    } else {
#pragma unroll
        for (int c = 0; c < 32; c++) d[c] = 0.f;
        mm.ok = false;
    }
    // D is exact-scaled by the vector's scale and the matrix rows' scale, which
    // is 2^-emax for every row (each row holds an entry of magnitude 1)
    const float sc = bad ? __int_as_float(0x7fffffff) : exp2i(sv - emax);
    const float2 sc2 = make_float2(sc, sc);
#pragma unroll
    for (int k = 0; k < 16; k++) y[k] = mul2_rn(make_float2(d[2 * k], d[2 * k + 1]), sc2);
}

// (w.re y.re - w.im y.im, w.re y.im + w.im y.re), each product rounded (the
// library is built without multiply-add contraction)
__device__ __forceinline__ float2 cmul(float2 w, float2 y) {
    return make_float2(__fsub_rn(__fmul_rn(w.x, y.x), __fmul_rn(w.y, y.y)),
                       __fadd_rn(__fmul_rn(w.x, y.y), __fmul_rn(w.y, y.x)));
}

__device__ __forceinline__ float2 scale2(float2 v, float s) {
    return make_float2(__fmul_rn(v.x, s), __fmul_rn(v.y, s));
}

// Buffers of the slice a CTA works on, resolved once per slice (a CTA walks
// a contiguous range of tiles, so the slice rarely changes between tiles).
struct SliceCache {
    int slice = -1;
    const float2* in;
    float2* out;
    int k;          // prescale exponent (when with_k)
};

__device__ __forceinline__ void resolve(const Args& a, int slice, bool with_k, SliceCache& c) {
    if (c.slice == slice) return;
    c.slice = slice;
    const SliceStats* st;
    if (a.ref) {
        const SliceRef r = a.ref[slice];
        c.in = r.in;
        c.out = r.out;
        st = r.st;
    } else {
        const size_t b = (size_t)slice * a.n0 * a.n1;
        c.in = a.in + b;
        c.out = a.out + b;
        st = a.st + slice;
    }
    c.k = with_k ? st->k : 0;
}

// Issue the cp.async copies of one tile (transforms t0 .. t0 + T - 1 of the
// slice whose input is in) into buffer buf (8 x 16 B per thread).
template <int LOGN, int DIM, int NT>
__device__ __forceinline__ void load_tile(const Args& a, const float2* in, int t0, uint32_t buf) {
    using G = Geo<LOGN, NT>;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int q = threadIdx.x + i * NT;            // 16-byte chunk of the tile
        const float2* src;
        int t, e;
        const size_t slice_pts = (size_t)a.n0 * a.n1;
        (void)slice_pts;
        if (DIM == 1) {
            t = q >> (LOGN - 1);
            e = 2 * (q & ((G::n >> 1) - 1));
            src = in + MX_BND((size_t)(t0 + t) * a.n1 + e, slice_pts - 1);
        } else {
            e = q >> (G::LGT - 1);
            t = 2 * (q & ((G::T >> 1) - 1));
            src = in + MX_BND((size_t)e * a.n1 + t0 + t, slice_pts - 1);
        }
        cp_async16(buf + 8u * (uint32_t)slot<LOGN, DIM, NT>(t, e), src);
    }
}

// FOLD (columns pass, n <= 1024): also accumulate the output's statistics
// (MXFFT_OPT_FOLD_STATS); a separate instance, so that the other passes carry
// none of its code.
template <int FMT, int DIM, int LOGN, bool FOLD, int NT>
__global__ void __launch_bounds__(NT, Cta<NT>::min_blocks)
tc16_pass_kernel(const Args a) {
    using G = Geo<LOGN, NT>;
    constexpr int r = G::r, M = G::M, T = G::T;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t sAm[NT];   // block maxima exchange (k > 32)
    uint8_t* sB = smem + G::OFF_B;
    float2* sTwA = reinterpret_cast<float2*>(smem + G::OFF_TWA);
    float2* sTwC = reinterpret_cast<float2*>(smem + G::OFF_TWC);
    float2* bufs = reinterpret_cast<float2*>(smem + G::OFF_BUF);
    const uint32_t buf_u32 = smem_u32(bufs);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int other = DIM == 1 ? a.n0 : a.n1;
    const int per_slice = other / T;
    const int ntiles = a.batch * per_slice;
    const int emax = FMT == 0 ? 8 : 15;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(Cta<NT>::tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 64) reinterpret_cast<uint4*>(sB)[tid] = __ldg(reinterpret_cast<const uint4*>(a.bmat) + tid);
    // n = 128 has no C2 twiddles: its 8-point pair matrix takes their place
    if (G::R8 && tid < 64)
        reinterpret_cast<uint4*>(sTwC)[tid] = __ldg(reinterpret_cast<const uint4*>(a.bmat2) + tid);
    for (int i = tid; i < M * 16; i += NT) sTwA[(i >> 4) * kTwRow + (i & 15)] = __ldg(a.twA + i);
    if (r > 1 && tid < r * 16) sTwC[(tid >> 4) * kTwRow + (tid & 15)] = __ldg(a.twC + tid);
    // CTA b takes the contiguous tiles [tile_begin, tile_end), shares equal to
    // within one tile.  Exception: a columns pass whose tiles are 2 columns
    // (16 bytes of each row; n = 2048 with 256 threads, n = 1024 with 128):
    // there CTA b takes the tiles b, b +
    // grid, ..., so that the CTAs working at the same time read and write
    // adjacent columns and share every DRAM sector (a contiguous range would
    // leave each sector's other half to the same CTA's next tile, after the
    // sector has left L2).
    constexpr bool kStrided = DIM == 0 && T == 2;   // n = 2048 (NT = 256), n = 1024 (NT = 128)
    const int share = ntiles / (int)gridDim.x, extra = ntiles % (int)gridDim.x;
    const int tile_begin = kStrided ? (int)blockIdx.x
                                    : (int)blockIdx.x * share + min((int)blockIdx.x, extra);
    const int tile_step = kStrided ? (int)gridDim.x : 1;
    const int my_tiles = kStrided
        ? ((int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0)
        : share + ((int)blockIdx.x < extra ? 1 : 0);
    const bool with_k = a.prologue == PRO_PRESCALE || a.epilogue != EPI_RAW;
    const size_t slice_pts = (size_t)a.n0 * a.n1;      // bounds of the debug build
    (void)slice_pts;
    SliceCache ld, cs;   // slices of the tile being loaded and of the current tile
    // Alg. 1 statistics of this pass's output for the next transform's
    // prescale (the round trip's inverse), columns pass only: every stored
    // value goes through the statistics kernel's StatAcc; a run of tiles of
    // one slice is one segment, flushed into the slice's record with its tile
    // count when the slice changes and at the end (the flush that completes
    // the slice's tiles selects k).  Not for the strided n = 2048 columns
    // pass, whose tiles of a slice are spread over all CTAs.
    constexpr bool fold = FOLD && DIM == 0 && !kStrided;
    // 8 histograms by lane (a shared atomic per counted point: lane l adds
    // into copy l % 8, so at most 4 lanes of one atomic meet in a copy, where
    // neighbouring columns, whose values often share a bin, sit in
    // neighbouring lanes), summed into so_hist at each flush
    constexpr int kCopies = fold ? 8 : 1;
    __shared__ uint32_t so_whist[kCopies][fold ? kHistBins : 1];
    __shared__ uint32_t so_hist[fold ? kHistBins : 1];
    __shared__ uint32_t so_misc[4];
    uint32_t* so_wh = so_whist[tid % kCopies];
    StatAcc oacc;
    int seg_slice = -1, seg_tiles = 0;
    SliceStats* seg_st = nullptr;
    if (fold)
        for (int b = tid; b < kCopies * kHistBins; b += NT) (&so_whist[0][0])[b] = 0;
    (void)seg_slice; (void)seg_tiles; (void)so_misc; (void)so_wh;
    auto flush_out = [&]() {
        if (seg_st) {
            __syncthreads();
            for (int b = tid; b < kHistBins; b += NT) {
                uint32_t c = 0;
#pragma unroll
                for (int w = 0; w < kCopies; w++) c += so_whist[w][b];
                so_hist[b] = c;
            }
            __syncthreads();
            stats_flush_and_select_n(oacc, so_hist, so_misc, seg_st, (uint32_t)seg_tiles,
                                     (uint32_t)per_slice, a.kp);
            __syncthreads();
            for (int b = tid; b < kCopies * kHistBins; b += NT) (&so_whist[0][0])[b] = 0;
            oacc = StatAcc();
            __syncthreads();
        }
    };
    if (my_tiles > 0) {
        const int sl = tile_begin / per_slice;
        resolve(a, sl, false, ld);
        load_tile<LOGN, DIM, NT>(a, ld.in, (tile_begin - sl * per_slice) * T, buf_u32);
    }
    cp_async_commit();
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    Mma mm;
    mm.sA = smem;
    mm.sa = smem_u32(smem);
    mm.sb = smem_u32(sB);
    mm.sb8 = smem_u32(sTwC);
    mm.mbar = smem_u32(&mbar);
    mm.tbase = tmem_base;
    mm.phase = 0;
    mm.ok = true;

    int cur = 0;
    for (int it = 0; it < my_tiles; it++, cur ^= 1) {
        const int tile = tile_begin + it * tile_step;
        // prefetch the next tile into the other buffer (free since the last
        // barrier of the previous iteration), then wait for this one
        const int next = tile + tile_step;
        if (it + 1 < my_tiles) {
            const int sl = next / per_slice;
            resolve(a, sl, false, ld);
            load_tile<LOGN, DIM, NT>(a, ld.in, (next - sl * per_slice) * T,
                                 buf_u32 + (uint32_t)((cur ^ 1) * G::BUF_SLOTS * 8));
        }
        cp_async_commit();
        const int slice = tile / per_slice;
        const int t0 = (tile - slice * per_slice) * T;
        if (fold && slice != seg_slice) {
            flush_out();
            seg_slice = slice;
            seg_tiles = 0;
            seg_st = a.ref ? a.ref[slice].st_out : (a.st_out ? a.st_out + slice : nullptr);
        }
        seg_tiles++;
        const bool fold_tile = fold && seg_st != nullptr;   // the same for the whole CTA
        // the slice's exponent is fetched while the tile's copies land
        resolve(a, slice, with_k, cs);
        const int kslice = cs.k;
        cp_async_wait_prev();
        __syncthreads();

        float2* d = bufs + cur * G::BUF_SLOTS;
        float2* __restrict__ out = cs.out;

        // ---- round A: vector (t, j2), elements x[M j1 + j2] ----------------
        {
            const int v = tid;
            int t, j2;
            if (DIM == 1) { t = v >> G::LGM; j2 = v & (M - 1); }
            else { t = v & (T - 1); j2 = v >> G::LGT; }
            float2 x[16], y[16];
            if (a.prologue == PRO_PRESCALE) {
                const float pre = exp2i(kslice);
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = mul2_rn(d[slot<LOGN, DIM, NT>(t, M * j + j2)], make_float2(pre, pre));
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = d[slot<LOGN, DIM, NT>(t, M * j + j2)];
            }
            dft16_round<FMT, DIM, NT>(x, y, mm, mm.sb, a.idesc, emax, !a.stall, a.g, G::LGT, sAm);
            const float4* tw = reinterpret_cast<const float4*>(sTwA + j2 * kTwRow);
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float4 w = tw[k >> 1];
                d[slot<LOGN, DIM, NT>(t, M * k + j2)] = cmul(make_float2(w.x, w.y), y[k]);
                d[slot<LOGN, DIM, NT>(t, M * (k + 1) + j2)] = cmul(make_float2(w.z, w.w), y[k + 1]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }

        float post = 1.0f;
        if (a.epilogue == EPI_UNSCALE) post = exp2i(-kslice);
        else if (a.epilogue == EPI_RT_FINAL) post = exp2i(-kslice - a.lg_total);
        const bool scale_out = a.epilogue != EPI_RAW;

        if (G::R8) {
            // ---- n = 128, round B: 8-point DFTs over j2 of Y[k1][j2] for the
            // pair k1 = 2 p, 2 p + 1 (elements 16 p .. 16 p + 15 of the round-A
            // layout): one MMA row, both vectors one MX block, the B operand
            // two 8-point DFTs on the diagonal; X[k1 + 16 k2] ------------------
            const int v = tid;
            int t, p;
            if (DIM == 1) { t = v >> 3; p = v & 7; }
            else { t = v & (T - 1); p = v >> G::LGT; }
            float2 x[16], y[16];
            if (DIM == 1) {
                const float4* g = reinterpret_cast<const float4*>(d + slot_row<LOGN, NT>(t, 16 * p));
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    const float4 q = g[c];
                    x[2 * c] = make_float2(q.x, q.y);
                    x[2 * c + 1] = make_float2(q.z, q.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = d[slot_col<LOGN, NT>(t, 16 * p + j)];
            }
            dft16_round<FMT, DIM, NT>(x, y, mm, mm.sb8, a.idesc, emax, !a.stall, a.g, G::LGT, sAm);
#pragma unroll
            for (int k2 = 0; k2 < 8; k2++) {
                const float2 v0 = scale_out ? scale2(y[k2], post) : y[k2];        // X[2 p + 16 k2]
                const float2 v1 = scale_out ? scale2(y[8 + k2], post) : y[8 + k2];  // X[2 p + 1 + 16 k2]
                if (fold_tile) {
                    oacc.add_plain(v0.x, v0.y, so_wh);
                    oacc.add_plain(v1.x, v1.y, so_wh);
                }
                const int e = 2 * p + 16 * k2;
                if (DIM == 1) {
                    *reinterpret_cast<float4*>(out + MX_BND((size_t)(t0 + t) * a.n1 + e, slice_pts - 1)) =
                        make_float4(v0.x, v0.y, v1.x, v1.y);
                } else {
                    out[MX_BND((size_t)e * a.n1 + t0 + t, slice_pts)] = v0;
                    out[MX_BND((size_t)(e + 1) * a.n1 + t0 + t, slice_pts)] = v1;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            // the tile is done and its buffer free for the next prefetch
            if (__syncthreads_or(!mm.ok)) break;
            continue;
        }

        // ---- round C1: vector (t, k1, j22), elements Y[M k1 + r j21 + j22] -
        {
            const int v = tid;
            int t, rem;
            if (DIM == 1) { t = v >> G::LGM; rem = v & (M - 1); }
            else { t = v & (T - 1); rem = v >> G::LGT; }
            const int k1 = rem >> G::LGR;
            const int j22 = rem & (r - 1);
            float2 x[16], y[16];
            if (DIM == 1 && r == 1) {
                // own group of 16 consecutive elements, as 16-byte pairs
                const float4* g = reinterpret_cast<const float4*>(d + slot_row<LOGN, NT>(t, M * k1));
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    const float4 q = g[c];
                    x[2 * c] = make_float2(q.x, q.y);
                    x[2 * c + 1] = make_float2(q.z, q.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) x[j] = d[slot<LOGN, DIM, NT>(t, M * k1 + r * j + j22)];
            }
            dft16_round<FMT, DIM, NT>(x, y, mm, mm.sb, a.idesc, emax, !a.stall, a.g, G::LGT, sAm);
            if (r == 1) {
                // X[k1 + 16 k2]
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    const float2 val = scale_out ? scale2(y[k], post) : y[k];
                    if (fold_tile) oacc.add_plain(val.x, val.y, so_wh);
                    const int e = k1 + 16 * k;
                    if (DIM == 1) out[MX_BND((size_t)(t0 + t) * a.n1 + e, slice_pts)] = val;
                    else out[MX_BND((size_t)e * a.n1 + t0 + t, slice_pts)] = val;
                }
            } else {
                const float4* tw = reinterpret_cast<const float4*>(sTwC + j22 * kTwRow);
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const float4 w = tw[k >> 1];
                    d[slot<LOGN, DIM, NT>(t, M * k1 + r * k + j22)] = cmul(make_float2(w.x, w.y), y[k]);
                    d[slot<LOGN, DIM, NT>(t, M * k1 + r * (k + 1) + j22)] = cmul(make_float2(w.z, w.w), y[k + 1]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        // r = 1: the tile is done and its buffer free for the next prefetch;
        // r = 2: C1's results are visible to C2.  A CTA whose wait timed out
        // stops at the end of the tile.
        if (r == 1) {
            if (__syncthreads_or(!mm.ok)) break;
            continue;
        }
        __syncthreads();

        if (r == 4) {
            // ---- C2: radix-4 over j22 (W_4 = -+i exact): X[k1 + 16 (k21 + 16 k22)]
            const float sg = a.inv ? 1.0f : -1.0f;         // W_4 = sg i
#pragma unroll 2
            for (int i = 0; i < 4; i++) {
                const int u = tid + i * NT;       // (t, k1, k21), T x 16 x 16
                int t, k1, k21;
                if (DIM == 1) { k1 = u & 15; k21 = (u >> 4) & 15; t = u >> 8; }
                else if (T == 4) { t = u & 3; k21 = 4 * ((u >> 2) & 3) + (u >> 8); k1 = (u >> 4) & 15; }
                else {   // T = 2 (NT = 128): the half-warp covers k21 bits 0, 2, 3
                    t = u & 1;
                    k21 = (((u >> 1) & 3) << 2) | ((u >> 3) & 1) | (((u >> 8) & 1) << 1);
                    k1 = (u >> 4) & 15;
                }
                const int e = M * k1 + 4 * k21;
                float2 U0, U1, U2, U3;
                if (DIM == 1) {
                    // two 16-byte reads; lanes with k1 bit 2 set read the upper
                    // pair first, so a quarter-warp covers 8 distinct chunks
                    const float4* q = reinterpret_cast<const float4*>(d + slot_row<LOGN, NT>(t, e));
                    const int par = (k1 >> 2) & 1;
                    const float4 f0 = q[par], f1 = q[par ^ 1];
                    const float4 lo = par ? f1 : f0, hi = par ? f0 : f1;
                    U0 = make_float2(lo.x, lo.y);
                    U1 = make_float2(lo.z, lo.w);
                    U2 = make_float2(hi.x, hi.y);
                    U3 = make_float2(hi.z, hi.w);
                } else {
                    U0 = d[slot_col<LOGN, NT>(t, e)];
                    U1 = d[slot_col<LOGN, NT>(t, e + 1)];
                    U2 = d[slot_col<LOGN, NT>(t, e + 2)];
                    U3 = d[slot_col<LOGN, NT>(t, e + 3)];
                }
                const float2 a0 = make_float2(__fadd_rn(U0.x, U2.x), __fadd_rn(U0.y, U2.y));
                const float2 a1 = make_float2(__fsub_rn(U0.x, U2.x), __fsub_rn(U0.y, U2.y));
                const float2 b0 = make_float2(__fadd_rn(U1.x, U3.x), __fadd_rn(U1.y, U3.y));
                const float2 b1 = make_float2(__fsub_rn(U1.x, U3.x), __fsub_rn(U1.y, U3.y));
                const float2 wb = make_float2(-sg * b1.y, sg * b1.x);     // W_4 b1, exact
                float2 X[4];
                X[0] = make_float2(__fadd_rn(a0.x, b0.x), __fadd_rn(a0.y, b0.y));
                X[1] = make_float2(__fadd_rn(a1.x, wb.x), __fadd_rn(a1.y, wb.y));
                X[2] = make_float2(__fsub_rn(a0.x, b0.x), __fsub_rn(a0.y, b0.y));
                X[3] = make_float2(__fsub_rn(a1.x, wb.x), __fsub_rn(a1.y, wb.y));
#pragma unroll
                for (int k22 = 0; k22 < 4; k22++) {
                    const float2 val = scale_out ? scale2(X[k22], post) : X[k22];
                    if (fold_tile) oacc.add_plain(val.x, val.y, so_wh);
                    const int eo = k1 + 16 * k21 + 256 * k22;
                    if (DIM == 1) out[MX_BND((size_t)(t0 + t) * a.n1 + eo, slice_pts)] = val;
                    else out[MX_BND((size_t)eo * a.n1 + t0 + t, slice_pts)] = val;
                }
            }
            // the buffer is refilled by the next iteration's prefetch
            if (__syncthreads_or(!mm.ok)) break;
        }
        if (r == 8) {
            // ---- C2: radix 8 over j22 = radix 4 on the even and the odd
            // inputs, then X[k] = E[k] + W_8^k O[k], X[k + 4] = E[k] - W_8^k O[k]
            const float sg = a.inv ? 1.0f : -1.0f;         // W_8 = (1 + sg i) / sqrt(2)
            const float c8 = 0.70710678118654752f;          // sqrt(1/2), rounded to FP32
#pragma unroll 1
            for (int i = 0; i < 2; i++) {
                const int u = tid + i * NT;       // (t, k1, k21), T x 16 x 16
                int t, k1, k21;
                if (DIM == 1) { k1 = u & 15; k21 = (u >> 4) & 15; t = u >> 8; }
                else { t = u & 1; k21 = 2 * ((u >> 1) & 7) + (u >> 8); k1 = (u >> 4) & 15; }
                const int e = M * k1 + 8 * k21;
                float2 U[8];
                if (DIM == 1) {
                    // four 16-byte reads; a lane reads its chunks in the order
                    // c ^ x, x = (k1 >> 1) & 3, so a quarter-warp covers 8
                    // distinct chunks, then undoes the permutation
                    const float4* q = reinterpret_cast<const float4*>(d + slot_row<LOGN, NT>(t, e));
                    const int x = (k1 >> 1) & 3;
                    float4 f[4];
#pragma unroll
                    for (int c = 0; c < 4; c++) f[c] = q[c ^ x];
                    if (x & 1) {
                        float4 s0 = f[0]; f[0] = f[1]; f[1] = s0;
                        float4 s2 = f[2]; f[2] = f[3]; f[3] = s2;
                    }
                    if (x & 2) {
                        float4 s0 = f[0]; f[0] = f[2]; f[2] = s0;
                        float4 s1 = f[1]; f[1] = f[3]; f[3] = s1;
                    }
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        U[2 * c] = make_float2(f[c].x, f[c].y);
                        U[2 * c + 1] = make_float2(f[c].z, f[c].w);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; j++) U[j] = d[slot_col<LOGN, NT>(t, e + j)];
                }
                float2 E[4], O[4];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const float2 x0 = U[h], x1 = U[h + 2], x2 = U[h + 4], x3 = U[h + 6];
                    const float2 a0 = make_float2(__fadd_rn(x0.x, x2.x), __fadd_rn(x0.y, x2.y));
                    const float2 a1 = make_float2(__fsub_rn(x0.x, x2.x), __fsub_rn(x0.y, x2.y));
                    const float2 b0 = make_float2(__fadd_rn(x1.x, x3.x), __fadd_rn(x1.y, x3.y));
                    const float2 b1 = make_float2(__fsub_rn(x1.x, x3.x), __fsub_rn(x1.y, x3.y));
                    const float2 wb = make_float2(-sg * b1.y, sg * b1.x);     // W_4 b1, exact
                    float2* R = h == 0 ? E : O;
                    R[0] = make_float2(__fadd_rn(a0.x, b0.x), __fadd_rn(a0.y, b0.y));
                    R[1] = make_float2(__fadd_rn(a1.x, wb.x), __fadd_rn(a1.y, wb.y));
                    R[2] = make_float2(__fsub_rn(a0.x, b0.x), __fsub_rn(a0.y, b0.y));
                    R[3] = make_float2(__fsub_rn(a1.x, wb.x), __fsub_rn(a1.y, wb.y));
                }
                // W_8^k O[k]: k = 1 (1 + sg i) / sqrt 2, k = 2 sg i (exact),
                // k = 3 (-1 + sg i) / sqrt 2
                float2 P[4];
                P[0] = O[0];
                P[1] = make_float2(__fmul_rn(__fsub_rn(O[1].x, sg * O[1].y), c8),
                                   __fmul_rn(__fadd_rn(O[1].y, sg * O[1].x), c8));
                P[2] = make_float2(-sg * O[2].y, sg * O[2].x);
                P[3] = make_float2(-__fmul_rn(__fadd_rn(O[3].x, sg * O[3].y), c8),
                                   __fmul_rn(__fsub_rn(sg * O[3].x, O[3].y), c8));
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int k4 = k & 3;
                    float2 X = k < 4 ? make_float2(__fadd_rn(E[k4].x, P[k4].x), __fadd_rn(E[k4].y, P[k4].y))
                                     : make_float2(__fsub_rn(E[k4].x, P[k4].x), __fsub_rn(E[k4].y, P[k4].y));
                    if (scale_out) X = scale2(X, post);
                    if (fold_tile) oacc.add_plain(X.x, X.y, so_wh);
                    const int eo = k1 + 16 * k21 + 256 * k;
                    if (DIM == 1) out[MX_BND((size_t)(t0 + t) * a.n1 + eo, slice_pts)] = X;
                    else out[MX_BND((size_t)eo * a.n1 + t0 + t, slice_pts)] = X;
                }
            }
            // the buffer is refilled by the next iteration's prefetch
            if (__syncthreads_or(!mm.ok)) break;
        }
        if (r == 2) {
            // ---- C2: radix-2 over j22: X[k1 + 16 (k21 + 16 k22)] ----------
#pragma unroll 2
            for (int i = 0; i < 8; i++) {
                const int u = tid + i * NT;       // (t, k1, k21), T x 16 x 16
                int t, k1, k21;
                if (DIM == 1) { k1 = u & 15; k21 = (u >> 4) & 15; t = u >> 8; }
                else if (T == 8) { t = u & 7; k21 = 8 * ((u >> 3) & 1) + (u >> 8); k1 = (u >> 4) & 15; }
                else {   // T = 4 (NT = 128): the half-warp covers k21 bits 0 and 3
                    t = u & 3;
                    k21 = (((u >> 2) & 1) << 3) | ((u >> 3) & 1) | (((u >> 8) & 3) << 1);
                    k1 = (u >> 4) & 15;
                }
                const int e = M * k1 + 2 * k21;
                float2 p, q;
                if (DIM == 1) {
                    const float4 pq = *reinterpret_cast<const float4*>(d + slot_row<LOGN, NT>(t, e));
                    p = make_float2(pq.x, pq.y);
                    q = make_float2(pq.z, pq.w);
                } else {
                    p = d[slot_col<LOGN, NT>(t, e)];
                    q = d[slot_col<LOGN, NT>(t, e + 1)];
                }
                float2 s0 = make_float2(__fadd_rn(p.x, q.x), __fadd_rn(p.y, q.y));
                float2 s1 = make_float2(__fsub_rn(p.x, q.x), __fsub_rn(p.y, q.y));
                if (scale_out) { s0 = scale2(s0, post); s1 = scale2(s1, post); }
                if (fold_tile) {
                    oacc.add_plain(s0.x, s0.y, so_wh);
                    oacc.add_plain(s1.x, s1.y, so_wh);
                }
                const int e0 = k1 + 16 * k21, e1 = e0 + 256;
                if (DIM == 1) {
                    out[MX_BND((size_t)(t0 + t) * a.n1 + e0, slice_pts)] = s0;
                    out[MX_BND((size_t)(t0 + t) * a.n1 + e1, slice_pts)] = s1;
                } else {
                    out[MX_BND((size_t)e0 * a.n1 + t0 + t, slice_pts)] = s0;
                    out[MX_BND((size_t)e1 * a.n1 + t0 + t, slice_pts)] = s1;
                }
            }
            // the buffer is refilled by the next iteration's prefetch
            if (__syncthreads_or(!mm.ok)) break;
        }
    }
    if (fold) flush_out();
    cp_async_wait_all();

    // ---- teardown: an abandoned product is waited for once more, then the
    // tensor memory is returned
    if (!mm.ok) {
        wait_phase(mm.mbar, mm.phase ^ 1u);
        if ((tid & 31) == 0) atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(mm.tbase), "r"(Cta<NT>::tmem_cols));
}

// CTAs of one kernel instance that an SM holds at once: registers (allocated
// per warp in units of 256), shared memory (with the per-CTA reservation),
// tensor-memory columns and threads.
template <int NT>
int fit_per_sm(const void* k, size_t smem) {
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, reserved = 0;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return 1;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 65536 / ((NT / 32) * (warp_regs > 0 ? warp_regs : 256));
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + reserved);
    const int by_tmem = 512 / (int)Cta<NT>::tmem_cols;
    int fit = by_regs < by_smem ? by_regs : by_smem;
    fit = fit < by_tmem ? fit : by_tmem;
    fit = fit < 2048 / NT ? fit : 2048 / NT;
    return fit > 0 ? fit : 1;
}

template <int FMT, int DIM, int LOGN, bool FOLD, int NT>
cudaError_t launch_inst(const Args& a, int cps, cudaStream_t s) {
    using G = Geo<LOGN, NT>;
    const size_t smem = G::SMEM;
    void (*k)(const Args) = tc16_pass_kernel<FMT, DIM, LOGN, FOLD, NT>;
    // per kernel instance: shared-memory opt-in, the SM count and the CTAs
    // an SM holds
    static int sms = 0, fit = 0;
    if (sms == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0, count = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        fit = fit_per_sm<NT>((const void*)k, smem);
        sms = count;
    }
    // the persistent grid: cps CTAs per SM when given (at most what fits),
    // else all that fit (256 threads: 2)
    const int per_sm = cps >= 1 && cps <= fit ? cps : fit;
    const int resident = per_sm * sms;
    const int other = DIM == 1 ? a.n0 : a.n1;
    const int ntiles = a.batch * (other / G::T);
    const int blocks = ntiles < resident ? ntiles : resident;
    k<<<blocks, NT, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

// tile: 2048 for the 128-thread CTAs (n <= 1024), else the 256-thread ones
template <int FMT, int DIM, int LOGN>
cudaError_t launch_one(const Args& a, int cps, int tile, cudaStream_t s) {
    constexpr int L = LOGN <= 10 ? LOGN : 10;     // instances that exist for the fold / 128 threads
    const bool fold = DIM == 0 && LOGN <= 10 && a.stats_out;
    if (LOGN <= 10 && tile == 2048)
        return fold ? launch_inst<FMT, 0, L, true, 128>(a, cps, s) : launch_inst<FMT, DIM, L, false, 128>(a, cps, s);
    return fold ? launch_inst<FMT, 0, L, true, 256>(a, cps, s) : launch_inst<FMT, DIM, LOGN, false, 256>(a, cps, s);
}

template <int FMT>
cudaError_t launch_fmt(const Args& a, int cps, int tile, cudaStream_t s) {
    const bool rows = a.dim == 1;
    if (a.n == 128)
        return rows ? launch_one<FMT, 1, 7>(a, cps, tile, s) : launch_one<FMT, 0, 7>(a, cps, tile, s);
    if (a.n == 256)
        return rows ? launch_one<FMT, 1, 8>(a, cps, tile, s) : launch_one<FMT, 0, 8>(a, cps, tile, s);
    if (a.n == 512)
        return rows ? launch_one<FMT, 1, 9>(a, cps, tile, s) : launch_one<FMT, 0, 9>(a, cps, tile, s);
    if (a.n == 1024)
        return rows ? launch_one<FMT, 1, 10>(a, cps, tile, s) : launch_one<FMT, 0, 10>(a, cps, tile, s);
    return rows ? launch_one<FMT, 1, 11>(a, cps, tile, s) : launch_one<FMT, 0, 11>(a, cps, tile, s);
}

}  // namespace tc16

bool tc16_supported(int n, int other, int fmt) {
    // n = 128 or 256 r (r = 1, 2, 4, 8), 8-bit element formats, whole tiles of
    // 4096 / n transforms
    if (n != 128 && n != 256 && n != 512 && n != 1024 && n != 2048) return false;
    const int T = 4096 / n;
    return other >= T && other % T == 0 && (fmt == 0 || fmt == 1);
}

cudaError_t launch_tc16_pass_geo(const Tc16Args& a, int fmt, int batch, int tile, int ctas_per_sm,
                                 cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    Tc16Args b = a;
    b.batch = batch;
    if (fmt == 0) return tc16::launch_fmt<0>(b, ctas_per_sm, tile, s);
    if (fmt == 1) return tc16::launch_fmt<1>(b, ctas_per_sm, tile, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_tc16_pass(const Tc16Args& a, int fmt, int batch, cudaStream_t s) {
    const int other = a.dim == 1 ? a.n0 : a.n1;
    int tile = 0, cps = 0;
    tc16_geo_tuned(a.n, other, a.dim, fmt, a.g, batch, &tile, &cps);
    return launch_tc16_pass_geo(a, fmt, batch, tile, cps, s);
}

MX_BOUNDS_COUNTER(tc16)

}  // namespace mxfft
