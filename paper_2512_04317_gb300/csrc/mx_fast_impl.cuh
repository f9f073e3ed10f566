// Register-resident MX radix-2 pass for transform lengths n = 64..2048 and
// MX blocks of m <= 16 butterflies (k <= 32 real elements), m = 32 (k = 64)
// for n >= 128 with groups of 8 transforms and m = 64 (k = 128) for n >= 128
// with groups of 4.
//
// Data layout and work split:
//   * A CTA owns NG groups of TG transforms (rows or columns) of one slice.
//     A group's data live in shared memory as [element e][transform tau]
//     (row stride S complex), so the TG lanes that share an element index
//     touch consecutive 8-byte words and 64-bit accesses are conflict-free.
//   * Lanes of a warp are transforms (lane % TG) and the rest of the thread
//     index is a "slot" sigma in [0, n/32): every thread holds 32 elements of
//     one transform in registers.
//   * Phase A (stages h = 1..16, all inside a 32-element chunk of the
//     bit-reversed order): slot sigma holds chunk sigma, i.e. the inputs
//     x[rev(sigma) + j n/32], j = 0..31.  Every MX block of these stages lies
//     inside one chunk for m <= 16, so the block maxima are register-local.
//   * Phase B (stages h >= 32): stage pairs (h, 2h); slot sigma = G*(h/8) + r
//     holds the 8-element runs P + 8r + q h, q = 0..3, P = 4hG, which carry
//     whole butterfly groups of both stages.  An MX block of m = 16 spans the
//     runs r and r^1, held by the lanes sigma and sigma^1 (lane ^ TG): one
//     xor shuffle (m = 32: runs r .. r^3, two shuffles, TG = 8 so that the
//     four slots share a warp; in phase A its two chunks, one shuffle; m = 64:
//     8 runs and three shuffles, TG = 4, in phase A four chunks, and at the
//     first stage pair (h = 32, 64), where a block spans both run pairs of a
//     slot, 16 butterflies per lane over 4 lanes).  An odd last stage h = n/2
//     pairs runs sigma and sigma+n/32.
//   * Element quantisation uses the sm_100-family conversions
//     cvt.rn.satfinite.<fmt>x2.f32 and cvt.rn.f16x2.<fmt>x2 (round to nearest
//     even, saturating, signed zeros and subnormals kept), the element-space
//     product uses fma.rn.f32.f16 on the exact f16 element values (a product
//     of two element values is exact, so the only rounding is the add, as in
//     Alg. 2), and u +- c 2^s^ is one FMA per component because c 2^s^ is
//     always an exact FP32 value (s^ >= -127 and the element grid step is >=
//     2^-16).  The scalings and these FMAs run as packed FP32 pairs
//     (__fmul2_rn / __ffma2_rn: each component rounded as its scalar form).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "mx_device.cuh"

namespace mxfft {
namespace fast {

// ---- element conversions: f16x2 bits {lo: Q(a), hi: Q(b)} -----------------
template <int FMT> struct Cvt;
template <> struct Cvt<0> {  // E4M3
    static __device__ __forceinline__ uint32_t q2(float a, float b) {
        unsigned short p; uint32_t h;
        asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(p) : "f"(b), "f"(a));
        asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h) : "h"(p));
        return h;
    }
};
template <> struct Cvt<1> {  // E5M2
    static __device__ __forceinline__ uint32_t q2(float a, float b) {
        unsigned short p; uint32_t h;
        asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(p) : "f"(b), "f"(a));
        asm("cvt.rn.f16x2.e5m2x2 %0, %1;" : "=r"(h) : "h"(p));
        return h;
    }
};
template <> struct Cvt<2> {  // E2M3
    static __device__ __forceinline__ uint32_t q2(float a, float b) {
        unsigned short p; uint32_t h;
        asm("cvt.rn.satfinite.e2m3x2.f32 %0, %1, %2;" : "=h"(p) : "f"(b), "f"(a));
        asm("cvt.rn.f16x2.e2m3x2 %0, %1;" : "=r"(h) : "h"(p));
        return h;
    }
};
template <> struct Cvt<3> {  // E3M2
    static __device__ __forceinline__ uint32_t q2(float a, float b) {
        unsigned short p; uint32_t h;
        asm("cvt.rn.satfinite.e3m2x2.f32 %0, %1, %2;" : "=h"(p) : "f"(b), "f"(a));
        asm("cvt.rn.f16x2.e3m2x2 %0, %1;" : "=r"(h) : "h"(p));
        return h;
    }
};
template <> struct Cvt<4> {  // E2M1
    static __device__ __forceinline__ uint32_t q2(float a, float b) {
        unsigned short p; uint32_t h;
        asm("{.reg .b8 t; cvt.rn.satfinite.e2m1x2.f32 t, %1, %2; cvt.u16.u8 %0, t;}"
            : "=h"(p) : "f"(b), "f"(a));
        asm("{.reg .b8 t; cvt.u8.u16 t, %1; cvt.rn.f16x2.e2m1x2 %0, t;}" : "=r"(h) : "h"(p));
        return h;
    }
};

// a.x * b.y + c with f16 halves (x, y in {lo, hi}) and FP32 c, d
#define MX_FMA_H(NAME, AH, BH)                                                              \
    __device__ __forceinline__ float NAME(uint32_t a, uint32_t b, float c) {                \
        float d;                                                                            \
        asm("{.reg .b16 a0, a1, b0, b1; mov.b32 {a0, a1}, %1; mov.b32 {b0, b1}, %2;"      \
            " fma.rn.f32.f16 %0, " AH ", " BH ", %3;}"                                      \
            : "=f"(d) : "r"(a), "r"(b), "f"(c));                                            \
        return d;                                                                           \
    }
MX_FMA_H(fma_ll, "a0", "b0")
MX_FMA_H(fma_lh, "a0", "b1")
MX_FMA_H(fma_hl, "a1", "b0")
MX_FMA_H(fma_hh, "a1", "b1")
#undef MX_FMA_H

__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}


// Shared exponent from a nonnegative block maximum (NaN/Inf handled by caller).
__device__ __forceinline__ int scale_of(float amax, int emax) {
    return mx_scale_exp(__float_as_uint(amax), emax);
}


// max(|a|, |b|, |c|), NaN if any input is NaN (three-input max of sm_100+).
__device__ __forceinline__ float max3_abs_nan(float a, float b, float c) {
    float d;
    asm("max.NaN.abs.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Largest magnitude of the 2 NB components of the pairs *X[t] (NaN if any is
// NaN), as a tree of three-input maxima: 17 instructions for 32 values.
template <int NB>
__device__ __forceinline__ float block_max_abs(float2* const (&X)[NB]) {
    constexpr int N = 2 * NB;
    float a[N];
#pragma unroll
    for (int t = 0; t < NB; t++) {
        a[2 * t] = X[t]->x;
        a[2 * t + 1] = X[t]->y;
    }
#pragma unroll
    for (int w = 1; w < N; w *= 3)
#pragma unroll
        for (int t = 0; t < N; t += 3 * w) {
            if (t + 2 * w < N) a[t] = max3_abs_nan(a[t], a[t + w], a[t + 2 * w]);
            else if (t + w < N) a[t] = max3_abs_nan(a[t], a[t + w], a[t + w]);
        }
    return a[0];
}

// Alg. 2 on one MX block of NB butterflies whose u/v live in registers.
// Steps: block max of v -> s_v; y = Q(v 2^-s_v); p = x y (exact products, one
// rounding each), written over v, which is dead by then; block max of p -> s^;
// c = Q(p 2^(s_w + s_v - s^)); u +- c 2^s^.  A block holding Inf/NaN decodes
// to NaN (OCP MX NaN scale).  A block of NB butterflies per lane spread over
// 2^NRED lanes (lane ^ red << i, i < NRED) also reduces the two block maxima
// over those lanes.
template <int FMT, int NB, int NRED>
__device__ __forceinline__ void mx_block(float2* const (&U)[NB], float2* const (&V)[NB],
                                         const uint32_t (&W)[NB], int sw, unsigned red,
                                         const FmtParams& fp) {
    float A = block_max_abs<NB>(V);
#pragma unroll
    for (int i = 0; i < NRED; i++) A = fmax_nan(A, __shfl_xor_sync(0xffffffffu, A, red << i));
    const bool bad = !(A <= 3.402823466e38f);
    const int sv = scale_of(A, fp.emax);
    const float inv = exp2i(-sv);
    const float2 inv2 = make_float2(inv, inv);
#pragma unroll
    for (int t = 0; t < NB; t++) {
        // packed FP32 pairs (each component rounded as its scalar operation)
        const float2 vs = __fmul2_rn(*V[t], inv2);
        const uint32_t y = Cvt<FMT>::q2(vs.x, vs.y);
        const uint32_t w = W[t];
        const float pr = fma_ll(w, y, -fma_hh(w, y, -0.0f));
        const float pi = fma_hl(w, y, fma_lh(w, y, -0.0f));
        *V[t] = make_float2(pr, pi);
    }
    float P = block_max_abs<NB>(V);
#pragma unroll
    for (int i = 0; i < NRED; i++) P = fmaxf(P, __shfl_xor_sync(0xffffffffu, P, red << i));
    const int so = sw + sv;
    const uint32_t Pb = __float_as_uint(P);
    const int sh = Pb ? min(max(so + ilogb_bits(Pb) - fp.emax, -127), 127) : so;
    const float f = exp2i(so - sh);
    const float d = bad ? __int_as_float(0x7fffffff) : exp2i(sh);
    const float2 f2 = make_float2(f, f), d2 = make_float2(d, d), nd2 = make_float2(-d, -d);
#pragma unroll
    for (int t = 0; t < NB; t++) {
        const float2 ps = __fmul2_rn(*V[t], f2);
        const uint32_t c = Cvt<FMT>::q2(ps.x, ps.y);
        const __half2 ch = *reinterpret_cast<const __half2*>(&c);
        const float cr = __low2float(ch), ci = __high2float(ch);
        const float2 u = *U[t];
        // u +- c 2^s^ as packed FP32 pairs (each component rounded as __fmaf_rn)
        *U[t] = __ffma2_rn(make_float2(cr, ci), d2, u);
        *V[t] = __ffma2_rn(make_float2(cr, ci), nd2, u);
    }
}

// Phase A stage H on a 32-element chunk r[] (chunk-local butterfly t = 0..15:
// group t / H, index j = t % H).  Chunk sigma holds the stage's butterflies
// 16 sigma .. 16 sigma + 15, so a block of m = 32 is the chunks sigma and
// sigma ^ 1, held by the lanes tg apart.
template <int FMT, int LOGM, int H>
__device__ __forceinline__ void stage_a(float2 (&r)[32], const TwA& tw, const FmtParams& fp,
                                        unsigned tg) {
    constexpr int M = 1 << LOGM;
    constexpr int MB = M < 16 ? M : 16;        // butterflies of a block held by this thread
    constexpr int NRED = M > 16 ? LOGM - 4 : 0;
#pragma unroll
    for (int b0 = 0; b0 < 16; b0 += MB) {
        float2* U[MB];
        float2* V[MB];
        uint32_t W[MB];
#pragma unroll
        for (int q = 0; q < MB; q++) {
            const int t = b0 + q;
            const int iu = 2 * H * (t / H) + (t % H);
            U[q] = &r[iu];
            V[q] = &r[iu + H];
            W[q] = tw.h2[H - 1 + (t % H)];
        }
        mx_block<FMT, MB, NRED>(U, V, W, tw.sw[H - 1 + (b0 % H)], tg, fp);
    }
}

// Phase B: one stage on 8 butterflies u = Ru[i], v = Rv[i], j = jb + i, with
// twiddles at twh[j] / tws[j] (already offset to stage h: the f16x2 table at
// index h + j, 32-byte aligned runs of 8 since jb is a multiple of 8; the
// exponents at h - 1 + j).
template <int FMT, int LOGM>
__device__ __forceinline__ void stage_b8(float2 (&Ru)[8], float2 (&Rv)[8],
                                         const uint32_t* __restrict__ twh,
                                         const int8_t* __restrict__ tws, int jb, unsigned red,
                                         const FmtParams& fp) {
    constexpr int M = 1 << LOGM;
    constexpr int ML = M < 8 ? M : 8;  // butterflies of a block held by this thread
    const uint4* t4 = reinterpret_cast<const uint4*>(twh + jb);
    const uint4 wa = __ldg(t4), wb = __ldg(t4 + 1);
    const uint32_t w8[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int b0 = 0; b0 < 8; b0 += ML) {
        float2* U[ML];
        float2* V[ML];
        uint32_t W[ML];
#pragma unroll
        for (int q = 0; q < ML; q++) {
            U[q] = &Ru[b0 + q];
            V[q] = &Rv[b0 + q];
            W[q] = w8[b0 + q];
        }
        mx_block<FMT, ML, (M > 8 ? LOGM - 3 : 0)>(U, V, W, __ldg(tws + jb + b0), red, fp);
    }
}

// Phase B with m = 64 at the first stage pair (stage 32, and its second stage
// 64): one MX block covers 8 butterflies of each of two run pairs per lane (u =
// RuA[i], v = RvA[i], j = jbA + i, and u = RuB[i], v = RvB[i], j = jbB + i),
// over 4 lanes.
template <int FMT>
__device__ __forceinline__ void stage_b_dual(float2 (&RuA)[8], float2 (&RvA)[8],
                                             float2 (&RuB)[8], float2 (&RvB)[8],
                                             const uint32_t* __restrict__ twh,
                                             const int8_t* __restrict__ tws, int jbA, int jbB,
                                             unsigned red, const FmtParams& fp) {
    const uint4* ta = reinterpret_cast<const uint4*>(twh + jbA);
    const uint4* tb = reinterpret_cast<const uint4*>(twh + jbB);
    const uint4 a0 = __ldg(ta), a1 = __ldg(ta + 1), b0 = __ldg(tb), b1 = __ldg(tb + 1);
    const uint32_t W[16] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                            b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    float2* U[16];
    float2* V[16];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        U[i] = &RuA[i];
        V[i] = &RvA[i];
        U[8 + i] = &RuB[i];
        V[8 + i] = &RvB[i];
    }
    mx_block<FMT, 16, 2>(U, V, W, __ldg(tws + jbA), red, fp);
}

// Compile-time 5-bit reversal of the chunk position.
__host__ __device__ constexpr int rev5(int t) {
    return ((t & 1) << 4) | ((t & 2) << 2) | (t & 4) | ((t & 8) >> 2) | ((t & 16) >> 4);
}

struct FastArgs {
    PassArgs a;
    TwA twa;
    const uint32_t* twh;   // f16x2 twiddle element values, index h + j (entry 0 unused)
    int TG;                // transforms per group (16, or 8 for n = 2048)
    int lgTG;              // log2(TG)
    int S;                 // shared row stride (complex) of a group: TG or TG + 1
    int NG;                // groups per CTA
    int fused;             // 1: columns forward then inverse (fused round trip)
    TwA twa2;              // inverse twiddles of the fused launch (as twa / twh)
    const uint32_t* twh2;
};

// Arguments of the groups of one ragged launch (mx_fast_ragged.cu), passed as
// one kernel parameter (at most 32 KB of parameters).
constexpr int kMaxRaggedGroups = 48;
struct RaggedGroups {
    int n;
    FastArgs g[kMaxRaggedGroups];
};
static_assert(sizeof(RaggedGroups) <= 32000, "ragged groups fit the kernel parameter space");

}  // namespace fast
}  // namespace mxfft
