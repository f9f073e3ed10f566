// Device-side building blocks of the MX-FFT: exact power-of-two scaling,
// exponent extraction, the element quantiser, |x| and the exponent selection
// of Alg. 1.  Every FP32 operation is an explicit round-to-nearest intrinsic
// and the library is compiled with -fmad=false -ftz=false -prec-sqrt=true, so
// results are bit-reproducible.
#pragma once

#include <stdint.h>
#include "mx_internal.h"

namespace mxfft {

// 2^e as a float for e in [-149, 127] (subnormal below -126).
__device__ __forceinline__ float exp2i(int e) {
    return e >= -126 ? __uint_as_float((uint32_t)(e + 127) << 23)
                     : __uint_as_float(1u << (e + 149));
}

// floor(log2 x) for the bits of a positive finite float (normal or subnormal).
__device__ __forceinline__ int ilogb_bits(uint32_t b) {
    uint32_t ex = b >> 23;
    return ex ? (int)ex - 127 : (31 - __clz((int)b)) - 149;
}

// MX shared exponent of a block whose largest |component| has bits amax_bits:
// floor(log2 amax) - emax, within the E8M0 range; 0 for an all-zero block
// (OCP MX v1.0; EncodeBlockMX of Alg. 2).
__device__ __forceinline__ int mx_scale_exp(uint32_t amax_bits, int emax) {
    if (amax_bits == 0) return 0;
    int s = ilogb_bits(amax_bits) - emax;
    return min(max(s, -127), 127);
}

// Round x (already divided by the block scale) to the element grid: nearest,
// ties to even, saturating at maxnorm, sign of zero kept.
// The grid spacing at |x| is q = 2^(max(E, emin) - mbits), E = floor(log2|x|).
// Adding c = 1.5 * 2^23 * q puts |x| + c in the binade [2^23 q, 2^24 q) whose
// ulp is q, so the FP32 adder performs exactly the round-half-even to a
// multiple of q; subtracting c is exact.  c's bits are built from |x|'s
// exponent field, floored at emin.  Clamping before rounding equals rounding
// then saturating because maxnorm lies on the grid.
__device__ __forceinline__ float q_elem(float x, const FmtParams& f) {
    float a = fminf(fabsf(x), f.maxnorm);
    uint32_t eb = __float_as_uint(a) & 0x7F800000u;
    uint32_t cb = max(eb, f.qmin_bits) + f.qadd_bits;
    float c = __uint_as_float(cb);
    float r = __fsub_rn(__fadd_rn(a, c), c);
    return __uint_as_float(__float_as_uint(r) | (__float_as_uint(x) & 0x80000000u));
}

// |x| of a finite complex value: both components scaled by 2^-e with e the
// larger frexp exponent of the nonzero components, FP32 sum of squares,
// correctly rounded sqrt, scaled back by 2^e.  Every power-of-two scaling is
// one correctly rounded multiply (split in two exact steps where 2^e would
// leave the float range).
__device__ __forceinline__ float mag_c3(float re, float im) {
    uint32_t br = __float_as_uint(re) & 0x7fffffffu;
    uint32_t bi = __float_as_uint(im) & 0x7fffffffu;
    if ((br | bi) == 0) return 0.0f;
    int er = br ? ilogb_bits(br) + 1 : -100000;
    int ei = bi ? ilogb_bits(bi) + 1 : -100000;
    int e = max(er, ei);              // frexp exponent, in [-148, 128]
    float a, b;
    if (-e <= 127) {
        float s = exp2i(-e);
        a = __fmul_rn(re, s);
        b = __fmul_rn(im, s);
    } else {                          // e <= -128: scale up in two exact steps
        float s1 = exp2i(64), s2 = exp2i(-e - 64);
        a = __fmul_rn(__fmul_rn(re, s1), s2);
        b = __fmul_rn(__fmul_rn(im, s1), s2);
    }
    float s = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
    float r = __fsqrt_rn(s);
    if (e <= 127) return __fmul_rn(r, exp2i(e));
    return __fmul_rn(__fmul_rn(r, exp2i(64)), exp2i(e - 64));
}

__device__ __forceinline__ bool is_finite_bits(uint32_t b) {
    return (b & 0x7f800000u) != 0x7f800000u;
}

// The same |x| for finite inputs, with a short path: when each component is
// zero or has magnitude in [2^-62, 2^62], the unscaled sqrt(re^2 + im^2)
// performs the scaled computation of mag_c3 times exact powers of two (every
// intermediate stays normal, or the smaller square is below half an ulp of the
// larger in both forms), so the rounded results are identical.
__device__ __forceinline__ float mag_c3_fast(float re, float im) {
    const uint32_t br = __float_as_uint(re) & 0x7fffffffu;
    const uint32_t bi = __float_as_uint(im) & 0x7fffffffu;
    const uint32_t lo = (uint32_t)(127 - 62) << 23, hi = (uint32_t)(127 + 63) << 23;
    const bool okr = br == 0 || (br >= lo && br < hi);
    const bool oki = bi == 0 || (bi >= lo && bi < hi);
    if (okr && oki) return __fsqrt_rn(__fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im)));
    return mag_c3(re, im);
}

// Alg. 1 exponent selection from a slice's statistics, exact integer form.
//   k1 = round(log2(2^t / max(a_max, 1e-30))) = t - (e_a + [M_a^2 >= 2^47])
//        (a_max = M_a 2^(e_a - 23), 24-bit significand; ties cannot occur);
//        a_max < 1e-30 gives round(log2 1e-30) = -100.
//   k2 = ceil(log2(2^e_tau / max(p_tau, 1e-30))) = e_tau - max(floor(log2 p_tau), -100)
//        (floor(log2 1e-30) = -100), and floor(log2 p_tau) is the histogram bin
//        holding rank r = floor(fl32(tau * fl32(n_nz - 1))) of the sorted nonzeros.
// Called by one full warp with the slice's totals (hist_at(bin) returns the
// count of a bin); returns k in every lane.
template <class HistAt>
__device__ __forceinline__ int select_k_core(uint32_t nonfinite, uint32_t ab, uint32_t nnz,
                                             HistAt hist_at, const KParams& kp) {
    const int lane = threadIdx.x & 31;
    if (nonfinite || ab == 0 || nnz == 0) return 0;
    float rf = __fmul_rn(kp.tau, (float)(int)(nnz - 1));
    int r = (int)floorf(rf);
    r = min(max(r, 0), (int)nnz - 1);
    // each lane owns 9 consecutive bins (32 * 9 = 288 >= 277)
    int base = lane * 9;
    uint32_t c[9];
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int bin = base + i;
        c[i] = bin < kHistBins ? hist_at(bin) : 0u;
        tot += c[i];
    }
    uint32_t incl = tot;   // inclusive warp scan of the lane totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t excl = incl - tot;
    int bin_found = 0x7fffffff;
    if (excl <= (uint32_t)r && (uint32_t)r < incl) {
        uint32_t cum = excl;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            cum += c[i];
            if (cum > (uint32_t)r && bin_found == 0x7fffffff) bin_found = base + i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bin_found = min(bin_found, __shfl_xor_sync(0xffffffffu, bin_found, o));
    int ep = bin_found - 149;                         // floor(log2 p_tau)
    // round(log2 max(a_max, 1e-30))
    int ra;
    const uint32_t eps_bits = 0x0DA24260u;            // 1e-30f, the float just above 1e-30
    if (ab < eps_bits) {
        ra = -100;
    } else {
        int e = ilogb_bits(ab);
        uint32_t M = (ab >> 23) ? ((ab & 0x7fffffu) | 0x800000u) : (ab << (__clz((int)ab) - 8));
        ra = e + (((uint64_t)M * (uint64_t)M) >= (1ull << 47) ? 1 : 0);
    }
    int k1 = kp.t_exp - ra;
    int k2 = kp.taumin_exp - max(ep, -100);
    int k = max(k1, k2);
    return min(max(k, kp.kmin), kp.kmax);
}

// The selection from a slice's record in global memory (after the atomics of
// every CTA of the slice).  Called by one full warp; returns k in every lane.
__device__ __forceinline__ int select_k_warp(const SliceStats* st, const KParams& kp) {
    return select_k_core(__ldcg(&st->nonfinite), __ldcg(&st->amax_bits), __ldcg(&st->nnz),
                         [st](int bin) { return __ldcg(&st->hist[bin]); }, kp);
}

// Accumulates one value's contribution to Alg. 1's statistics in per-thread
// registers and the CTA's shared histogram.  When the whole warp executes the
// call, lanes that hit the same bin are merged first (__match_any_sync), so a
// bin shared by many lanes costs one shared atomic instead of one per lane.
// add<true> is for call sites that every lane of the warp reaches (a loop with
// a warp-uniform trip count); add<false> checks the active mask first.
struct StatAcc {
    uint32_t amax_bits = 0;   // max |x| (mag_c3) over points outside the fast range
    uint32_t smax_bits = 0;   // max re^2 + im^2 over points inside it
    uint32_t nnz = 0;
    uint32_t nonfinite = 0;
    // Fast range: each component zero or of magnitude in [2^-62, 2^63).  There
    // |x| = fl(sqrt(s)), s = fl(fl(re^2) + fl(im^2)), exactly as mag_c3
    // computes it (see mag_c3_fast), and s is zero or normal.  The square root
    // is correctly rounded, and for the largest float below 2^(2j), 2^(2j) (1 -
    // 2^-24), it rounds to a value below 2^j; so fl(sqrt(s)) is in [2^j,
    // 2^(j+1)) exactly when s is in [2^(2j), 2^(2j+2)).  Hence the bin
    // floor(log2 |x|) is floor(floor(log2 s) / 2), and max |x| = fl(sqrt(max s))
    // because the rounded square root is monotone: no square root per point.
    template <bool kConverged = false>
    __device__ __forceinline__ void add(float re, float im, uint32_t* sh_hist) {
        const uint32_t br = __float_as_uint(re) & 0x7fffffffu;
        const uint32_t bi = __float_as_uint(im) & 0x7fffffffu;
        const uint32_t lo = (uint32_t)(127 - 62) << 23, hi = (uint32_t)(127 + 63) << 23;
        int bin = -1;
        // (b - 1 wraps zero to the top, so "b == 0 or b >= lo" is one compare)
        if (min(br - 1u, bi - 1u) >= lo - 1u && max(br, bi) < hi) {
            const uint32_t sb = __float_as_uint(__fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im)));
            if (sb) {
                smax_bits = max(smax_bits, sb);
                nnz++;
                bin = (((int)(sb >> 23) - 127) >> 1) + 149;
            }
        } else if (max(br, bi) >= 0x7f800000u) {
            nonfinite = 1;
        } else {
            const uint32_t mb = __float_as_uint(mag_c3(re, im));
            if (!is_finite_bits(mb)) {
                nonfinite = 1;
            } else if (mb != 0) {
                amax_bits = max(amax_bits, mb);
                nnz++;
                bin = ilogb_bits(mb) + 149;
            }
        }
        if (kConverged || __activemask() == 0xffffffffu) {
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            // the lowest lane of its group adds the group's count
            const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
            if (bin >= 0 && (same & below) == 0u)
                atomicAdd(&sh_hist[bin], (uint32_t)__popc(same));
        } else if (bin >= 0) {
            atomicAdd(&sh_hist[bin], 1u);
        }
    }
    // The same accumulation with one shared atomic per counted point (no
    // match), into a histogram that only this warp updates.
    __device__ __forceinline__ void add_plain(float re, float im, uint32_t* wh) {
        const uint32_t br = __float_as_uint(re) & 0x7fffffffu;
        const uint32_t bi = __float_as_uint(im) & 0x7fffffffu;
        const uint32_t lo = (uint32_t)(127 - 62) << 23, hi = (uint32_t)(127 + 63) << 23;
        int bin = -1;
        if (min(br - 1u, bi - 1u) >= lo - 1u && max(br, bi) < hi) {
            const uint32_t sb = __float_as_uint(__fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im)));
            if (sb) {
                smax_bits = max(smax_bits, sb);
                nnz++;
                bin = (((int)(sb >> 23) - 127) >> 1) + 149;
            }
        } else if (max(br, bi) >= 0x7f800000u) {
            nonfinite = 1;
        } else {
            const uint32_t mb = __float_as_uint(mag_c3(re, im));
            if (!is_finite_bits(mb)) {
                nonfinite = 1;
            } else if (mb != 0) {
                amax_bits = max(amax_bits, mb);
                nnz++;
                bin = ilogb_bits(mb) + 149;
            }
        }
        if (bin >= 0) atomicAdd(&wh[bin], 1u);
    }
    // bits of max |x| over everything added
    __device__ __forceinline__ uint32_t amax() const {
        return max(amax_bits, __float_as_uint(__fsqrt_rn(__uint_as_float(smax_bits))));
    }
};

// CTA-wide flush of StatAcc into a slice's global statistics, then the last
// CTA of the slice selects k.  Every thread of the CTA must call it; sh_hist
// must have been zeroed and the CTA synchronised after the adds.  sh_misc
// needs 4 words of shared memory.
__device__ __forceinline__ void stats_flush_and_select_n(StatAcc acc, uint32_t* sh_hist,
                                                         uint32_t* sh_misc, SliceStats* st,
                                                         uint32_t contrib, uint32_t total,
                                                         const KParams& kp);

__device__ __forceinline__ void stats_flush_and_select(StatAcc acc, uint32_t* sh_hist,
                                                       uint32_t* sh_misc, SliceStats* st,
                                                       uint32_t ctas_per_slice,
                                                       const KParams& kp) {
    stats_flush_and_select_n(acc, sh_hist, sh_misc, st, 1u, ctas_per_slice, kp);
}

// The same flush for a CTA that covered `contrib` of the slice's `total`
// units (tiles of a persistent pass): the flush that completes the slice
// selects k.
__device__ __forceinline__ void stats_flush_and_select_n(StatAcc acc, uint32_t* sh_hist,
                                                         uint32_t* sh_misc, SliceStats* st,
                                                         uint32_t contrib, uint32_t total,
                                                         const KParams& kp) {
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    // warp reductions
    acc.amax_bits = acc.amax();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.amax_bits = max(acc.amax_bits, __shfl_xor_sync(0xffffffffu, acc.amax_bits, o));
        acc.nnz += __shfl_xor_sync(0xffffffffu, acc.nnz, o);
        acc.nonfinite |= __shfl_xor_sync(0xffffffffu, acc.nonfinite, o);
    }
    if (tid == 0) { sh_misc[0] = 0; sh_misc[1] = 0; sh_misc[2] = 0; }
    __syncthreads();
    if ((tid & 31) == 0) {
        atomicMax(&sh_misc[0], acc.amax_bits);
        atomicAdd(&sh_misc[1], acc.nnz);
        atomicOr(&sh_misc[2], acc.nonfinite);
    }
    __syncthreads();
    if (tid == 0) {
        if (sh_misc[0]) atomicMax(&st->amax_bits, sh_misc[0]);
        if (sh_misc[1]) atomicAdd(&st->nnz, sh_misc[1]);
        if (sh_misc[2]) atomicOr(&st->nonfinite, sh_misc[2]);
    }
    for (int b = tid; b < kHistBins; b += nthr) {
        uint32_t c = sh_hist[b];
        if (c) atomicAdd(&st->hist[b], c);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        uint32_t prev = atomicAdd(&st->done, contrib);
        sh_misc[3] = (prev + contrib == total) ? 1u : 0u;
    }
    __syncthreads();
    if (sh_misc[3] && tid < 32) {
        __threadfence();
        int k = select_k_warp(st, kp);
        if (tid == 0) st->k = k;
    }
}

}  // namespace mxfft
