// One pass of the 2D MX-FFT: radix-2 decimation-in-time transforms of length n
// along rows (dim 1) or columns (dim 0) of each slice, every butterfly being
// the MX-scaled complex butterfly of Alg. 2.
//
// A CTA owns `tpc` whole 1D transforms of one slice, held in shared memory in
// bit-reversed order.  For every stage a warp takes 64 consecutive butterflies
// (two per lane: b and b + 32) of one transform; the butterflies of an MX
// block (m consecutive b, m <= 64) therefore sit in aligned groups of lanes,
// and the block maxima of Alg. 2 are reduced with xor shuffles.
#include <cuda_fp16.h>

#include "mx_debug.cuh"
#include "mx_device.cuh"
#include "mxfft.h"

namespace mxfft {

namespace {

constexpr int kPassThreads = 256;

struct Bf {
    float2 u, v;
    float xr, xi;   // twiddle element values (block scale removed)
    int sw;         // twiddle block scale exponent
    int iu, iv;
    bool ok;
};

__device__ __forceinline__ uint32_t abs_max_bits(float a, float b) {
    return max(__float_as_uint(a) & 0x7fffffffu, __float_as_uint(b) & 0x7fffffffu);
}

// Reduce a block maximum over the lanes holding one MX block.  For m <= 32 a
// block is m consecutive lanes of the same half (b or b + 32); for m = 64 it is
// both halves of all 32 lanes.
__device__ __forceinline__ void block_max2(uint32_t& a0, uint32_t& a1, int m) {
    if (m >= 64) { a0 = max(a0, a1); a1 = a0; m = 32; }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (o < m) {
            a0 = max(a0, __shfl_xor_sync(0xffffffffu, a0, o));
            a1 = max(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        }
    }
}

__device__ __forceinline__ void load_bf(Bf& q, const float2* A, int b, int nb, int h,
                                        const float2* __restrict__ tw,
                                        const int8_t* __restrict__ tws) {
    q.ok = b < nb;
    if (q.ok) {
        int j = b & (h - 1);
        q.iu = 2 * b - j;          // 2h*g + j with g = b / h
        q.iv = q.iu + h;
        q.u = A[MX_BND(q.iu, 2 * nb)];
        q.v = A[MX_BND(q.iv, 2 * nb)];
        float2 w = __ldg(tw + (h - 1) + j);
        q.xr = w.x;
        q.xi = w.y;
        q.sw = __ldg(tws + (h - 1) + j);
    } else {
        q.u = q.v = make_float2(0.f, 0.f);
        q.xr = q.xi = 0.f;
        q.sw = 0;
        q.iu = q.iv = 0;
    }
}

// Alg. 2 on the pair of butterflies a lane holds, in the element domain:
//   y = Q(v 2^-s_v)            EncodeBlockMX(v) + MantissasBlock
//   p = x * y (FP32)           element-space complex multiply
//   s_out = s_w + s_v; s^ = clamp(s_out + floor(log2 max|p|) - emax)
//   c = Q(p 2^(s_out - s^))    EncodeFromMantBlock, a fresh MX block
//   wv = c 2^s^                DecodeBlockMX
//   (u + wv, u - wv)           FP32
// The M_max renormalisation of Alg. 2 rescales p and s_out by the same power
// of two before a fresh re-encode, which leaves c and s^ unchanged, so it is
// not performed.
__device__ __forceinline__ void mx_butterfly_pair(float2* A, int b0, int nb, int h, int m,
                                                  const float2* __restrict__ tw,
                                                  const int8_t* __restrict__ tws,
                                                  const FmtParams& fp) {
    Bf q0, q1;
    load_bf(q0, A, b0, nb, h, tw, tws);
    load_bf(q1, A, b0 + 32, nb, h, tw, tws);

    uint32_t a0 = q0.ok ? abs_max_bits(q0.v.x, q0.v.y) : 0u;
    uint32_t a1 = q1.ok ? abs_max_bits(q1.v.x, q1.v.y) : 0u;
    block_max2(a0, a1, m);
    const int sv0 = mx_scale_exp(a0, fp.emax);
    const int sv1 = mx_scale_exp(a1, fp.emax);
    const float inv0 = exp2i(-sv0), inv1 = exp2i(-sv1);

    const float y0r = q_elem(__fmul_rn(q0.v.x, inv0), fp);
    const float y0i = q_elem(__fmul_rn(q0.v.y, inv0), fp);
    const float y1r = q_elem(__fmul_rn(q1.v.x, inv1), fp);
    const float y1i = q_elem(__fmul_rn(q1.v.y, inv1), fp);

    const float p0r = __fsub_rn(__fmul_rn(q0.xr, y0r), __fmul_rn(q0.xi, y0i));
    const float p0i = __fadd_rn(__fmul_rn(q0.xr, y0i), __fmul_rn(q0.xi, y0r));
    const float p1r = __fsub_rn(__fmul_rn(q1.xr, y1r), __fmul_rn(q1.xi, y1i));
    const float p1i = __fadd_rn(__fmul_rn(q1.xr, y1i), __fmul_rn(q1.xi, y1r));

    uint32_t P0 = q0.ok ? abs_max_bits(p0r, p0i) : 0u;
    uint32_t P1 = q1.ok ? abs_max_bits(p1r, p1i) : 0u;
    block_max2(P0, P1, m);

    const int so0 = q0.sw + sv0, so1 = q1.sw + sv1;
    const int sh0 = P0 ? min(max(so0 + ilogb_bits(P0) - fp.emax, -127), 127) : so0;
    const int sh1 = P1 ? min(max(so1 + ilogb_bits(P1) - fp.emax, -127), 127) : so1;
    const float f0 = exp2i(so0 - sh0), f1 = exp2i(so1 - sh1);
    const float d0 = exp2i(sh0), d1 = exp2i(sh1);

    // a block holding Inf/NaN has the NaN shared scale of OCP MX: all NaN
    const float nan0 = a0 >= 0x7f800000u ? __int_as_float(0x7fffffff) : 1.0f;
    const float nan1 = a1 >= 0x7f800000u ? __int_as_float(0x7fffffff) : 1.0f;
    if (q0.ok) {
        const float wr = __fmul_rn(__fmul_rn(q_elem(__fmul_rn(p0r, f0), fp), d0), nan0);
        const float wi = __fmul_rn(__fmul_rn(q_elem(__fmul_rn(p0i, f0), fp), d0), nan0);
        A[MX_BND(q0.iu, 2 * nb)] = make_float2(__fadd_rn(q0.u.x, wr), __fadd_rn(q0.u.y, wi));
        A[MX_BND(q0.iv, 2 * nb)] = make_float2(__fsub_rn(q0.u.x, wr), __fsub_rn(q0.u.y, wi));
    }
    if (q1.ok) {
        const float wr = __fmul_rn(__fmul_rn(q_elem(__fmul_rn(p1r, f1), fp), d1), nan1);
        const float wi = __fmul_rn(__fmul_rn(q_elem(__fmul_rn(p1i, f1), fp), d1), nan1);
        A[MX_BND(q1.iu, 2 * nb)] = make_float2(__fadd_rn(q1.u.x, wr), __fadd_rn(q1.u.y, wi));
        A[MX_BND(q1.iv, 2 * nb)] = make_float2(__fsub_rn(q1.u.x, wr), __fsub_rn(q1.u.y, wi));
    }
}

// FP16 positive control (Sec. 2.2): the twiddle product in IEEE binary16
// arithmetic -- twiddle (a binary16 value) and v rounded to binary16, each
// product, sum and difference rounded once (__hmul_rn is never contracted into
// an FMA) -- then u +- wv in FP32.
__device__ __forceinline__ float2 fp16_product(float2 w, float2 v) {
    const __half wr = __float2half_rn(w.x), wi = __float2half_rn(w.y);   // exact
    const __half vr = __float2half_rn(v.x), vi = __float2half_rn(v.y);
    const __half pr = __hsub(__hmul_rn(wr, vr), __hmul_rn(wi, vi));
    const __half pi = __hadd(__hmul_rn(wr, vi), __hmul_rn(wi, vr));
    return make_float2(__half2float(pr), __half2float(pi));
}

__device__ __forceinline__ void fp16_butterfly_pair(float2* A, int b0, int nb, int h,
                                                    const float2* __restrict__ tw) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int b = b0 + 32 * r;
        if (b >= nb) continue;
        const int j = b & (h - 1);
        const int iu = 2 * b - j, iv = iu + h;
        const float2 u = A[MX_BND(iu, 2 * nb)];
        const float2 p = fp16_product(__ldg(tw + (h - 1) + j), A[MX_BND(iv, 2 * nb)]);
        A[MX_BND(iu, 2 * nb)] = make_float2(__fadd_rn(u.x, p.x), __fadd_rn(u.y, p.y));
        A[MX_BND(iv, 2 * nb)] = make_float2(__fsub_rn(u.x, p.x), __fsub_rn(u.y, p.y));
    }
}

// FP32 reference ablation: the twiddle product and u +- wv in FP32, every
// operation rounded once (the intrinsics are never contracted into an FMA).
__device__ __forceinline__ void fp32_butterfly_pair(float2* A, int b0, int nb, int h,
                                                    const float2* __restrict__ tw) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int b = b0 + 32 * r;
        if (b >= nb) continue;
        const int j = b & (h - 1);
        const int iu = 2 * b - j, iv = iu + h;
        const float2 u = A[MX_BND(iu, 2 * nb)];
        const float2 v = A[MX_BND(iv, 2 * nb)];
        const float2 w = __ldg(tw + (h - 1) + j);
        const float pr = __fsub_rn(__fmul_rn(w.x, v.x), __fmul_rn(w.y, v.y));
        const float pi = __fadd_rn(__fmul_rn(w.x, v.y), __fmul_rn(w.y, v.x));
        A[MX_BND(iu, 2 * nb)] = make_float2(__fadd_rn(u.x, pr), __fadd_rn(u.y, pi));
        A[MX_BND(iv, 2 * nb)] = make_float2(__fsub_rn(u.x, pr), __fsub_rn(u.y, pi));
    }
}

__device__ __forceinline__ float to_fp16(float x) { return __half2float(__float2half_rn(x)); }

__global__ void __launch_bounds__(kPassThreads)
pass_kernel(PassArgs a) {
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int n = a.n, logn = a.logn, tpc = a.tpc;
    const int per_slice = (a.dim == 1 ? a.n0 : a.n1) / tpc;
    const int slice = blockIdx.x / per_slice;
    const int t0 = (blockIdx.x - slice * per_slice) * tpc;
    const size_t sbase = (size_t)slice * a.n0 * a.n1;
    const size_t slice_pts = (size_t)a.n0 * a.n1;     // bounds of the debug build
    (void)slice_pts;
    const float2* __restrict__ in = a.ref ? a.ref[slice].in : a.in + sbase;
    float2* __restrict__ out = a.ref ? a.ref[slice].out : a.out + sbase;
    const SliceStats* stp = a.ref ? a.ref[slice].st : a.st + slice;

    // load (with the Alg. 1 prescale on the first pass) in bit-reversed order
    const float pre = a.prologue == PRO_PRESCALE ? exp2i(stp->k) : 1.0f;
    const bool fp16 = a.fmt == MXFFT_FP16, fp32 = a.fmt == MXFFT_FP32_REF;
    const int total = tpc * n;
    for (int idx = tid; idx < total; idx += nthr) {
        int t, i;
        size_t g;
        if (a.dim == 1) {
            t = idx >> logn;
            i = idx & (n - 1);
            g = (size_t)(t0 + t) * a.n1 + i;
        } else {
            i = idx / tpc;
            t = idx - i * tpc;
            g = (size_t)i * a.n1 + t0 + t;
        }
        float2 v = in[MX_BND(g, slice_pts)];
        if (a.prologue == PRO_PRESCALE) {
            v.x = __fmul_rn(v.x, pre);
            v.y = __fmul_rn(v.y, pre);
            if (fp16) { v.x = to_fp16(v.x); v.y = to_fp16(v.y); }   // input rounding
        }
        sm[MX_BND(t * n + (int)(__brev((unsigned)i) >> (32 - logn)), total)] = v;
    }
    __syncthreads();

    const int nb = n >> 1;
    const int sb_per = (nb + 63) >> 6;
    const int tasks = tpc * sb_per;
    for (int s = 0; s < logn; s++) {
        const int h = 1 << s;
        for (int task = warp; task < tasks; task += nwarps) {
            const int t = task / sb_per;
            const int sb = task - t * sb_per;
            if (fp16) fp16_butterfly_pair(sm + t * n, sb * 64 + lane, nb, h, a.tw);
            else if (fp32) fp32_butterfly_pair(sm + t * n, sb * 64 + lane, nb, h, a.tw);
            else mx_butterfly_pair(sm + t * n, sb * 64 + lane, nb, h, a.m, a.tw, a.tws, a.fp);
        }
        __syncthreads();
    }

    // epilogue: natural order out
    float post = 1.0f;
    if (a.epilogue == EPI_UNSCALE) post = exp2i(-stp->k);
    else if (a.epilogue == EPI_RT_FINAL) post = exp2i(-stp->k - a.lg_total);
    for (int idx = tid; idx < total; idx += nthr) {
        int t, i;
        size_t g;
        if (a.dim == 1) {
            t = idx >> logn;
            i = idx & (n - 1);
            g = (size_t)(t0 + t) * a.n1 + i;
        } else {
            i = idx / tpc;
            t = idx - i * tpc;
            g = (size_t)i * a.n1 + t0 + t;
        }
        float2 v = sm[MX_BND(t * n + i, total)];
        if (a.epilogue != EPI_RAW) {
            // FP16 control: output rounding in the prescaled domain, then the
            // exact unscale
            if (fp16) { v.x = to_fp16(v.x); v.y = to_fp16(v.y); }
            v.x = __fmul_rn(v.x, post);
            v.y = __fmul_rn(v.y, post);
        }
        out[MX_BND(g, slice_pts)] = v;
    }
}

}  // namespace

cudaError_t launch_pass(const PassArgs& a, int batch, cudaStream_t s) {
    const int per_slice = (a.dim == 1 ? a.n0 : a.n1) / a.tpc;
    const size_t smem = (size_t)a.tpc * a.n * sizeof(float2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    pass_kernel<<<batch * per_slice, kPassThreads, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

MX_BOUNDS_COUNTER(pass)

}  // namespace mxfft
