// Building blocks of the tensor-core kernels (mx_tc16.cu, mx_tc2d.cu):
// shared-memory matrix descriptors, 8-bit element conversion, bounded
// mbarrier waits, tensor-memory loads, asynchronous copies and the cluster
// primitives (rank, barrier, distributed shared memory).  Inline PTX for
// sm_100-family GPUs (sm_103a here).
#pragma once

#include <stdint.h>

namespace mxfft {
namespace tcg {

constexpr uint64_t kWaitNs = 100000000;   // bound of one completion wait: 100 ms

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

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase of parity `phase` to complete, at most kWaitNs.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase) {
    uint32_t done = 0;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
                     " selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(mbar), "r"(phase));
        if (done || globaltimer_ns() - t0 > kWaitNs) break;
    }
    return done != 0;
}

// The same bounded wait with the hardware suspending the thread between
// checks (try_wait with a suspend-time hint: the thread sleeps until the
// phase completes or the hint elapses), for a waiter that should not take
// issue slots from the other warps.
__device__ __forceinline__ bool wait_phase_sleep(uint32_t mbar, uint32_t phase) {
    uint32_t done = 0;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;"
                     " selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(mbar), "r"(phase), "r"(1000000u));
        if (done || globaltimer_ns() - t0 > kWaitNs) break;
    }
    return done != 0;
}

// A CTA-wide bounded wait: warp 0 waits on the mbarrier phase, the other
// warps on the CTA barrier (which takes no issue slots); every thread gets
// whether the phase completed.  Every thread of the CTA must call it.  After
// it, shared-memory data that completed the phase (bulk copies) are visible
// to every thread; before reading tensor memory a thread still issues
// tcgen05.fence::after_thread_sync.
__device__ __forceinline__ bool wait_phase_cta(uint32_t mbar, uint32_t phase) {
    bool ok = true;
    if (threadIdx.x < 32) ok = __all_sync(0xffffffffu, wait_phase_sleep(mbar, phase));
    return __syncthreads_or(!ok) == 0;
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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {   // all but the newest group
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}


// ---- packed FP32 arithmetic and block maxima ----------------------------------

// Packed FP32 pairs with an explicit rounding mode: each component is one
// correctly rounded operation.  (A multiply feeding an add may still be
// merged into one fused multiply-add by the code generator: the products
// below are arranged so that such a merge changes no result.)
__device__ __forceinline__ float2 mul2_rn(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5};"
        " mul.rn.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 add2_rn(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5};"
        " add.rn.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5};"
        " sub.rn.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// max(|a|, |b|, |c|), NaN if any input is NaN.
__device__ __forceinline__ float max3_abs_nan(float a, float b, float c) {
    float d;
    asm("max.NaN.abs.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Largest |component| of 16 complex values (NaN if any is NaN): a tree of
// three-input maxima, 17 instructions for 32 values.
__device__ __forceinline__ float vec_max_abs(const float2 (&x)[16]) {
    float a[32];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        a[2 * j] = x[j].x;
        a[2 * j + 1] = x[j].y;
    }
#pragma unroll
    for (int w = 1; w < 32; w *= 3)
#pragma unroll
        for (int t = 0; t < 32; t += 3 * w) {
            if (t + 2 * w < 32) a[t] = max3_abs_nan(a[t], a[t + w], a[t + 2 * w]);
            else if (t + w < 32) a[t] = max3_abs_nan(a[t], a[t + w], a[t + w]);
        }
    return a[0];
}

// ---- thread-block clusters ---------------------------------------------------

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_idx() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives; shared-memory writes made
// before it are visible to the cluster's loads after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// ---- bulk copies into shared memory (completion counted on an mbarrier) ------

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count));
}
// One arrival that also expects `bytes` of copies to complete on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(mbar), "r"(bytes) : "memory");
}
// size bytes (a multiple of 16, both addresses 16-byte aligned) from global
// memory into this CTA's shared memory.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t size, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(size), "r"(mbar) : "memory");
}

}  // namespace tcg
}  // namespace mxfft
