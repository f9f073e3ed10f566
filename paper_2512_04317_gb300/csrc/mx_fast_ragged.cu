// Ragged register-resident pass: one launch covers one axis of the passes of
// many plans (slices of different sizes, formats, directions and epilogues)
// for MX blocks of 16 butterflies (k = 32).  Every CTA has the same shape,
// 256 threads: groups of TG transforms of length n, NG groups per CTA with TG
// (n / 32) NG = 256 (TG = 16, or 8 for n = 1024).  CTA b reads its work from
// a device table, (group, slice of the group, first transform), copies the
// group's arguments (the plan's pass: shape, twiddles, prologue, epilogue,
// slice references) into shared memory and runs the same per-CTA body as
// fast_pass_kernel, with the element format chosen at run time.  Each slice's
// arithmetic is therefore that of the per-plan launch, bit for bit.
#include "mx_fast_kernel.cuh"

namespace mxfft {
namespace fast {
namespace {

constexpr int kRaggedThreads = 256;
constexpr int kRaggedLogM = 4;        // MX blocks of 16 butterflies

template <int DIM, bool FUSED>
__device__ __forceinline__ void ragged_body(const FastArgs& fa, int slice, int t0) {
    switch (fa.a.fmt) {
        case 0: fast_body<0, kRaggedLogM, DIM, FUSED>(fa, slice, t0); break;
        case 1: fast_body<1, kRaggedLogM, DIM, FUSED>(fa, slice, t0); break;
        case 2: fast_body<2, kRaggedLogM, DIM, FUSED>(fa, slice, t0); break;
        case 3: fast_body<3, kRaggedLogM, DIM, FUSED>(fa, slice, t0); break;
        default: fast_body<4, kRaggedLogM, DIM, FUSED>(fa, slice, t0); break;
    }
}

// ctas[b] = (group, slice index within the group's references, first
// transform, unused).  The groups' arguments are one kernel parameter (read
// through the constant bank, like fast_pass_kernel's), so that a per-CTA
// group index costs no registers beyond the per-plan launch.
// WITH_FUSED (columns only): the launch holds fused round-trip groups, whose
// CTAs run both column transforms; it is a separate instance because the
// second body raises register pressure for every group of the launch.
template <int DIM, bool WITH_FUSED>
__global__ void __launch_bounds__(kRaggedThreads, 2)
fast_ragged_kernel(const __grid_constant__ RaggedGroups g, const int4* __restrict__ ctas) {
    const int4 c = ctas[blockIdx.x];
    const FastArgs& fa = g.g[c.x];
    if (WITH_FUSED && fa.fused) ragged_body<0, true>(fa, c.y, c.z);
    else ragged_body<DIM, false>(fa, c.y, c.z);
}

}  // namespace

cudaError_t launch_ragged(const RaggedGroups& groups, const int4* ctas, int nctas, int dim,
                          size_t smem, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    if (groups.n < 1 || groups.n > kMaxRaggedGroups) return cudaErrorInvalidValue;
    bool fused = false;
    for (int i = 0; i < groups.n; i++) fused |= groups.g[i].fused != 0;
    if (fused && dim != 0) return cudaErrorInvalidValue;
    const int kind = dim == 1 ? 0 : (fused ? 2 : 1);
    void (*k)(const RaggedGroups, const int4*) =
        kind == 0 ? fast_ragged_kernel<1, false>
                  : (kind == 1 ? fast_ragged_kernel<0, false> : fast_ragged_kernel<0, true>);
    // raise the opt-in limit only (launches captured earlier may need more)
    static size_t smem_limit[3] = {0, 0, 0};
    if (smem > smem_limit[kind]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_limit[kind] = smem;
    }
    k<<<nctas, kRaggedThreads, smem, s>>>(groups, ctas);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fast
}  // namespace mxfft
