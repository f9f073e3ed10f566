// Plan object shared by the C ABI (mxfft_api.cu) and the batch executor
// (mx_engine.cu), with the pass helpers both use.
#pragma once

#include <vector>

#include "mx_internal.h"
#include "mxfft.h"

namespace mxfft {
struct ProfRec {
    int kind;                  // 0 stats, 1 pass
    cudaEvent_t a, b;
};
}  // namespace mxfft

using mxfft::ProfRec;

struct mxfft_plan_s {
    int n0, n1, fmt, kblk;
    float tau;
    int t_exp;                 // target = 2^t_exp
    int taumin_exp;            // tau_min = 2^taumin_exp
    int kmin, kmax;
    mxfft::FmtParams fp;
    int m[2];                  // MX block size in butterflies per axis (0: n0, 1: n1)
    float2* d_tw[2][2];        // [axis][0 forward, 1 inverse]
    int8_t* d_tws[2];          // [axis] twiddle block exponents
    uint32_t* d_twh[2][2];     // [axis][dir] f16x2 twiddle element values
    mxfft::TwA twa[2][2];             // [axis][dir] stages h <= 16 for the register pass
    int force_generic;         // 1: always use the generic pass kernel
    int path;                  // 0 radix-2 MX, 1 tensor-core radix-16
    int test_stall;            // MXFFT_OPT_TEST_STALL
    uint8_t* d_bmat[2];        // [dir] tensor-core DFT matrix codes (core-matrix layout)
    uint8_t* d_bmat8[2];       // [dir] the same for two 8-point DFTs (n = 128 axes)
    float2* d_twA[2][2];       // [axis][dir] radix-16 stage twiddles
    float2* d_twC[2][2];       // [axis][dir] twiddles before the radix-2 stage (n = 512)
    float4* d_tw4A[2][2];      // [axis][dir] radix-16 stage twiddles as (re, re, -im, im)
    float4* d_tw4C[2][2];      // [axis][dir] twiddles before the radix-2 stage
    int fused2d;               // MXFFT_OPT_FUSED2D: fused 2D transform where it applies
    int fold_stats;            // MXFFT_OPT_FOLD_STATS: round-trip inverse statistics in the columns pass
    int* d_err;                // device flag: a bounded wait gave up
    mxfft::SliceStats* d_st;          // 2 * st_cap records: forward, inverse
    int st_cap;
    int last_batch, last_op;   // of the last transform
    cudaStream_t last_stream;
    int device;
    bool prof;                 // record per-kernel event pairs
    std::vector<ProfRec>* recs;
};

namespace mxfft {

// mxfft_status of a CUDA error code.
int cuda_status(cudaError_t e);
// Exponent selection parameters of a plan.
KParams kparams(const mxfft_plan_s* p);
// Arguments of a pass of plan p along dim (1 rows, 0 columns) in direction dir
// (0 forward, 1 inverse); st, prologue and epilogue are left for the caller.
PassArgs pass_args(const mxfft_plan_s* p, int dim, int dir, const float2* in, float2* out);
// Whether a plan's forward / inverse transforms run as the fused 2D
// tensor-core kernel; its arguments for one launch (dir 0 forward, 1 inverse).
// Arguments of the tensor-core pass for pass a of plan p in direction dir.
mxfft::Tc16Args tc16_args(const mxfft_plan_s* p, const mxfft::PassArgs& a, int dir);
// true when the tensor-core columns pass of a round trip accumulates the
// inverse's prescale statistics of its output (no separate statistics pass)
bool tc16_folds_stats(const mxfft_plan_s* p);
bool uses_tc2d(const mxfft_plan_s* p);
Tc2dArgs tc2d_args(const mxfft_plan_s* p, int dir, const float2* in, float2* out, SliceStats* st,
                   int epilogue);
// The fused 2D launch (profiled as kind 4); cudaErrorNotSupported when the
// device cannot run it (the caller then runs the passes).
cudaError_t timed_tc2d(mxfft_plan_s* p, const Tc2dArgs& a, int batch, cudaStream_t s);
// Launch one pass over batch slices with the plan's kernel choice.
cudaError_t timed_pass(mxfft_plan_s* p, const PassArgs& a, int batch, cudaStream_t s);
cudaError_t fused_cols_pass(mxfft_plan_s* p, const PassArgs& a, int batch, cudaStream_t s);
// Copy the per-slice "non-finite input" flags of an engine's last run to
// pinned host memory, asynchronously on s (mx_engine.cu).
cudaError_t engine_flags_async(mxfft_engine_t e, uint32_t* h_flags, cudaStream_t s);

}  // namespace mxfft
