// Internal declarations shared by the translation units of libmxfft.
// Not part of the public C ABI (include/mxfft.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace mxfft {

// Kernel launches made by this library in the process (each launcher adds
// one per kernel it enqueues); the executor reports per-run differences.
extern std::atomic<long long> g_kernel_launches;
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

// Element-format constants in the form the device quantiser uses.
struct FmtParams {
    int emax;            // unbiased exponent of the largest normal
    int emin;            // unbiased exponent of the smallest normal
    int mbits;           // mantissa bits
    float maxnorm;       // largest finite magnitude
    uint32_t qmin_bits;  // float bits of 2^emin with a zero mantissa: (emin+127) << 23
    uint32_t qadd_bits;  // ((23 - mbits) << 23) | 0x400000: turns 2^E into 1.5 * 2^(E+23-mbits)
};

#ifdef MXFFT_DEBUG_BOUNDS
// Readers of the bounds-check counters of the instrumented translation units
// (each returns its count and clears it; ~0 on a CUDA error).
unsigned long long bounds_take_fast_f0();
unsigned long long bounds_take_fast_f1();
unsigned long long bounds_take_fast_f2();
unsigned long long bounds_take_fast_f3();
unsigned long long bounds_take_fast_f4();
unsigned long long bounds_take_pass();
unsigned long long bounds_take_tc16();
unsigned long long bounds_take_tc2d();
#endif

// Element-format constants of an mxfft_format code (false for an unknown code).
bool fmt_params(int code, FmtParams* fp);

// Per-slice statistics of Alg. 1 (one record per slice and transform).
// Zeroed before every transform that accumulates into it.
struct SliceStats {
    uint32_t amax_bits;   // bits of max |x| (nonnegative floats order as integers)
    uint32_t nnz;         // number of nonzero magnitudes
    uint32_t nonfinite;   // nonzero when some |x| was Inf/NaN
    uint32_t done;        // CTAs finished (the last one selects k)
    int32_t k;            // selected prescale exponent
    uint32_t pad[3];
    uint32_t hist[280];   // counts of floor(log2 |x|) + 149, bins 0..276
};
static_assert(sizeof(SliceStats) % 16 == 0, "SliceStats alignment");

constexpr int kHistBins = 277;   // floor(log2 m) in [-149, 127]

// Integer parameters of the exponent selection (Alg. 1).
struct KParams {
    float tau;        // percentile fraction
    int t_exp;        // target = 2^t_exp
    int taumin_exp;   // tau_min = 2^taumin_exp
    int kmin, kmax;   // clip bounds
};

// Prologue / epilogue modes of a pass.
enum PassPrologue { PRO_NONE = 0, PRO_PRESCALE = 1 };
enum PassEpilogue {
    EPI_RAW = 0,          // store the FP32 stage output
    EPI_UNSCALE = 1,      // store 2^-k * A
    EPI_RT_FINAL = 3      // store 2^(-k - lg_total) * A (k of the inverse)
};

// Buffers of one slice when the slices of a launch are not one strided batch
// (the ragged batch executor): the slice reads in, writes out and takes its
// prescale exponent from *st.
struct SliceRef {
    const float2* in;
    float2* out;
    SliceStats* st;
    SliceStats* st_out;     // non-null: accumulate the statistics of this pass's
                            // output here (the round trip's inverse prescale)
};
static_assert(sizeof(SliceRef) == 32, "32-byte slice references");

struct PassArgs {
    const float2* in;
    float2* out;
    const SliceRef* ref;  // non-null: slice i uses ref[i] instead of in/out/st + i
    int n0, n1;           // slice shape
    int dim;              // 1: transform rows (length n1); 0: columns (length n0)
    int n, logn;          // transform length and log2
    int tpc;              // transforms per CTA
    int m;                // MX block size in butterflies: min(k/2, n/2)
    const float2* tw;     // twiddle element values, index (h - 1) + j per stage h
    const int8_t* tws;    // twiddle block scale exponent for the same index
    SliceStats* st;       // statistics holding k for the prologue / epilogue
    SliceStats* st_out;   // non-null (strided batches): statistics of the output
    int stats_out;        // 1: accumulate the output's statistics (st_out / ref[i].st_out)
    int prologue, epilogue;
    int lg_total;         // log2(n0 * n1) for EPI_RT_FINAL
    int fmt;              // element format code (mxfft_format)
    FmtParams fp;
    KParams kp;           // exponent selection parameters of the plan
};

// Twiddles of stages h = 1..16 (index h - 1 + j) for the register-resident
// pass: identical for every 32-element chunk, passed as kernel parameters.
struct TwA {
    uint32_t h2[32];   // f16x2 {re, im} twiddle element values
    int8_t sw[32];     // twiddle block scale exponents
};

// Arguments of the tensor-core radix-16 pass (mx_tc16.cu).
struct Tc16Args {
    const float2* in;
    float2* out;
    const SliceRef* ref;              // as in PassArgs
    int n0, n1, dim, n, r;            // n = 256 r, r in {1, 2, 4, 8}, or n = 128 (r = 0)
    int batch;                        // slices (set by launch_tc16_pass)
    const uint8_t* bmat;              // B operand: 32 x 32 element codes, core-matrix layout (1 KB)
    const uint8_t* bmat2;             // n = 128: the 8-point DFT twice on the diagonal (same layout)
    const float2* twA;                // [j2 < 16 r][k1 < 16] twiddle element values x 2^s
    const float2* twC;                // [j22 < r][k21 < 16] (r > 1)
    SliceStats* st;
    int prologue, epilogue, lg_total;
    uint32_t idesc;                   // tcgen05 instruction descriptor
    int* err;                         // set when a bounded wait gives up
    int stall;                        // test hook: issue no matrix product
    int g;                            // vectors per MX block: k / 32 (1, 2, 4)
    int inv;                          // 1: inverse transform (sign of the radix-4 stage)
    SliceStats* st_out;               // columns pass, strided batches: Alg. 1 statistics of
                                      // the output accumulated here (see SliceRef::st_out)
    int stats_out;                    // 1: accumulate output statistics (records per slice
                                      // from st_out or the references; null records skipped)
    KParams kp;                       // exponent selection of those statistics
};

// Arguments of the fused 2D tensor-core transform (mx_tc2d.cu): every slice
// [n0][n1] (n0, n1 in {256, 512}) on one thread-block cluster, Alg. 1's
// statistics taken on chip (k written to the slice's record), rows and
// columns, the epilogue scaling.
struct Tc2dArgs {
    const float2* in;
    float2* out;
    const SliceRef* ref;              // as in PassArgs
    SliceStats* st;
    int batch, n0, n1;
    const uint8_t* bmat;              // B operand: 32 x 32 element codes (core-matrix layout)
    const float4* twA1;               // rows: [j2 < M1][k1 < 16] (w.re, w.re, -w.im, w.im) x 2^s
    const float4* twC1;               // rows: [j22 < r1][k21 < 16]
    const float4* twA0;               // columns
    const float4* twC0;
    int epilogue;                     // EPI_UNSCALE, EPI_RT_FINAL (k of this transform) or EPI_RAW
    int lg_total;
    uint32_t idesc;                   // tcgen05 instruction descriptor (M 128, N 32)
    int* err;                         // set when a bounded wait gives up
    int stall;                        // test hook: issue no matrix product
    KParams kp;
};

// One slice of a ragged statistics launch (slices of different sizes and
// plans in one grid): its points, its record, its point count (even), the
// number of CTAs that cover it and its plan's selection parameters.
struct StatsRef {
    const float2* x;
    SliceStats* st;
    int npts;
    uint32_t ctas;
    KParams kp;
};
constexpr int kStatsPtsPerCta = 4096;   // points per CTA of the statistics pass

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_stats(const float2* x, int batch, int n0, int n1, SliceStats* st,
                         KParams kp, cudaStream_t s);
// Ragged statistics: CTA c covers chunk cta_tab[c].y (kStatsPtsPerCta points)
// of slice refs[cta_tab[c].x]; the tables are device memory.
cudaError_t launch_stats_ref(const StatsRef* refs, const int2* cta_tab, int nctas, cudaStream_t s);
cudaError_t launch_pass(const PassArgs& a, int batch, cudaStream_t s);
// Register-resident pass for n in [64, 2048] and m <= 16; returns
// cudaErrorNotSupported (launching nothing) outside that range.
bool fast_pass_supported(const PassArgs& a);
cudaError_t launch_fast_pass(const PassArgs& a, const uint32_t* twh, const TwA& twa, int batch,
                             cudaStream_t s);
// Forward then inverse columns of the fused round trip in one launch (dim 0,
// forward twiddles in twh / twa, inverse in twh_inv / twa_inv).
cudaError_t launch_fast_pass_fused(const PassArgs& a, const uint32_t* twh, const TwA& twa,
                                   const uint32_t* twh_inv, const TwA& twa_inv, int batch,
                                   cudaStream_t s);
// The root-sum-of-squares coil combine of one item: images x coils consecutive
// complex slices of npts points -> images real slices (mx_rss.cu).
struct RssRef {
    const float2* z;
    float* out;
    int coils;
    int images;
    long long npts;
};
// With dev non-null the kernel reads the item from device memory (so that a
// captured graph follows table updates); else it uses val.
cudaError_t launch_rss(const RssRef& val, const RssRef* dev, long long images, long long npts,
                       cudaStream_t s);

// Groups of TG transforms per CTA of the register-resident pass: valid values
// for (n, other), the tuned value for a launch (0 if none), and the table the
// autotuner fills (mx_tune.cu).
int fast_ng_candidates(int n, int other, int m, int* out, int max);
int fast_ng_tuned(int n, int other, int dim, int fmt, int m, int batch);
void fast_ng_store(int n, int other, int dim, int fmt, int m, int batch, int ng, double us);
// Ragged register-resident pass: one launch over many plans' passes along
// one axis (k = 32, n in [64, 1024]), every CTA 256 threads.  A group's
// arguments are filled on the host into fast_ragged_arg_size() bytes (with
// twa2 / twh2 for the fused round trip's columns); tpc receives the
// transforms per CTA and smem the CTA's dynamic shared memory.  ctas[b] =
// (group, slice within the group's references, first transform, 0).
bool fast_ragged_supported(const PassArgs& a);
size_t fast_ragged_arg_size();
bool fast_ragged_fill(void* dst, const PassArgs& a, const uint32_t* twh, const TwA& twa,
                      const uint32_t* twh2, const TwA* twa2, int* tpc, size_t* smem);
// groups: ngroups filled records on the host (at most fast_ragged_max_groups()).
int fast_ragged_max_groups();
cudaError_t launch_fast_ragged(const void* groups, int ngroups, const int4* ctas, int nctas, int dim,
                               size_t smem, cudaStream_t s);
// The register-resident pass with ng groups per CTA (ng = 0: tuned or default).
cudaError_t launch_fast_pass_ng(const PassArgs& a, const uint32_t* twh, const TwA& twa, int batch,
                                int ng, cudaStream_t s);
// Fused 2D tensor-core transform: n0, n1 in {256, 512}, 8-bit formats, k = 32;
// cudaErrorNotSupported (launching nothing) when the device cannot hold the
// kernel's cluster.
bool tc2d_supported(int n0, int n1, int fmt, int kblk);
// Clusters of the fused kernel for this shape and format that the current
// device holds at once (0: it cannot run it).
int tc2d_resident_clusters(int n0, int n1, int fmt);
cudaError_t launch_tc2d(const Tc2dArgs& a, int fmt, cudaStream_t s);
// Tensor-core radix-16 pass: n in {128, 256, 512, 1024, 2048}, 8-bit formats,
// other a multiple of 4096 / n.  Launch geometry: tiles of 4096 points on
// CTAs of 256 threads, or (n <= 1024) tiles of 2048 points on CTAs of 128
// threads; the persistent grid holds ctas_per_sm CTAs per SM (at most what
// an SM holds; 0: all of them).  launch_tc16_pass takes the tuned geometry
// (tile 0: 4096, all that fit).
bool tc16_supported(int n, int other, int fmt);
cudaError_t launch_tc16_pass(const Tc16Args& a, int fmt, int batch, cudaStream_t s);
cudaError_t launch_tc16_pass_geo(const Tc16Args& a, int fmt, int batch, int tile, int ctas_per_sm,
                                 cudaStream_t s);
constexpr int kTc16MaxCtasPerSm = 8;
// The autotuner's table (mx_tune.cu): the tuned (tile, CTAs per SM) of a
// tensor-core launch (0, 0 if none), and storing one.
void tc16_geo_tuned(int n, int other, int dim, int fmt, int g, int batch, int* tile, int* ctas);
void tc16_geo_store(int n, int other, int dim, int fmt, int g, int batch, int tile, int ctas,
                    double us);

}  // namespace mxfft
