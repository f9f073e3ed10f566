/*
 * mxfft.h -- C ABI of the GB300 (sm_103a) MX-scaled low-precision 2D FFT.
 *
 * The method is "A mixed precision FFT with applications in MRI"
 * (arXiv 2512.04317): a single power-of-two global prescale per 2D slice
 * (Alg. 1, Sec. 2.1), then radix-2 iterative decimation-in-time butterflies
 * along rows and then columns, where the twiddle multiply of every butterfly
 * is the MX-scaled complex multiply of Alg. 2 (Sec. 2.2): operands re-encoded
 * as MX blocks of k real elements sharing a power-of-two scale, quantised to
 * an OCP element format (FP8 e4m3/e5m2, FP6 e2m3/e3m2, FP4 e2m1), multiplied
 * in FP32, re-encoded, decoded and accumulated in FP32.  The round trip is
 * (1/(n0 n1)) F^-1{F{x}} of Eq. (1).
 *
 * Conventions shared by every entry point:
 *   - Data are interleaved complex64 (float re, float im), laid out
 *     [batch][n0][n1] with n1 contiguous.  "Rows" are the length-n1
 *     transforms along the contiguous axis; rows are transformed first.
 *   - Data pointers are DEVICE pointers owned by the caller, 16-byte aligned.
 *     in == out (in place) is allowed; any other overlap is not.
 *   - The stream argument is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  Transforms are asynchronous on that stream;
 *     argument errors are reported synchronously by the return value.
 *   - Every function returns an mxfft_status (0 = MXFFT_OK).  Nothing aborts,
 *     prints or throws.  Conditions found on the device (a non-finite
 *     magnitude in an input) are recorded in the plan and read back with
 *     mxfft_get_status after the stream has been synchronised.
 *   - A plan is not safe for concurrent calls from two host threads or on two
 *     streams at once; use one plan per stream.
 */
#ifndef MXFFT_H
#define MXFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MXFFT_OK = 0,
    MXFFT_ERR_INVALID = 1,      /* bad argument (size, pointer, alignment, value) */
    MXFFT_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement */
    MXFFT_ERR_NOMEM = 3,        /* device or host allocation failed */
    MXFFT_ERR_CUDA = 4,         /* a CUDA runtime call failed (no device, launch error) */
    MXFFT_ERR_NONFINITE = 5,    /* an input slice held a non-finite magnitude */
    MXFFT_ERR_TIMEOUT = 6       /* a bounded device wait gave up */
} mxfft_status;

/* Element formats of the MX blocks (OCP 8-bit FP and OCP MX v1.0 types), and
 * the FP16 positive control. */
typedef enum {
    MXFFT_E4M3 = 0,   /* FP8, 3 mantissa bits, largest normal 448 */
    MXFFT_E5M2 = 1,   /* FP8, 2 mantissa bits, largest normal 57344 */
    MXFFT_E2M3 = 2,   /* FP6, 3 mantissa bits, largest normal 7.5 */
    MXFFT_E3M2 = 3,   /* FP6, 2 mantissa bits, largest normal 28 */
    MXFFT_E2M1 = 4,   /* FP4, 1 mantissa bit, largest normal 6 */
    MXFFT_FP16 = 5    /* the FP16 positive control of Sec. 2.2, not an MX format: the same
                         prescale and radix-2 dataflow, each transform's input (after the
                         prescale) and output (before the exact unscale) rounded to IEEE
                         binary16 -- the control runs in the prescaled domain --
                         each butterfly's twiddle product formed in binary16 arithmetic
                         (twiddle and v in binary16, every operation rounded once), u +- wv
                         in FP32.  k is ignored; tau_min default 2^-24 (binary16's smallest
                         magnitude), so the prescale sets the peak to the target and stage
                         values stay below n0 n1 target (no overflow up to 256x256 at
                         target 0.5); products overflow to infinity above 65504. */,
    MXFFT_FP32_REF = 6 /* reference ablation, not an MX format: the same prescale, radix-2
                         dataflow and unscale with no quantisation -- twiddles rounded once to
                         FP32 (exact at multiples of pi/4), the butterfly's complex product and
                         u +- wv in FP32, each operation rounded once -- so that its distance
                         to an MX format's result is the quantisation error alone.  Default
                         tau_min 2^-126.  Radix-2 path only. */
} mxfft_format;

/* Keys of mxfft_set_option. */
typedef enum {
    MXFFT_OPT_TAU_MIN = 0,  /* tail floor tau_min of Alg. 1; a power of two.
                               Default 2^-10 (e4m3, FP6, FP4), 2^-12 (e5m2), 2^-24 (FP16). */
    MXFFT_OPT_K_MIN = 1,    /* lower clip k_min of Alg. 1, integer in [-126, 126]; default -126 */
    MXFFT_OPT_K_MAX = 2,    /* upper clip k_max of Alg. 1, integer in [-126, 126]; default 126 */
    MXFFT_OPT_GENERIC = 3,  /* 1: run every pass on the generic shared-memory kernel instead of
                               the register-resident one (same results; for testing); default 0 */
    MXFFT_OPT_PATH = 4      /* 0: radix-2 MX path (Alg. 2 in every butterfly, bit-exact with the
                               oracle), the default.  1: tensor-core variant: radix-16 sub-DFTs
                               as MXFP8 matrix products on tcgen05 (FP32 accumulation), each
                               16-point input vector one MX block for k = 32 (k = 64 / 128: a
                               block of 2 / 4 consecutive vectors of a transform; other k
                               MXFFT_ERR_UNSUPPORTED), MX-quantised twiddles between the
                               radix-16 stages (n = 128: 16 x 8, the 8-point DFTs of the second
                               round two per matrix row); approximate, not bit-exact.
                               Needs n0, n1 in {128, 256, 512, 1024, 2048} and format E4M3 or
                               E5M2, else MXFFT_ERR_UNSUPPORTED. */,
    MXFFT_OPT_TEST_STALL = 5, /* test hook of the bounded wait, 0 or 1; default 0.  1: the
                               tensor-core kernels withhold their matrix products, so every
                               CTA's wait for their completion runs out (after 100 ms), the CTA
                               stops issuing work, and mxfft_get_status returns
                               MXFFT_ERR_TIMEOUT (device flag bit 1); the outputs of such a
                               call are undefined.  No effect on the radix-2 path. */
    MXFFT_OPT_FUSED2D = 6     /* tensor-core path only, 0 or 1; default 0.  1: forward,
                               inverse and round trip of n0, n1 in {256, 512} with k = 32 run
                               as one fused kernel per transform: each slice is spread over
                               one thread-block cluster (n0 n1 / 16384 CTAs, one per SM), its
                               prescale statistics (Alg. 1) are reduced on chip, and rows and
                               columns are transformed without the slice leaving the chip
                               (16 bytes of HBM traffic per point and transform).  Same
                               arithmetic per element as the per-axis tensor-core passes.
                               0: the statistics pass and the two per-axis passes, which
                               are faster on GB300 (all SMs busy, loads overlapped with
                               compute; the fused kernel keeps one CTA per SM and at 512x512
                               only 7 sixteen-CTA clusters fit at once).  When the device
                               cannot hold the cluster the passes run instead.  The fused
                               round trip (mxfft_roundtrip_fused) always runs the passes. */,
    MXFFT_OPT_FOLD_STATS = 7  /* tensor-core path only, 0 or 1; default 0.  1: the round
                               trip's forward columns pass accumulates the inverse's Alg. 1
                               statistics of the values it stores (n0 != 2048), so no
                               statistics pass re-reads the forward output; same exponents
                               and results.  Off by default: the histogram work lands on
                               the pass's critical path and costs about as much time as
                               the statistics pass it removes (more at 512x512). */
} mxfft_option;

typedef struct mxfft_plan_s *mxfft_plan_t;

/*
 * mxfft_plan -- create a plan for n0 x n1 slices.
 *   n0, n1  powers of two in [2, 2048].
 *   format  an mxfft_format.
 *   k       MX block size in REAL elements (the paper's B, Sec. 2.2: B = 32 is
 *           "32 real elements", B = 2 one complex value): a power of two in
 *           [2, 128].  A block holds min(k/2, n/2) complex values: a run of
 *           consecutive butterflies of one stage of one 1D transform, in the
 *           order b = g*h + j (g the butterfly group, j the index in it).
 *   tau     tail percentile of Alg. 1 as a FRACTION in (0, 1) (1e-3 means the
 *           0.1th percentile); the "lower" order statistic of the nonzero
 *           magnitudes, rank floor(fl32(tau * fl32(n_nz - 1))).
 *   target  target peak of Alg. 1; a positive power of two (the paper uses 0.5).
 *   out     receives the plan (owned by the caller; free with mxfft_destroy).
 * Allocates the device twiddle tables (prequantised per stage and block at
 * plan time) and the per-slice statistics; needs a current CUDA device.
 * Returns MXFFT_ERR_INVALID for out-of-range arguments, MXFFT_ERR_UNSUPPORTED
 * for a target that is not a power of two, MXFFT_ERR_CUDA / _NOMEM on
 * device failures.
 */
int mxfft_plan(int n0, int n1, int format, int k, float tau, float target,
               mxfft_plan_t *out);

/* mxfft_set_option -- set an mxfft_option on a plan (see the enum for ranges).
 * Returns MXFFT_ERR_INVALID for an unknown key or an out-of-range value. */
int mxfft_set_option(mxfft_plan_t plan, int key, double value);

/*
 * mxfft_forward -- forward MX-FFT of `batch` slices (Alg. 1, then Alg. 2 in
 * every butterfly of the row pass and the column pass; Eq. 1 "forward").
 * Each slice gets its own prescale exponent k (Alg. 1) and its output is
 * unscaled by 2^-k.  batch >= 0 (0 is a no-op).  The plan's statistics grow
 * with the largest batch seen (a synchronous device allocation on growth).
 */
int mxfft_forward(mxfft_plan_t plan, const void *in, void *out, int batch,
                  void *stream);

/* mxfft_inverse -- inverse MX-FFT: conjugate twiddles, its own prescale,
 * unnormalised (Eq. 1 applies 1/N^2 outside the inverse). */
int mxfft_inverse(mxfft_plan_t plan, const void *in, void *out, int batch,
                  void *stream);

/*
 * mxfft_roundtrip -- (1/(n0 n1)) F^-1{F{x}} per slice (Eq. 1 "round-trip"):
 * the forward output y = 2^-k A is formed, the inverse takes its own prescale
 * k_inv from y, and one scaling by 2^(-k_inv - log2(n0 n1)) ends it.
 * `out` also serves as the intermediate buffer.  On the tensor-core path
 * with MXFFT_OPT_FOLD_STATS (n0 != 2048) the forward columns pass
 * accumulates y's statistics as it stores y, so no separate statistics pass
 * over y runs; k_inv is the same exponent either way.
 */
int mxfft_roundtrip(mxfft_plan_t plan, const void *in, void *out, int batch,
                    void *stream);

/*
 * mxfft_roundtrip_fused -- the fused encode -> F -> F^-1 -> decode round trip
 * of Sec. 4.3, a declared variant of mxfft_roundtrip: one prescale k of the
 * input (Alg. 1), the forward transform (rows, then columns), the inverse
 * applied directly to the forward result A (no unscale, no second prescale),
 * columns first and then rows, and one scaling by 2^(-k - log2(n0 n1)).  Both
 * column transforms of a tile run in one kernel on chip where the
 * register-resident pass applies, so the call makes one statistics pass and
 * three passes over the slice instead of two and four.  Same MX blocks as the
 * separate transforms; the result differs from mxfft_roundtrip only through
 * the inverse's axis order and the missing second prescale.  Arguments as for
 * mxfft_roundtrip.  MXFFT_ERR_UNSUPPORTED for the FP16 control (its binary16
 * products would overflow at the unscaled intermediate size).  k_out of
 * mxfft_get_status: [batch], the one prescale exponent per slice.
 */
int mxfft_roundtrip_fused(mxfft_plan_t plan, const void *in, void *out, int batch,
                          void *stream);

/*
 * mxfft_get_status -- after the stream of the last call has been synchronised
 * (this function synchronises it), report what the device saw in that call.
 *   device_flags  nullable; receives bit 0 = some slice had a non-finite
 *                 magnitude (its k was forced to 0, its output is undefined),
 *                 bit 1 = a bounded wait of the tensor-core path gave up (its
 *                 output is undefined).
 *   k_out         nullable; receives the prescale exponents of the last call:
 *                 [batch] for forward / inverse / fused round trip,
 *                 [batch][2] (forward k, inverse k) for the round trip.
 * Returns MXFFT_ERR_NONFINITE when bit 0 is set, MXFFT_ERR_TIMEOUT when bit 1
 * is set, else MXFFT_OK (or a CUDA error).
 */
int mxfft_get_status(mxfft_plan_t plan, int *device_flags, int32_t *k_out);

/* mxfft_destroy -- free a plan and its device memory (NULL is a no-op).
 * Synchronises the device work of the plan first. */
int mxfft_destroy(mxfft_plan_t plan);

/*
 * Instrumentation (no counterpart in the paper): per-kernel device time.
 * mxfft_profile(plan, 1) makes the plan record a CUDA event pair on the
 * caller's stream around every kernel it launches; mxfft_profile(plan, 0)
 * stops recording.  mxfft_profile_read synchronises on the recorded events,
 * writes for each kernel kind i < nkinds the summed device time total_ms[i]
 * and the launch count launches[i], and clears the records.  Kinds:
 * 0 = statistics kernel (Alg. 1), 1 = generic MX butterfly pass kernel,
 * 2 = register-resident MX butterfly pass kernel (rows and columns of
 * length 64..2048 with k <= 32, and of length 128..2048 with k = 64 or 128),
 * 3 = tensor-core radix-16 pass kernel, 4 = fused 2D tensor-core kernel (a
 * whole transform per launch).  Returns MXFFT_ERR_INVALID for a NULL plan or
 * nkinds < 1.
 */
int mxfft_profile(mxfft_plan_t plan, int enable);
int mxfft_profile_read(mxfft_plan_t plan, double *total_ms, int *launches, int nkinds);

/*
 * mxfft_prescale_exponents_noalloc -- allocation-free entry point; the paper
 * has no counterpart (it is a deployment facility).
 *
 * For callers that cannot allocate device memory when they call in: a thread
 * that runs inside another framework's fixed memory pool, a real-time
 * acquisition and reconstruction loop that must not reach the CUDA allocator,
 * or code that has already committed all free device memory.  It computes the
 * prescale exponent k of each of `batch` slices -- the same exponents that
 * mxfft_forward selects for them, by the same statistics kernel -- without a
 * plan and without any cudaMalloc, cudaFree or allocating library call.
 *   in      device pointer to [batch][n0][n1] complex64, 16-byte aligned.
 *   batch   0 .. MXFFT_NOALLOC_MAX_SLICES; a larger batch returns
 *           MXFFT_ERR_INVALID because the scratch is a fixed static array
 *           (split the batch into several calls).
 *   n0, n1, format, tau, target  as for mxfft_plan, with the plan defaults for
 *           tau_min and (k_min, k_max).
 *   k_out   device pointer to `batch` int32 exponents (4-byte aligned),
 *           written asynchronously on `stream`; a slice holding a non-finite
 *           magnitude gets 0, like the transforms.
 * Scratch: one file-scope device array of MXFFT_NOALLOC_MAX_SLICES per-slice
 * records (about 1.2 MB).  Every call uses it and it keeps the last call's
 * contents; each call clears the records it needs first.  Calls that overlap
 * on the GPU (two streams, or two host threads without ordering) race on it:
 * serialise them.
 * Set-up: the CUDA runtime loads this library's device code, array included,
 * lazily, on a device's first use of it; from then on the device holds the
 * array until the process exits.  The first call on a device, made with that
 * device current, looks up the array's device address (cudaGetSymbolAddress)
 * and so may be the call that loads the module, which itself takes device
 * memory.  Make that first call at initialisation time, while memory is still
 * free and before any stream capture; later calls allocate nothing.  After a
 * cudaDeviceReset the next call looks the address up again in the new
 * context (and loads the module again).
 */
#define MXFFT_NOALLOC_MAX_SLICES 1024
int mxfft_prescale_exponents_noalloc(const void *in, int batch, int n0, int n1, int format,
                                     float tau, float target, int32_t *k_out, void *stream);

/* ======================================================================
 * Ragged batch executor.  Not a construct of the paper: it runs many
 * independent 2D transforms of the method (each exactly as mxfft_forward /
 * mxfft_inverse / mxfft_roundtrip would on its own) in one set of launches:
 * one statistics launch over every slice of every item (Alg. 1), then for
 * the radix-2 plans with k = 32 and n0, n1 <= 1024 one ragged launch per
 * axis and stage over all of them (every CTA takes its slice, plan and
 * transforms from a device table), so any mix of such plans takes at most 6
 * launches (statistics, rows, columns, and for round trips statistics,
 * inverse rows, inverse columns); other plans (tensor-core, other k, the
 * generic pass) one launch per pass and (plan, direction) group, as parallel
 * branches (with MXFFT_ENGINE_FOLD_STATS, round trips on the tensor-core
 * path take their inverse statistics in the forward columns pass: no second
 * statistics launch for them).
 * Results are bit-identical to the per-plan calls.
 * ====================================================================== */
typedef enum {
    MXFFT_OP_FORWARD = 0,
    MXFFT_OP_INVERSE = 1,
    MXFFT_OP_ROUNDTRIP = 2,
    MXFFT_OP_ROUNDTRIP_FUSED = 3   /* mxfft_roundtrip_fused */
} mxfft_op;

/* One work item: `slices` independent [n0][n1] slices (slices x coils of an
 * MRI volume) transformed with the plan (n0, n1, format, k) of the engine's
 * tau and target.  in / out are device pointers, 16-byte aligned; in == out
 * is allowed, other overlaps (also between items) are not. */
typedef struct {
    int n0, n1;
    int format;
    int k;
    int op;          /* mxfft_op */
    int slices;
    const void *in;
    void *out;
    int coils;       /* with rss: coil images per RSS image (slices a multiple of it) */
    int reserved;    /* 0 */
    void *rss;       /* optional device float [slices / coils][n0][n1], 16-byte aligned:
                        mxfft_rss of out after the transform; NULL: none */
} mxfft_item;

typedef struct mxfft_engine_s *mxfft_engine_t;

/* Engine flags. */
#define MXFFT_ENGINE_GRAPHS 1  /* capture each batch signature into a CUDA graph, replay it */
#define MXFFT_ENGINE_TC16 2    /* tensor-core radix-16 passes where a plan supports them */
#define MXFFT_ENGINE_FUSED2D 4 /* with MXFFT_ENGINE_TC16: MXFFT_OPT_FUSED2D on the engine's plans */
#define MXFFT_ENGINE_FOLD_STATS 16 /* with MXFFT_ENGINE_TC16: MXFFT_OPT_FOLD_STATS on the
                                      engine's plans */
#define MXFFT_ENGINE_NO_RAGGED 8 /* one launch per pass and plan group instead of the ragged
                                    launches (same results; for comparison) */

/*
 * mxfft_engine_create -- executor bound to the current device, with its own
 *   plan cache (plans and twiddle tables stay resident), fork streams, and
 *   for MXFFT_ENGINE_GRAPHS a cache of instantiated graphs keyed by the batch
 *   signature (the items' shapes, formats, ops and slice counts).  A graph
 *   reads every buffer address from a table in device memory that is
 *   refreshed before each replay, so one signature is captured once whatever
 *   buffers later calls pass.
 * mxfft_engine_run -- enqueue the items on the stream (asynchronous).
 *   Errors: MXFFT_ERR_INVALID for a bad item (the checks of mxfft_plan and of
 *   the data pointers), MXFFT_ERR_NOMEM, MXFFT_ERR_CUDA.  Before rewriting a
 *   table that an earlier run may still be reading, the call waits for that
 *   run.  Not safe for concurrent calls on one engine.
 * mxfft_engine_get_status -- after the stream has been synchronised: flags
 *   of the last run (bit 0 a non-finite input magnitude, bit 1 a bounded wait
 *   timed out) and, if k_out is not NULL, 2 int32 per slice in item order
 *   (prescale exponent of the transform; of the inverse for round trips, else
 *   0), at most k_out_len values written.
 */
int mxfft_engine_create(float tau, float target, int flags, mxfft_engine_t *out);
int mxfft_engine_run(mxfft_engine_t e, const mxfft_item *items, int n_items, void *stream);
int mxfft_engine_get_status(mxfft_engine_t e, int *device_flags, int32_t *k_out, int k_out_len);
/* mxfft_engine_launches -- number of kernels the last mxfft_engine_run
 *   enqueued (for a graph replay: the kernels of the captured graph); 0
 *   before the first run.  MXFFT_ERR_INVALID for NULL arguments. */
int mxfft_engine_launches(mxfft_engine_t e, int *launches);
/* mxfft_engine_destroy -- waits for the engine's last run, then frees its
 *   graphs, plans, events, streams and buffers.  Unlike mxfft_destroy, NULL
 *   returns MXFFT_ERR_INVALID. */
int mxfft_engine_destroy(mxfft_engine_t e);

/* ======================================================================
 * Launch-geometry autotuner.  Measures, for a plan's passes at a given
 * batch, the CTA shapes of the radix-2 pass kernel (transform groups per CTA)
 * or, on the tensor-core path (MXFFT_OPT_PATH = 1), the tile and the
 * resident CTAs per SM of its persistent grid (4096-point tiles on 256
 * threads, 1 or 2 per SM; for n <= 1024 also 2048-point tiles on 128
 * threads, 2 to 6 per SM), and keeps the fastest in a process-wide table
 * that later launches of the same (length, other extent, axis, format, block
 * size, batch class) use.  Every shape computes the same bits.  The table can
 * be saved to and loaded from a JSON file (tensor-core entries carry
 * "kind": 1, "tile" and "ctas_per_sm").
 *
 * mxfft_tune -- synchronous; allocates a scratch batch on the device,
 *   times each candidate with CUDA events on the stream, frees the scratch.
 *   n_measured (nullable) receives the number of candidates timed.
 * mxfft_tune_save / mxfft_tune_load -- write / merge the table (JSON, UTF-8).
 *   MXFFT_ERR_INVALID for an unreadable or malformed file.
 * mxfft_tune_clear -- forget every entry.
 * ====================================================================== */
int mxfft_tune(mxfft_plan_t p, int batch, void *stream, int *n_measured);
int mxfft_tune_save(const char *path);
int mxfft_tune_load(const char *path);
int mxfft_tune_clear(void);

/* ======================================================================
 * Request server with continuous batching.  Not a construct of the paper.
 * Requests (host buffers) are queued; a worker thread admits them in arrival
 * order into batches as execution slots (streams) and device memory free
 * up, copies each batch in, runs it through an engine and copies it out,
 * while earlier batches still run on other slots, so work of requests that
 * arrive while others are on the GPU overlaps on the device.  Each result
 * is bit-identical to the same request run alone.
 * ====================================================================== */
typedef struct {
    int n0, n1, format, k, op, slices;   /* as in mxfft_item */
    const void *host_in;                 /* [slices][n0][n1] complex64; pinned for overlap */
    void *host_out;                      /* same size, written when the request completes;
                                            may be NULL when host_rss is given */
    uint64_t tag;                        /* returned in the completion */
    int coils;                           /* with host_rss: coil images per RSS image */
    int reserved;                        /* 0 */
    void *host_rss;                      /* optional float [slices / coils][n0][n1]: the
                                            RSS images of the result (Eq. (1)); NULL: none */
} mxfft_request;

typedef struct {
    uint64_t tag;
    int status;                          /* mxfft_status of the request */
    int device_flags;                    /* bit 0: a non-finite input magnitude */
    double t_submit_us, t_admit_us, t_done_us;   /* server clock */
} mxfft_completion;

typedef struct {
    int slots;                 /* batches in flight (streams), >= 1 */
    int max_batch_slices;      /* slices per batch, >= 1 */
    uint64_t mem_budget;       /* device bytes for request data; 0: 80% of free memory */
    float tau, target;         /* of every plan */
    int engine_flags;          /* MXFFT_ENGINE_* */
    uint64_t max_batch_bytes;  /* request bytes per batch (a larger request forms a batch
                                  alone); 0: no limit */
} mxfft_server_config;

typedef struct mxfft_server_s *mxfft_server_t;

/*
 * mxfft_server_create -- start the worker thread on the current device.
 * mxfft_server_submit -- queue a request (copied; the host buffers must stay
 *   valid until its completion is polled).  MXFFT_ERR_INVALID for a bad
 *   request; a request larger than the whole memory budget completes with
 *   MXFFT_ERR_NOMEM.
 * mxfft_server_poll -- move up to max finished completions to out; *n_out
 *   receives their number.  A request completes when its own result is in
 *   host memory (each request's copy-out ends with its own host callback).
 * mxfft_server_wait -- block until every submitted request has completed or
 *   timeout_s has passed (MXFFT_ERR_TIMEOUT).
 * mxfft_server_stats -- counters: batches launched, peak device bytes held by
 *   admitted requests (never above the budget), the budget.
 * mxfft_server_destroy -- finish outstanding work, stop the thread, free
 *   (NULL returns MXFFT_ERR_INVALID).
 */
int mxfft_server_create(const mxfft_server_config *cfg, mxfft_server_t *out);
int mxfft_server_submit(mxfft_server_t s, const mxfft_request *r);
int mxfft_server_poll(mxfft_server_t s, mxfft_completion *out, int max, int *n_out);
int mxfft_server_wait(mxfft_server_t s, double timeout_s);
int mxfft_server_stats(mxfft_server_t s, uint64_t *batches, uint64_t *peak_bytes, uint64_t *budget);
int mxfft_server_destroy(mxfft_server_t s);

/*
 * mxfft_rss -- root-sum-of-squares coil combine of Eq. (1) (Sec. 2.3):
 *   out[i][p] = (sum over c of |z[i * coils + c][p]|^2)^(1/2), the coils of
 *   image i being consecutive [n0][n1] complex64 slices of z; out is float
 *   [images][n0][n1].  FP32, coils added in order c = 0, 1, ..., then one
 *   correctly rounded square root.  z, out: device, 16-byte aligned, not
 *   overlapping; n0 * n1 even.  Asynchronous on the stream; MXFFT_ERR_INVALID
 *   for bad arguments.
 */
int mxfft_rss(const void *z, void *out, int images, int coils, int n0, int n1, void *stream);

/*
 * mxfft_quantize -- the element rounding Q of Alg. 2 (Sec. 2.2: the
 * quantisation inside EncodeBlockMX / EncodeFromMantBlock, applied to values
 * already divided by their block's power-of-two scale): round to the nearest
 * value of the element format, ties to the even code, saturating at the
 * largest normal, signed zeros and subnormals kept; run on the device with
 * the transforms' own code, for comparison with an independent
 * implementation.
 *   in, out  device arrays of n float32 values (out may equal in).
 *   format   MXFFT_E4M3 .. MXFFT_E2M1.
 *   path     0: the register-resident pass's conversions (the hardware
 *            cvt.rn.satfinite.<fmt>x2.f32 and back to exact f16 values;
 *            n even, 8-byte aligned arrays); 1: the generic pass's FP32
 *            add-and-subtract rounding (4-byte aligned arrays).
 * Asynchronous on stream; MXFFT_ERR_INVALID for bad arguments.  Finite
 * inputs only (the transforms handle Inf / NaN by the block scale).
 */
int mxfft_quantize(const void *in, void *out, long long n, int format, int path, void *stream);

/*
 * mxfft_test_fail_alloc -- test hook of the plan allocator (no counterpart in
 * the paper).  after >= 0: the device allocation of a plan (tables, statistics
 * records; mxfft_plan, mxfft_set_option, the statistics growth of a
 * transform call) that comes after `after` further successful ones fails as
 * if the device were out of memory, once; the call that made it returns
 * MXFFT_ERR_NOMEM and frees what it had allocated.  after = -1 disarms it.
 * Process-wide, not thread-safe; for tests of the failure paths only.
 */
int mxfft_test_fail_alloc(int after);

/*
 * mxfft_debug_bounds -- bounds-check build (no counterpart in the paper).  A
 * library built with MXFFT_DEBUG_BOUNDS defined checks the computed global
 * and shared-memory indices of its transform kernels (register-resident,
 * generic, tensor-core and fused 2D passes); an index outside its buffer is
 * counted and replaced by a valid one instead of being used.  This call
 * synchronises the device and returns *enabled = 1 and the number of
 * violations since the previous call (then clears the count); in the normal
 * build *enabled = 0 and *violations = 0.  MXFFT_ERR_INVALID for NULL
 * arguments.
 */
int mxfft_debug_bounds(int *enabled, unsigned long long *violations);

/* mxfft_status_string -- static description of a status code. */
const char *mxfft_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MXFFT_H */
