// Host side of libmxfft: plans, prequantised twiddle tables, the launch
// sequence of each transform and the C ABI declared in include/mxfft.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <nvtx3/nvToolsExt.h>

#include "mx_plan.h"

using namespace mxfft;

namespace {

// NVTX range around one enqueued call (shown by profilers on the host timeline).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Device allocations of a plan (its tables and statistics records) go
// through plan_malloc, so that a test can make the n-th one fail as if the
// device were out of memory (mxfft_test_fail_alloc).
std::atomic<int> g_fail_alloc_after{-1};

cudaError_t plan_malloc(void** p, size_t bytes) {
    const int c = g_fail_alloc_after.load();
    if (c == 0) {
        g_fail_alloc_after.store(-1);
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (c > 0) g_fail_alloc_after.store(c - 1);
    return cudaMalloc(p, bytes);
}

struct FmtHost {
    int emax, emin, mbits;
    double maxnorm;
};

// OCP element formats: unbiased exponents of the largest and smallest normal,
// mantissa bits and largest finite magnitude.
bool fmt_host(int code, FmtHost* f) {
    switch (code) {
        case MXFFT_E4M3: *f = {8, -6, 3, 448.0}; return true;
        case MXFFT_E5M2: *f = {15, -14, 2, 57344.0}; return true;
        case MXFFT_E2M3: *f = {2, 0, 3, 7.5}; return true;
        case MXFFT_E3M2: *f = {4, -2, 2, 28.0}; return true;
        case MXFFT_E2M1: *f = {2, 0, 1, 6.0}; return true;
        case MXFFT_FP16: *f = {15, -14, 10, 65504.0}; return true;   // IEEE binary16
        case MXFFT_FP32_REF: *f = {127, -126, 23, 3.4028234663852886e38}; return true;   // binary32
        default: return false;
    }
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) l++; return l; }

// Exponent e if v == 2^e exactly (v > 0), else a sentinel.
bool exact_pow2_exp(double v, int* e) {
    if (!(v > 0.0) || !std::isfinite(v)) return false;
    int ex;
    double fr = std::frexp(v, &ex);
    if (fr != 0.5) return false;
    *e = ex - 1;
    return true;
}

// Element rounding of an FP64 value already divided by its block scale:
// nearest grid value (ties to even), saturating, via the 2^52 add-and-subtract
// identity: |x| + 1.5 * 2^52 * q lands in a binade whose ulp is the grid
// spacing q, so the adder rounds half-even onto the grid.
double q_host(double x, const FmtHost& f) {
    if (x == 0.0) return x;
    double a = std::fabs(x);
    if (a > f.maxnorm) a = f.maxnorm;
    int ex;
    std::frexp(a, &ex);
    int E = ex - 1;
    if (E < f.emin) E = f.emin;
    const double c = std::ldexp(1.5, 52 + E - f.mbits);
    volatile double t = a + c;
    double r = t - c;
    return std::copysign(r, x);
}

// cos and sin of 2 pi j / N for 0 <= j < N/2, reduced to the first octant so
// that 0, +-1 and +-sqrt(1/2) come out exactly symmetric.
void unit_root(long j, long N, double* c, double* s) {
    const double two_pi = 6.283185307179586476925286766559;
    long j8 = 8 * j;
    if (j8 <= N) {                       // [0, pi/4]
        double a = two_pi * (double)j / (double)N;
        *c = std::cos(a); *s = std::sin(a);
        if (j8 == N) { *c = *s = std::sqrt(0.5); }
    } else if (j8 <= 2 * N) {            // (pi/4, pi/2]: angle pi/2 - a
        double a = two_pi * (double)(N / 4 - j) / (double)N;
        if (4 * j == N) { *c = 0.0; *s = 1.0; }
        else { *c = std::sin(a); *s = std::cos(a); }
    } else if (j8 <= 3 * N) {            // (pi/2, 3pi/4]: angle pi/2 + a
        double a = two_pi * (double)(j - N / 4) / (double)N;
        *c = -std::sin(a); *s = std::cos(a);
        if (j8 == 3 * N) { *c = -std::sqrt(0.5); *s = std::sqrt(0.5); }
    } else {                             // (3pi/4, pi): angle pi - a
        double a = two_pi * (double)(N / 2 - j) / (double)N;
        *c = -std::cos(a); *s = std::sin(a);
    }
}

// Prequantised twiddles of one axis of length n with MX blocks of m butterflies:
// stage h (h = 1, 2, ..., n/2) holds w_j = exp(-2 pi i j / (2h)), j < h, at
// index (h - 1) + j.  The MX blocks of a stage are the runs of m consecutive
// butterflies b = g*h + j; for h >= m a block covers j in [j0, j0 + m), for
// h < m it covers every j of the stage.  Each block gets its shared exponent
// s_w = floor(log2 max|w component|) - emax and element values Q(w 2^-s_w).
void build_twiddles(int n, int m, const FmtHost& f, std::vector<float2>& fwd,
                    std::vector<float2>& inv, std::vector<int8_t>& sw, bool plain) {
    fwd.assign(n, make_float2(0.f, 0.f));
    inv.assign(n, make_float2(0.f, 0.f));
    sw.assign(n, 0);
    for (int h = 1; h < n; h <<= 1) {
        const int bl = h >= m ? m : h;   // j-run per block
        for (int j0 = 0; j0 < h; j0 += bl) {
            std::vector<double> cs(bl), sn(bl);
            double amax = 0.0;
            for (int jj = 0; jj < bl; jj++) {
                unit_root(j0 + jj, 2L * h, &cs[jj], &sn[jj]);
                amax = std::fmax(amax, std::fmax(std::fabs(cs[jj]), std::fabs(sn[jj])));
            }
            int ex;
            std::frexp(amax, &ex);
            int s = (ex - 1) - f.emax;
            if (s < -127) s = -127;
            if (s > 127) s = 127;
            if (plain) s = 0;   // FP16 control / FP32 ablation: plain values, no block scale
            for (int jj = 0; jj < bl; jj++) {
                const double xr = q_host(std::ldexp(cs[jj], -s), f);
                const double xi = q_host(std::ldexp(-sn[jj], -s), f);
                const int idx = (h - 1) + j0 + jj;
                fwd[idx] = make_float2((float)xr, (float)xi);
                inv[idx] = make_float2((float)xr, (float)-xi);
                sw[idx] = (int8_t)s;
            }
        }
    }
}

// cos and sin of 2 pi j / N for any 0 <= j < N.
void unit_root_full(long j, long N, double* c, double* s) {
    if (2 * j < N) { unit_root(j, N, c, s); return; }
    unit_root(j - N / 2, N, c, s);
    *c = -*c;
    *s = -*s;
}

// MX block of 16 twiddles exp(sgn i 2 pi (m idx) / N), idx = 0..15: shared
// exponent from the block maximum, element values back-scaled (exact).
void twiddle_block16(long m, long N, int sgn, const FmtHost& f, float2* out) {
    double c[16], sn[16], amax = 0.0;
    for (int i = 0; i < 16; i++) {
        unit_root_full((m * i) % N, N, &c[i], &sn[i]);
        sn[i] *= sgn;
        amax = std::fmax(amax, std::fmax(std::fabs(c[i]), std::fabs(sn[i])));
    }
    int ex;
    std::frexp(amax, &ex);
    const int sc = (ex - 1) - f.emax;
    for (int i = 0; i < 16; i++)
        out[i] = make_float2((float)std::ldexp(q_host(std::ldexp(c[i], -sc), f), sc),
                             (float)std::ldexp(q_host(std::ldexp(sn[i], -sc), f), sc));
}

void free_plan_device(mxfft_plan_s* p) {
    for (int d = 0; d < 2; d++) {
        if (p->d_bmat[d]) cudaFree(p->d_bmat[d]);
        if (p->d_bmat8[d]) cudaFree(p->d_bmat8[d]);
        for (int a = 0; a < 2; a++) {
            if (p->d_twA[a][d]) cudaFree(p->d_twA[a][d]);
            if (p->d_twC[a][d]) cudaFree(p->d_twC[a][d]);
            if (p->d_tw4A[a][d]) cudaFree(p->d_tw4A[a][d]);
            if (p->d_tw4C[a][d]) cudaFree(p->d_tw4C[a][d]);
        }
    }
    if (p->d_err) cudaFree(p->d_err);
    for (int a = 0; a < 2; a++) {
        for (int d = 0; d < 2; d++) {
            if (p->d_tw[a][d]) cudaFree(p->d_tw[a][d]);
            if (p->d_twh[a][d]) cudaFree(p->d_twh[a][d]);
        }
        if (p->d_tws[a]) cudaFree(p->d_tws[a]);
    }
    if (p->d_st) cudaFree(p->d_st);
}

int ensure_stats(mxfft_plan_s* p, int batch) {
    if (batch <= p->st_cap) return MXFFT_OK;
    int cap = p->st_cap ? p->st_cap : 1;
    while (cap < batch) cap *= 2;
    if (p->d_st) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(p->d_st);
        p->d_st = nullptr;
        p->st_cap = 0;
    }
    cudaError_t e = plan_malloc((void**)&p->d_st, sizeof(SliceStats) * 2 * (size_t)cap);
    if (e != cudaSuccess) { p->d_st = nullptr; return cuda_status(e); }
    p->st_cap = cap;
    return MXFFT_OK;
}

// Real 32 x 32 matrix of the P-point DFT (sign sgn) for interleaved re/im
// vectors, each output row an MX block: element codes in the K-major
// core-matrix layout of the tensor-core B operand, and the row scales.  P =
// 16: one 16-point DFT; P = 8: the 8-point DFT twice on the diagonal (rows
// and columns 16 b .. 16 b + 15 for the b-th of two 8-point vectors).
void build_dft_matrix(int P, int sgn, int fmt, const FmtHost& f, std::vector<uint8_t>& codes,
                      std::vector<float>& scales) {
    codes.assign(1024, 0);
    scales.assign(32, 0.f);
    for (int m = 0; m < 16; m++) {
        double row[2][32] = {};
        const int b = m / P, mm = m % P;            // diagonal block, output index in it
        for (int j = 0; j < P; j++) {
            double c, s;
            unit_root_full((long)(j * mm) % P, P, &c, &s);
            s *= sgn;                                  // W = c + i s
            const int col = 2 * (b * P + j);
            row[0][col] = c;  row[0][col + 1] = -s;    // Re y: a c - b s
            row[1][col] = s;  row[1][col + 1] = c;     // Im y: a s + b c
        }
        for (int part = 0; part < 2; part++) {
            const int nrow = 2 * m + part;
            double amax = 0.0;
            for (int k = 0; k < 32; k++) amax = std::fmax(amax, std::fabs(row[part][k]));
            int ex;
            std::frexp(amax, &ex);
            const int sc = (ex - 1) - f.emax;
            scales[nrow] = (float)std::ldexp(1.0, sc);
            for (int k = 0; k < 32; k++) {
                const float q = (float)q_host(std::ldexp(row[part][k], -sc), f);
                uint8_t code;
                if (fmt == MXFFT_E4M3) { __nv_fp8_e4m3 v(q); std::memcpy(&code, &v, 1); }
                else { __nv_fp8_e5m2 v(q); std::memcpy(&code, &v, 1); }
                codes[(nrow >> 3) * 256 + (k >> 4) * 128 + (nrow & 7) * 16 + (k & 15)] = code;
            }
        }
    }
}

template <class T>
int upload(T** dst, const std::vector<T>& v) {
    int rc = cuda_status(plan_malloc((void**)dst, sizeof(T) * v.size()));
    if (rc == MXFFT_OK)
        rc = cuda_status(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return rc;
}

// Tables of the tensor-core path (built when the path is selected).
int build_tc16_tables(mxfft_plan_s* p) {
    FmtHost f;
    fmt_host(p->fmt, &f);
    int rc = MXFFT_OK;
    for (int d = 0; d < 2 && rc == MXFFT_OK; d++) {
        if (p->d_bmat[d]) continue;
        const int sgn = d == 0 ? -1 : 1;
        std::vector<uint8_t> codes, codes8;
        std::vector<float> scales, scales8;
        build_dft_matrix(16, sgn, p->fmt, f, codes, scales);
        build_dft_matrix(8, sgn, p->fmt, f, codes8, scales8);
        // the kernel folds the row scales into one constant: every row of the
        // matrix holds an entry of magnitude 1, so each row scale is 2^-emax
        for (float sc : scales)
            if (sc != (float)std::ldexp(1.0, -f.emax)) return MXFFT_ERR_UNSUPPORTED;
        for (float sc : scales8)
            if (sc != (float)std::ldexp(1.0, -f.emax)) return MXFFT_ERR_UNSUPPORTED;
        rc = upload(&p->d_bmat[d], codes);
        // n = 128 axes: the second round's pairs of 8-point DFTs
        if (rc == MXFFT_OK && (p->n0 == 128 || p->n1 == 128)) rc = upload(&p->d_bmat8[d], codes8);
        for (int axis = 0; axis < 2 && rc == MXFFT_OK; axis++) {
            const int n = axis == 0 ? p->n0 : p->n1;
            const int r = std::max(n / 256, 1), M = n / 16;
            std::vector<float2> twa((size_t)M * 16), twc((size_t)std::max(r, 1) * 16);
            for (int j2 = 0; j2 < M; j2++) twiddle_block16(j2, n, sgn, f, &twa[(size_t)j2 * 16]);
            for (int j22 = 0; n >= 512 && j22 < r; j22++) twiddle_block16(j22, M, sgn, f, &twc[(size_t)j22 * 16]);
            rc = upload(&p->d_twA[axis][d], twa);
            if (rc == MXFFT_OK) rc = upload(&p->d_twC[axis][d], twc);
            // the same twiddles as (re, re, -im, im) for packed multiplies
            std::vector<float4> t4a(twa.size()), t4c(twc.size());
            for (size_t i = 0; i < twa.size(); i++) t4a[i] = make_float4(twa[i].x, twa[i].x, -twa[i].y, twa[i].y);
            for (size_t i = 0; i < twc.size(); i++) t4c[i] = make_float4(twc[i].x, twc[i].x, -twc[i].y, twc[i].y);
            if (rc == MXFFT_OK) rc = upload(&p->d_tw4A[axis][d], t4a);
            if (rc == MXFFT_OK) rc = upload(&p->d_tw4C[axis][d], t4c);
        }
    }
    if (rc == MXFFT_OK && !p->d_err) {
        rc = cuda_status(plan_malloc((void**)&p->d_err, sizeof(int)));
        if (rc == MXFFT_OK) rc = cuda_status(cudaMemset(p->d_err, 0, sizeof(int)));
    }
    return rc;
}

bool aligned16(const void* q) { return ((uintptr_t)q & 15u) == 0; }

// Event pair around one launch when profiling is on (nullptr otherwise).
ProfRec* prof_begin(mxfft_plan_s* p, int kind, cudaStream_t s) {
    if (!p->prof) return nullptr;
    ProfRec rec{kind, nullptr, nullptr};
    if (cudaEventCreate(&rec.a) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&rec.b) != cudaSuccess) { cudaEventDestroy(rec.a); return nullptr; }
    cudaEventRecord(rec.a, s);
    p->recs->push_back(rec);
    return &p->recs->back();
}

void prof_end(ProfRec* r, cudaStream_t s) {
    if (r) cudaEventRecord(r->b, s);
}

void prof_clear(mxfft_plan_s* p) {
    if (!p->recs) return;
    for (ProfRec& r : *p->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    p->recs->clear();
}

// op: 0 forward, 1 inverse, 2 round trip, 3 fused round trip
int run(mxfft_plan_t p, const void* in, void* out, int batch, void* stream, int op) {
    static const char* const kNames[4] = {"mxfft_forward", "mxfft_inverse", "mxfft_roundtrip",
                                          "mxfft_roundtrip_fused"};
    NvtxRange range(kNames[op & 3]);
    if (!p || batch < 0) return MXFFT_ERR_INVALID;
    if (op == 3 && p->fmt == MXFFT_FP16) return MXFFT_ERR_UNSUPPORTED;
    if (batch == 0) return MXFFT_OK;
    if (!in || !out || !aligned16(in) || !aligned16(out)) return MXFFT_ERR_INVALID;
    const size_t bytes = (size_t)batch * p->n0 * p->n1 * sizeof(float2);
    const char* ci = (const char*)in;
    const char* co = (const char*)out;
    if (ci != co && ci < co + bytes && co < ci + bytes) return MXFFT_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return MXFFT_ERR_CUDA;
    int rc = ensure_stats(p, batch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    SliceStats* st_f = p->d_st;
    SliceStats* st_i = p->d_st + p->st_cap;
    cudaError_t e = cudaMemsetAsync(st_f, 0, sizeof(SliceStats) * (size_t)batch, s);
    if (e == cudaSuccess && op == 2) e = cudaMemsetAsync(st_i, 0, sizeof(SliceStats) * (size_t)batch, s);
    // the timeout flag reports this call only
    if (e == cudaSuccess && p->d_err) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_status(e);
    const float2* x = (const float2*)in;
    float2* y = (float2*)out;
    const int dir0 = op == 1 ? 1 : 0;
    if (op != 3 && uses_tc2d(p)) {
        // the fused 2D tensor-core transform: statistics, rows and columns of
        // each slice in one launch (the round trip: forward, then inverse)
        e = timed_tc2d(p, tc2d_args(p, dir0, x, y, st_f, EPI_UNSCALE), batch, s);
        if (e == cudaSuccess && op == 2)
            e = timed_tc2d(p, tc2d_args(p, 1, y, y, st_i, EPI_RT_FINAL), batch, s);
        if (e != cudaErrorNotSupported) {
            if (e != cudaSuccess) return cuda_status(e);
            p->last_batch = batch;
            p->last_op = op;
            p->last_stream = s;
            return MXFFT_OK;
        }
        // the device cannot hold the kernel's cluster: the per-axis passes
        // (nothing was launched)
    }
    {
        NvtxRange sr("mxfft statistics");
        ProfRec* r = prof_begin(p, 0, s);
        e = launch_stats(x, batch, p->n0, p->n1, st_f, kparams(p), s);
        prof_end(r, s);
    }
    if (e != cudaSuccess) return cuda_status(e);
    PassArgs rows = pass_args(p, 1, dir0, x, y);
    rows.st = st_f;
    rows.prologue = PRO_PRESCALE;
    rows.epilogue = EPI_RAW;
    if ((e = timed_pass(p, rows, batch, s)) != cudaSuccess) return cuda_status(e);
    PassArgs cols = pass_args(p, 0, dir0, y, y);
    cols.st = st_f;
    cols.prologue = PRO_NONE;
    cols.epilogue = op == 3 ? EPI_RAW : EPI_UNSCALE;
    if (op == 3) {
        // fused round trip (reading C17): forward and inverse columns on the
        // undecoded forward result, then the inverse rows with the one decode
        if ((e = fused_cols_pass(p, cols, batch, s)) != cudaSuccess) return cuda_status(e);
        PassArgs r2 = pass_args(p, 1, 1, y, y);
        r2.st = st_f;
        r2.prologue = PRO_NONE;
        r2.epilogue = EPI_RT_FINAL;
        if ((e = timed_pass(p, r2, batch, s)) != cudaSuccess) return cuda_status(e);
    } else {
        // the round trip on the tensor-core path: the forward columns pass
        // takes the inverse's prescale statistics of what it stores
        if (op == 2 && tc16_folds_stats(p)) {
            cols.st_out = st_i;
            cols.stats_out = 1;
        }
        if ((e = timed_pass(p, cols, batch, s)) != cudaSuccess) return cuda_status(e);
    }
    if (op == 2 && !cols.stats_out) {
        // the inverse's own prescale statistics, on the forward output y
        {
            NvtxRange sr("mxfft statistics");
            ProfRec* rs = prof_begin(p, 0, s);
            e = launch_stats(y, batch, p->n0, p->n1, st_i, kparams(p), s);
            prof_end(rs, s);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (op == 2) {
        PassArgs r2 = pass_args(p, 1, 1, y, y);
        r2.st = st_i;
        r2.prologue = PRO_PRESCALE;
        r2.epilogue = EPI_RAW;
        if ((e = timed_pass(p, r2, batch, s)) != cudaSuccess) return cuda_status(e);
        PassArgs c2 = pass_args(p, 0, 1, y, y);
        c2.st = st_i;
        c2.prologue = PRO_NONE;
        c2.epilogue = EPI_RT_FINAL;
        if ((e = timed_pass(p, c2, batch, s)) != cudaSuccess) return cuda_status(e);
    }
    p->last_batch = batch;
    p->last_op = op;
    p->last_stream = s;
    return MXFFT_OK;
}

}  // namespace

namespace mxfft {

std::atomic<long long> g_kernel_launches{0};

bool fmt_params(int code, FmtParams* fp) {
    FmtHost f;
    if (!fmt_host(code, &f)) return false;
    fp->emax = f.emax;
    fp->emin = f.emin;
    fp->mbits = f.mbits;
    fp->maxnorm = (float)f.maxnorm;
    fp->qmin_bits = (uint32_t)(f.emin + 127) << 23;
    fp->qadd_bits = ((uint32_t)(23 - f.mbits) << 23) | 0x400000u;
    return true;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MXFFT_OK;
    if (e == cudaErrorMemoryAllocation) return MXFFT_ERR_NOMEM;
    return MXFFT_ERR_CUDA;
}

KParams kparams(const mxfft_plan_s* p) {
    KParams kp;
    kp.tau = p->tau;
    kp.t_exp = p->t_exp;
    kp.taumin_exp = p->taumin_exp;
    kp.kmin = p->kmin;
    kp.kmax = p->kmax;
    return kp;
}

PassArgs pass_args(const mxfft_plan_s* p, int dim, int dir, const float2* in, float2* out) {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.n0 = p->n0;
    a.n1 = p->n1;
    a.dim = dim;
    a.n = dim == 1 ? p->n1 : p->n0;
    a.logn = ilog2(a.n);
    const int other = dim == 1 ? p->n0 : p->n1;
    int tpc = 8192 / a.n;
    if (tpc < 1) tpc = 1;
    if (tpc > other) tpc = other;
    a.tpc = tpc;
    a.m = p->m[dim];
    a.tw = p->d_tw[dim][dir];
    a.tws = p->d_tws[dim];
    a.fmt = p->fmt;
    a.fp = p->fp;
    a.kp = kparams(p);
    a.lg_total = ilog2(p->n0) + ilog2(p->n1);
    return a;
}

bool tc16_folds_stats(const mxfft_plan_s* p) {
    // the tensor-core columns pass keeps each slice's tiles on consecutive
    // tiles of a CTA except at n0 = 2048 (tiles of two columns, strided)
    return p->path == 1 && p->fold_stats && p->n0 != 2048;
}

bool uses_tc2d(const mxfft_plan_s* p) {
    return p->path == 1 && p->fused2d && tc2d_supported(p->n0, p->n1, p->fmt, p->kblk) &&
           tc2d_resident_clusters(p->n0, p->n1, p->fmt) > 0;
}

Tc2dArgs tc2d_args(const mxfft_plan_s* p, int dir, const float2* in, float2* out, SliceStats* st,
                   int epilogue) {
    Tc2dArgs t;
    std::memset(&t, 0, sizeof(t));
    t.in = in;
    t.out = out;
    t.st = st;
    t.n0 = p->n0;
    t.n1 = p->n1;
    t.bmat = p->d_bmat[dir];
    t.twA1 = p->d_tw4A[1][dir];
    t.twC1 = p->d_tw4C[1][dir];
    t.twA0 = p->d_tw4A[0][dir];
    t.twC0 = p->d_tw4C[0][dir];
    t.epilogue = epilogue;
    t.lg_total = ilog2(p->n0) + ilog2(p->n1);
    const uint32_t ft = p->fmt == MXFFT_E5M2 ? 1u : 0u;
    t.idesc = (1u << 4) | (ft << 7) | (ft << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    t.err = p->d_err;
    t.stall = p->test_stall;
    t.kp = kparams(p);
    return t;
}

cudaError_t timed_tc2d(mxfft_plan_s* p, const Tc2dArgs& a, int batch, cudaStream_t s) {
    NvtxRange range("mxfft fused 2D transform");
    Tc2dArgs b = a;
    b.batch = batch;
    ProfRec* r = prof_begin(p, 4, s);
    cudaError_t e = launch_tc2d(b, p->fmt, s);
    prof_end(r, s);
    return e;
}

Tc16Args tc16_args(const mxfft_plan_s* p, const PassArgs& a, int dir) {
    Tc16Args t;
    std::memset(&t, 0, sizeof(t));
    t.in = a.in;
    t.out = a.out;
    t.ref = a.ref;
    t.n0 = a.n0;
    t.n1 = a.n1;
    t.dim = a.dim;
    t.n = a.n;
    t.r = a.n / 256;
    t.bmat = p->d_bmat[dir];
    t.bmat2 = p->d_bmat8[dir];
    t.twA = p->d_twA[a.dim][dir];
    t.twC = p->d_twC[a.dim][dir];
    t.st = a.st;
    t.prologue = a.prologue;
    t.epilogue = a.epilogue;
    t.lg_total = a.lg_total;
    const uint32_t ft = p->fmt == MXFFT_E5M2 ? 1u : 0u;
    t.idesc = (1u << 4) | (ft << 7) | (ft << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    t.err = p->d_err;
    t.stall = p->test_stall;
    t.g = p->kblk / 32;
    t.inv = dir;
    t.st_out = a.st_out;
    t.stats_out = a.stats_out;
    t.kp = a.kp;
    return t;
}

// The tensor-core pass when that path is selected, else the register-resident
// kernel where it applies (n in [64, 2048], m <= 16; m = 32, 64 for n >= 128),
// else the generic shared-memory kernel.
cudaError_t timed_pass(mxfft_plan_s* p, const PassArgs& a, int batch, cudaStream_t s) {
    NvtxRange range(a.dim == 1 ? "mxfft rows pass" : "mxfft columns pass");
    const int dir = a.tw == p->d_tw[a.dim][1] ? 1 : 0;
    if (p->path == 1) {
        const Tc16Args t = tc16_args(p, a, dir);
        ProfRec* r = prof_begin(p, 3, s);
        cudaError_t e = launch_tc16_pass(t, p->fmt, batch, s);
        prof_end(r, s);
        return e;
    }
    const bool fast = !p->force_generic && fast_pass_supported(a);
    ProfRec* r = prof_begin(p, fast ? 2 : 1, s);
    cudaError_t e = fast ? launch_fast_pass(a, p->d_twh[a.dim][dir], p->twa[a.dim][dir], batch, s)
                         : launch_pass(a, batch, s);
    prof_end(r, s);
    return e;
}

// Forward then inverse column transforms of the fused round trip on the same
// slices (a: columns, forward twiddles, no prologue, raw epilogue): one
// register-resident launch that keeps each tile on chip between the two where
// that kernel applies, else the two passes one after the other (same results).
cudaError_t fused_cols_pass(mxfft_plan_s* p, const PassArgs& a, int batch, cudaStream_t s) {
    if (p->path != 1 && !p->force_generic && fast_pass_supported(a)) {
        ProfRec* r = prof_begin(p, 2, s);
        cudaError_t e = launch_fast_pass_fused(a, p->d_twh[0][0], p->twa[0][0], p->d_twh[0][1],
                                               p->twa[0][1], batch, s);
        prof_end(r, s);
        return e;
    }
    cudaError_t e = timed_pass(p, a, batch, s);
    if (e != cudaSuccess) return e;
    PassArgs b = a;
    b.tw = p->d_tw[0][1];
    return timed_pass(p, b, batch, s);
}

}  // namespace mxfft

extern "C" {

int mxfft_plan(int n0, int n1, int format, int k, float tau, float target, mxfft_plan_t* out) {
    if (!out) return MXFFT_ERR_INVALID;
    *out = nullptr;
    FmtHost f;
    if (!is_pow2(n0) || !is_pow2(n1) || n0 < 2 || n1 < 2 || n0 > 2048 || n1 > 2048)
        return MXFFT_ERR_INVALID;
    if (!fmt_host(format, &f)) return MXFFT_ERR_INVALID;
    if (!is_pow2(k) || k < 2 || k > 128) return MXFFT_ERR_INVALID;
    if (!(tau > 0.0f && tau < 1.0f)) return MXFFT_ERR_INVALID;
    if (!(target > 0.0f) || !std::isfinite(target)) return MXFFT_ERR_INVALID;
    int t_exp;
    if (!exact_pow2_exp((double)target, &t_exp)) return MXFFT_ERR_UNSUPPORTED;

    mxfft_plan_s* p = new (std::nothrow) mxfft_plan_s;
    if (!p) return MXFFT_ERR_NOMEM;
    std::memset(p, 0, sizeof(*p));
    p->n0 = n0;
    p->n1 = n1;
    p->fmt = format;
    p->kblk = k;
    p->tau = tau;
    p->t_exp = t_exp;
    // tail floor of Alg. 1: 2^-12 for e5m2, 2^-10 for the other MX formats; the
    // FP16 control uses binary16's smallest magnitude, 2^-24
    // FP32 reference ablation: binary32's smallest normal, 2^-126
    p->taumin_exp = format == MXFFT_E5M2 ? -12
                    : (format == MXFFT_FP16 ? -24 : (format == MXFFT_FP32_REF ? -126 : -10));
    p->kmin = -126;
    p->kmax = 126;
    p->fused2d = 0;
    p->fold_stats = 0;
    fmt_params(format, &p->fp);
    p->recs = new (std::nothrow) std::vector<ProfRec>();
    if (!p->recs) { delete p; return MXFFT_ERR_NOMEM; }
    p->recs->reserve(1024);
    p->m[0] = std::min(k / 2, n0 / 2);
    p->m[1] = std::min(k / 2, n1 / 2);

    int rc = MXFFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return MXFFT_ERR_CUDA; }
    for (int axis = 0; axis < 2 && rc == MXFFT_OK; axis++) {
        const int n = axis == 0 ? n0 : n1;
        std::vector<float2> fw, iv;
        std::vector<int8_t> sw;
        build_twiddles(n, p->m[axis], f, fw, iv, sw, format == MXFFT_FP16 || format == MXFFT_FP32_REF);
        for (int d = 0; d < 2 && rc == MXFFT_OK; d++) {
            const std::vector<float2>& t = d == 0 ? fw : iv;
            rc = cuda_status(plan_malloc((void**)&p->d_tw[axis][d], sizeof(float2) * t.size()));
            if (rc == MXFFT_OK)
                rc = cuda_status(cudaMemcpy(p->d_tw[axis][d], t.data(), sizeof(float2) * t.size(),
                                            cudaMemcpyHostToDevice));
        }
        for (int d = 0; d < 2 && rc == MXFFT_OK; d++) {
            const std::vector<float2>& t = d == 0 ? fw : iv;
            std::vector<uint32_t> h2(t.size());
            for (size_t i = 0; i < t.size(); i++) {
                const __half2 hh = __floats2half2_rn(t[i].x, t[i].y);   // exact: element values
                std::memcpy(&h2[i], &hh, sizeof(uint32_t));
            }
            for (int i = 0; i < 32; i++) {
                p->twa[axis][d].h2[i] = i < (int)h2.size() ? h2[i] : 0u;
                p->twa[axis][d].sw[i] = i < (int)sw.size() ? sw[i] : (int8_t)0;
            }
            // device copy shifted by one entry (stage h at index h + j): every run
            // of 8 twiddles the register pass loads starts 32-byte aligned
            std::vector<uint32_t> h2s(h2.size() + 1, 0u);
            std::copy(h2.begin(), h2.end(), h2s.begin() + 1);
            rc = cuda_status(plan_malloc((void**)&p->d_twh[axis][d], sizeof(uint32_t) * h2s.size()));
            if (rc == MXFFT_OK)
                rc = cuda_status(cudaMemcpy(p->d_twh[axis][d], h2s.data(), sizeof(uint32_t) * h2s.size(),
                                            cudaMemcpyHostToDevice));
        }
        if (rc == MXFFT_OK) rc = cuda_status(plan_malloc((void**)&p->d_tws[axis], sw.size()));
        if (rc == MXFFT_OK)
            rc = cuda_status(cudaMemcpy(p->d_tws[axis], sw.data(), sw.size(), cudaMemcpyHostToDevice));
    }
    if (rc == MXFFT_OK) rc = ensure_stats(p, 1);
    if (rc != MXFFT_OK) {
        free_plan_device(p);
        delete p->recs;
        delete p;
        return rc;
    }
    *out = p;
    return MXFFT_OK;
}

int mxfft_set_option(mxfft_plan_t p, int key, double value) {
    if (!p) return MXFFT_ERR_INVALID;
    switch (key) {
        case MXFFT_OPT_TAU_MIN: {
            int e;
            if (!exact_pow2_exp(value, &e) || e < -149 || e > 127) return MXFFT_ERR_INVALID;
            p->taumin_exp = e;
            return MXFFT_OK;
        }
        case MXFFT_OPT_K_MIN:
        case MXFFT_OPT_K_MAX: {
            if (value != std::floor(value) || value < -126 || value > 126) return MXFFT_ERR_INVALID;
            const int v = (int)value;
            if (key == MXFFT_OPT_K_MIN) p->kmin = v; else p->kmax = v;
            return MXFFT_OK;
        }
        case MXFFT_OPT_PATH: {
            if (value != 0.0 && value != 1.0) return MXFFT_ERR_INVALID;
            if (value == 0.0) { p->path = 0; return MXFFT_OK; }
            if ((p->kblk != 32 && p->kblk != 64 && p->kblk != 128) ||
                !tc16_supported(p->n1, p->n0, p->fmt) ||
                !tc16_supported(p->n0, p->n1, p->fmt))
                return MXFFT_ERR_UNSUPPORTED;
            const int rc = build_tc16_tables(p);
            if (rc) return rc;
            p->path = 1;
            return MXFFT_OK;
        }
        case MXFFT_OPT_GENERIC:
            if (value != 0.0 && value != 1.0) return MXFFT_ERR_INVALID;
            p->force_generic = value != 0.0;
            return MXFFT_OK;
        case MXFFT_OPT_TEST_STALL:
            if (value != 0.0 && value != 1.0) return MXFFT_ERR_INVALID;
            p->test_stall = value != 0.0;
            return MXFFT_OK;
        case MXFFT_OPT_FUSED2D:
            if (value != 0.0 && value != 1.0) return MXFFT_ERR_INVALID;
            p->fused2d = value != 0.0;
            return MXFFT_OK;
        case MXFFT_OPT_FOLD_STATS:
            if (value != 0.0 && value != 1.0) return MXFFT_ERR_INVALID;
            p->fold_stats = value != 0.0;
            return MXFFT_OK;
        default:
            return MXFFT_ERR_INVALID;
    }
}

int mxfft_forward(mxfft_plan_t p, const void* in, void* out, int batch, void* stream) {
    return run(p, in, out, batch, stream, 0);
}

int mxfft_inverse(mxfft_plan_t p, const void* in, void* out, int batch, void* stream) {
    return run(p, in, out, batch, stream, 1);
}

int mxfft_roundtrip(mxfft_plan_t p, const void* in, void* out, int batch, void* stream) {
    return run(p, in, out, batch, stream, 2);
}

int mxfft_roundtrip_fused(mxfft_plan_t p, const void* in, void* out, int batch, void* stream) {
    return run(p, in, out, batch, stream, 3);
}

int mxfft_get_status(mxfft_plan_t p, int* device_flags, int32_t* k_out) {
    if (!p) return MXFFT_ERR_INVALID;
    if (device_flags) *device_flags = 0;
    if (p->last_batch == 0) return MXFFT_OK;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int b = p->last_batch;
    std::vector<SliceStats> hf(b), hi;
    e = cudaMemcpy(hf.data(), p->d_st, sizeof(SliceStats) * b, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (p->last_op == 2) {
        hi.resize(b);
        e = cudaMemcpy(hi.data(), p->d_st + p->st_cap, sizeof(SliceStats) * b, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
    }
    int flags = 0;
    for (int i = 0; i < b; i++) {
        if (hf[i].nonfinite || (p->last_op == 2 && hi[i].nonfinite)) flags |= 1;
        if (k_out) {
            if (p->last_op == 2) {
                k_out[2 * i] = hf[i].k;
                k_out[2 * i + 1] = hi[i].k;
            } else {
                k_out[i] = hf[i].k;
            }
        }
    }
    if (p->d_err) {
        int herr = 0;
        e = cudaMemcpy(&herr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
        if (herr) flags |= 2;
    }
    if (device_flags) *device_flags = flags;
    if (flags & 2) return MXFFT_ERR_TIMEOUT;
    return (flags & 1) ? MXFFT_ERR_NONFINITE : MXFFT_OK;
}

int mxfft_destroy(mxfft_plan_t p) {
    if (!p) return MXFFT_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev == p->device) cudaDeviceSynchronize();
    prof_clear(p);
    delete p->recs;
    free_plan_device(p);
    delete p;
    return MXFFT_OK;
}

int mxfft_profile(mxfft_plan_t p, int enable) {
    if (!p) return MXFFT_ERR_INVALID;
    p->prof = enable != 0;
    return MXFFT_OK;
}

int mxfft_profile_read(mxfft_plan_t p, double* total_ms, int* launches, int nkinds) {
    if (!p || nkinds < 1) return MXFFT_ERR_INVALID;
    for (int i = 0; i < nkinds; i++) {
        if (total_ms) total_ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    int rc = MXFFT_OK;
    for (ProfRec& r : *p->recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) { rc = cuda_status(e); break; }
        if (r.kind < nkinds) {
            if (total_ms) total_ms[r.kind] += ms;
            if (launches) launches[r.kind] += 1;
        }
    }
    prof_clear(p);
    return rc;
}

int mxfft_debug_bounds(int* enabled, unsigned long long* violations) {
    if (!enabled || !violations) return MXFFT_ERR_INVALID;
#ifdef MXFFT_DEBUG_BOUNDS
    using namespace mxfft;
    if (cudaDeviceSynchronize() != cudaSuccess) return MXFFT_ERR_CUDA;
    unsigned long long (*const take[])() = {bounds_take_fast_f0, bounds_take_fast_f1,
                                            bounds_take_fast_f2, bounds_take_fast_f3,
                                            bounds_take_fast_f4, bounds_take_pass,
                                            bounds_take_tc16, bounds_take_tc2d};
    unsigned long long total = 0;
    for (auto f : take) {
        const unsigned long long v = f();
        if (v == ~0ull) return MXFFT_ERR_CUDA;
        total += v;
    }
    *enabled = 1;
    *violations = total;
#else
    *enabled = 0;
    *violations = 0;
#endif
    return MXFFT_OK;
}

int mxfft_test_fail_alloc(int after) {
    if (after < -1) return MXFFT_ERR_INVALID;
    g_fail_alloc_after.store(after);
    return MXFFT_OK;
}

const char* mxfft_status_string(int status) {
    switch (status) {
        case MXFFT_OK: return "ok";
        case MXFFT_ERR_INVALID: return "invalid argument";
        case MXFFT_ERR_UNSUPPORTED: return "unsupported request";
        case MXFFT_ERR_NOMEM: return "out of memory";
        case MXFFT_ERR_CUDA: return "CUDA runtime error";
        case MXFFT_ERR_NONFINITE: return "non-finite input magnitude";
        case MXFFT_ERR_TIMEOUT: return "bounded device wait timed out";
        default: return "unknown status";
    }
}

}  // extern "C"
