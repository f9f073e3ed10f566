/*
 * mxfft_oracle.c -- plain, slow CPU oracle of the MX-scaled low-precision 2D FFT
 * ("A mixed precision FFT with applications in MRI", arXiv 2512.04317).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference against which the CUDA
 * path is checked.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA library; the library never calls it.
 *
 * What it computes, step by step, in the paper's order:
 *   - Alg. 1 (Sec. 2.1): one power-of-two prescale per 2D slice, from the peak
 *     and the tau-percentile of the nonzero magnitudes; x_s = ldexp(x, k).
 *   - Radix-2 iterative decimation-in-time FFT (Fig. 1B), rows first, then
 *     columns (Eq. 1 applies it to N x N coil images).
 *   - Every butterfly is Alg. 2 (Sec. 2.2): MX-encode the twiddle block and the
 *     v block, multiply the de-scaled element values in FP32, renormalise,
 *     re-encode the product as a fresh MX block, decode, then u +/- wv in FP32.
 *   - Inverse: conjugate twiddles, its own prescale, no 1/N factor (Eq. 1 puts
 *     1/N^2 outside); round trip = (1/(n0 n1)) F^-1{F{x}} (Eq. 1).
 *   - The fused encode -> F -> F^-1 -> decode round trip of Sec. 4.3 as a
 *     declared variant (reading C17).
 *   - An FP64 "exact" mode with the same dataflow and no quantisation, used only
 *     to pin the dataflow (bit reversal, stage indexing, twiddles) to a DFT.
 *   - The root-sum-of-squares coil combine of Eq. (1) (oracle_rss).
 *   - The FP16 positive control of Sec. 2.2 (format code 5): the same dataflow
 *     with binary16 inputs and outputs and binary16 twiddle products.
 *   - An FP32 reference ablation (format code 6, reading C18): the same
 *     prescale and radix-2 dataflow with no quantisation at all.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   C1 k1 uses round-to-nearest; target and tau_min are powers of two.
 *   C2 tau is a fraction; the percentile is the "lower" order statistic with
 *      index floor(fl32(tau * fl32(n_nz - 1))).
 *   C3 |x| is computed as ldexp(sqrtf(a*a + b*b), e) with a, b the components
 *      scaled by 2^-e, e the larger frexp exponent of the nonzero components.
 *   C4 MX blocks are runs of m = min(k/2, n/2) consecutive butterflies in the
 *      canonical order b = g*h + j of one stage of one 1D transform.
 *   C5 EncodeFromMantBlock recomputes the shared scale (a fresh MX block).
 *   C6 M_max is the element format's largest normal.
 *   C8 non-finite magnitudes give k = 0 and a flag; a_max = 0 gives k = 0;
 *      an MX block holding Inf/NaN gets the NaN shared scale of OCP MX v1.0,
 *      so each of its elements decodes to NaN.
 *   C9 the output is unscaled by 2^-k.
 *   C10 twiddles are exact FP64 values exp(-+ 2 pi i j / (2h)), quantised
 *       directly from FP64.
 *   C15 signed zeros and subnormals are kept (IEEE); no FMA contraction.
 *   C16 the FP16 control keeps Alg. 1's prescale (default tau_min 2^-24, the
 *       smallest binary16 magnitude, so that the prescale sets the peak to the
 *       target and stage values stay below n0 n1 target) and the radix-2
 *       dataflow; each transform's input is rounded to binary16 after the
 *       prescale and its output before the exact unscale (the control runs in
 *       the prescaled domain, where outputs stay below n0 n1 target); in each
 *       butterfly the
 *       twiddle (rounded from FP64) and v are binary16, the complex product is
 *       formed with binary16 operations (each rounded once), u +- wv stays FP32.
 *   C17 the fused round trip encodes once and decodes once: Alg. 1's prescale
 *       of the input, the forward transform (rows, then columns), then the
 *       inverse applied directly to the forward result at the input's scale
 *       (no unscale, no second prescale, no re-encode of the forward output),
 *       columns first and then rows (the mirror order, so that both column
 *       transforms of a tile can run back to back), and one decode by
 *       2^(-k - log2(n0 n1)).  Its MX blocks are those of the separate
 *       transforms; only the inverse's axis order and the missing second
 *       prescale change the result.  Not defined for the FP16 control (its
 *       binary16 products would overflow at the unscaled intermediate size).
 *   C18 the FP32 reference ablation separates the quantisation error from
 *       FP32 rounding: Alg. 1's prescale (default tau_min 2^-126, binary32's
 *       smallest normal) and unscale, bit reversal and the same butterflies,
 *       with the twiddle rounded once from FP64 to FP32 (exact values at the
 *       multiples of pi/4) and the product (wr vr - wi vi, wr vi + wi vr)
 *       and u +- wv in FP32, each operation rounded once.
 *
 * Floating-point contract: compile with -ffp-contract=off and without
 * fast-math.  Every FP32 result below is one IEEE operation on FP32 operands.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Element formats (OCP 8-bit floating point and OCP MX v1.0 element types).  */
/* ------------------------------------------------------------------------- */

typedef struct {
    int ebits;      /* exponent field width */
    int mbits;      /* mantissa field width */
    int bias;       /* exponent bias */
    int emax;       /* unbiased exponent of the largest normal */
    int emin;       /* unbiased exponent of the smallest normal: 1 - bias */
    double maxnorm; /* largest finite magnitude */
    int fp16;       /* 1: the FP16 positive control, not an MX element format */
    int fp32;       /* 1: the FP32 reference ablation (no quantisation) */
} elem_fmt;

/* Format codes shared with the Python wrapper: 0 E4M3, 1 E5M2, 2 E2M3,
 * 3 E3M2, 4 E2M1.  The largest normal follows from the bit layout:
 *   E4M3: the all-ones exponent still holds normals, only S.1111.111 is NaN,
 *         so the largest normal is 1.110b * 2^(15-7) = 448.
 *   E5M2: the all-ones exponent is Inf/NaN (IEEE-like), so the largest normal
 *         is 1.11b * 2^(30-15) = 57344.
 *   E2M3, E3M2, E2M1: no special values; every code is a number, so the
 *         largest normal is the all-ones exponent with the all-ones mantissa.
 */
static int get_fmt(int code, elem_fmt *f)
{
    switch (code) {
    case 0: f->ebits = 4; f->mbits = 3; f->bias = 7;  f->emax = 15 - 7;
            f->maxnorm = ldexp(1.0 + 6.0 / 8.0, f->emax); break;
    case 1: f->ebits = 5; f->mbits = 2; f->bias = 15; f->emax = 30 - 15;
            f->maxnorm = ldexp(1.0 + 3.0 / 4.0, f->emax); break;
    case 2: f->ebits = 2; f->mbits = 3; f->bias = 1;  f->emax = 3 - 1;
            f->maxnorm = ldexp(1.0 + 7.0 / 8.0, f->emax); break;
    case 3: f->ebits = 3; f->mbits = 2; f->bias = 3;  f->emax = 7 - 3;
            f->maxnorm = ldexp(1.0 + 3.0 / 4.0, f->emax); break;
    case 4: f->ebits = 2; f->mbits = 1; f->bias = 1;  f->emax = 3 - 1;
            f->maxnorm = ldexp(1.0 + 1.0 / 2.0, f->emax); break;
    case 5: f->ebits = 5; f->mbits = 10; f->bias = 15; f->emax = 30 - 15;   /* IEEE binary16 */
            f->maxnorm = ldexp(2.0 - 1.0 / 1024.0, f->emax); break;
    case 6: f->ebits = 8; f->mbits = 23; f->bias = 127; f->emax = 254 - 127;   /* IEEE binary32 */
            f->maxnorm = ldexp(2.0 - ldexp(1.0, -23), f->emax); break;
    default: return -1;
    }
    f->emin = 1 - f->bias;
    f->fp16 = code == 5;
    f->fp32 = code == 6;
    return 0;
}

/* IEEE 754 binary16 rounding, for the FP16 positive control (Sec. 2.2): round
 * to nearest with ties to even, subnormals below 2^-14 (spacing 2^-24), and
 * overflow to infinity from 65520 up: the midpoint between the largest finite
 * value 65504 (odd significand) and 2^16 rounds up to even, i.e. to infinity.
 * NaN stays NaN, zero keeps its sign. */
static double q_fp16(double x)
{
    if (x != x || x == 0.0) return x;
    double a = fabs(x);
    if (a >= 65520.0) return copysign(INFINITY, x);
    int ex;
    frexp(a, &ex);              /* a = m 2^ex, m in [0.5, 1) */
    int e = ex - 1;             /* floor(log2 a) */
    if (e < -14) e = -14;
    double q = ldexp(1.0, e - 10);
    return copysign(rint(a / q) * q, x);
}

/* Round x to the nearest value of the element grid, ties to the even code,
 * saturating to +-maxnorm, keeping the sign of zero.  The grid spacing at |x|
 * is 2^(max(floor(log2|x|), emin) - mbits): normals carry mbits fraction bits,
 * subnormals share the spacing of the smallest binade.  An even code is an even
 * multiple of that spacing, so rint (round-half-even) on |x|/spacing is exact. */
static double q_elem(double x, const elem_fmt *f)
{
    if (x == 0.0 || isnan(x)) return x;
    if (isinf(x)) return copysign(f->maxnorm, x);
    double a = fabs(x);
    int e2;
    frexp(a, &e2);            /* a = fr * 2^e2, fr in [0.5, 1) */
    int E = e2 - 1;           /* floor(log2 a) */
    if (E < f->emin) E = f->emin;
    double q = ldexp(1.0, E - f->mbits);
    double r = rint(a / q) * q;
    if (r > f->maxnorm) r = f->maxnorm;
    return copysign(r, x);
}

/* Shared MX scale exponent of a block whose largest |component| is amax:
 * floor(log2 amax) - emax, kept within the E8M0 range [-127, 127]; an all-zero
 * block gets exponent 0 (OCP MX v1.0, Sec. 6.3). */
static int mx_scale_exp(double amax, const elem_fmt *f)
{
    if (amax == 0.0) return 0;
    int e2;
    frexp(amax, &e2);
    int s = (e2 - 1) - f->emax;
    if (s < -127) s = -127;
    if (s > 127) s = 127;
    return s;
}

/* ------------------------------------------------------------------------- */
/* Alg. 2: the MX-scaled complex butterfly over one block.                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int renorm;      /* apply the M_max renormalisation of Alg. 2 (default 1) */
    int direct_enc;  /* alternative reading of EncodeFromMantBlock: quantise the
                        (renormalised) element products under s_out itself */
} bf_opts;

/* nb complex butterflies.  u, v: FP32 interleaved; wre/wim: exact FP64
 * twiddles; y0 = u + w v and y1 = u - w v, FP32 interleaved. */
static void mx_butterfly_block(int nb, const float *u, const float *v,
                               const double *wre, const double *wim,
                               float *y0, float *y1, const elem_fmt *f,
                               const bf_opts *o, float *scratch)
{
    float *xr = scratch, *xi = xr + nb, *yr = xi + nb, *yi = yr + nb;
    float *pr = yi + nb, *pi = pr + nb;

    /* EncodeBlockMX(w) + MantissasBlock: shared scale s_w, element values x */
    double aw = 0.0;
    for (int b = 0; b < nb; b++) {
        aw = fmax(aw, fabs(wre[b]));
        aw = fmax(aw, fabs(wim[b]));
    }
    int sw = mx_scale_exp(aw, f);
    for (int b = 0; b < nb; b++) {
        xr[b] = (float)q_elem(ldexp(wre[b], -sw), f);
        xi[b] = (float)q_elem(ldexp(wim[b], -sw), f);
    }

    /* EncodeBlockMX(v) + MantissasBlock: shared scale s_v, element values y.
     * A block holding an Inf or NaN gets the NaN shared scale of OCP MX, so
     * every element of it decodes to NaN (reading C8). */
    float av = 0.0f;
    int nonfinite = 0;
    for (int b = 0; b < nb; b++) {
        if (!isfinite(v[2 * b]) || !isfinite(v[2 * b + 1])) nonfinite = 1;
        av = fmaxf(av, fabsf(v[2 * b]));
        av = fmaxf(av, fabsf(v[2 * b + 1]));
    }
    if (nonfinite) {
        for (int b = 0; b < nb; b++) {
            y0[2 * b] = u[2 * b] + NAN;
            y0[2 * b + 1] = u[2 * b + 1] + NAN;
            y1[2 * b] = u[2 * b] - NAN;
            y1[2 * b + 1] = u[2 * b + 1] - NAN;
        }
        return;
    }
    int sv = mx_scale_exp((double)av, f);
    for (int b = 0; b < nb; b++) {
        yr[b] = (float)q_elem((double)ldexpf(v[2 * b], -sv), f);
        yi[b] = (float)q_elem((double)ldexpf(v[2 * b + 1], -sv), f);
    }

    /* complex multiply in element ("mantissa") space, FP32 */
    for (int b = 0; b < nb; b++) {
        float rr = xr[b] * yr[b];
        float ii = xi[b] * yi[b];
        float ri = xr[b] * yi[b];
        float ir = xi[b] * yr[b];
        pr[b] = rr - ii;
        pi[b] = ri + ir;
    }

    /* s_out = s_w * s_v as scales, i.e. the sum of the exponents */
    int sout = sw + sv;
    float pmax = 0.0f;
    for (int b = 0; b < nb; b++) {
        pmax = fmaxf(pmax, fabsf(pr[b]));
        pmax = fmaxf(pmax, fabsf(pi[b]));
    }
    /* renormalise when the block maximum exceeds M_max: the smallest r with
     * pmax <= M_max * 2^r, i.e. r = ceil(log2(pmax / M_max)) */
    if (o->renorm && (double)pmax > f->maxnorm) {
        int r = 0;
        while ((double)pmax > ldexp(f->maxnorm, r)) r++;
        for (int b = 0; b < nb; b++) {
            pr[b] = ldexpf(pr[b], -r);
            pi[b] = ldexpf(pi[b], -r);
        }
        sout += r;
        pmax = ldexpf(pmax, -r);
    }

    /* EncodeFromMantBlock + DecodeBlockMX */
    for (int b = 0; b < nb; b++) {
        float cr, ci;
        int shat;
        if (o->direct_enc) {
            shat = sout;
            cr = (float)q_elem((double)pr[b], f);
            ci = (float)q_elem((double)pi[b], f);
        } else {
            if (pmax == 0.0f) {
                shat = sout;
            } else {
                int e2;
                frexpf(pmax, &e2);
                int t = (e2 - 1) - f->emax;
                shat = sout + t;
                if (shat < -127) shat = -127;
                if (shat > 127) shat = 127;
            }
            cr = (float)q_elem((double)ldexpf(pr[b], sout - shat), f);
            ci = (float)q_elem((double)ldexpf(pi[b], sout - shat), f);
        }
        float wvr = ldexpf(cr, shat);
        float wvi = ldexpf(ci, shat);
        /* butterfly sum and difference, FP32 */
        y0[2 * b] = u[2 * b] + wvr;
        y0[2 * b + 1] = u[2 * b + 1] + wvi;
        y1[2 * b] = u[2 * b] - wvr;
        y1[2 * b + 1] = u[2 * b + 1] - wvi;
    }
}

/* ------------------------------------------------------------------------- */
/* Radix-2 iterative DIT FFT of one 1D sequence (contiguous, interleaved).    */
/* ------------------------------------------------------------------------- */

static int ilog2i(int n) { int l = 0; while ((1 << l) < n) l++; return l; }

static int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

typedef struct {
    float *U, *V, *Y0, *Y1, *scr;
    double *Wr, *Wi;
    float *tmp;
} fft_ws;

static int ws_init(fft_ws *w, int nmax)
{
    int nb = nmax / 2 > 0 ? nmax / 2 : 1;
    w->U = malloc(sizeof(float) * 2 * nb);
    w->V = malloc(sizeof(float) * 2 * nb);
    w->Y0 = malloc(sizeof(float) * 2 * nb);
    w->Y1 = malloc(sizeof(float) * 2 * nb);
    w->scr = malloc(sizeof(float) * 6 * nb);
    w->Wr = malloc(sizeof(double) * nb);
    w->Wi = malloc(sizeof(double) * nb);
    w->tmp = malloc(sizeof(float) * 2 * nmax);
    return (w->U && w->V && w->Y0 && w->Y1 && w->scr && w->Wr && w->Wi && w->tmp) ? 0 : -1;
}

static void ws_free(fft_ws *w)
{
    free(w->U); free(w->V); free(w->Y0); free(w->Y1); free(w->scr);
    free(w->Wr); free(w->Wi); free(w->tmp);
}

/* FP16 positive control (Sec. 2.2): the twiddle product of each butterfly in
 * IEEE binary16 arithmetic -- the twiddle rounded to binary16 from FP64, v
 * rounded to binary16, every product, sum and difference rounded once to
 * binary16 (its exact value is formed in FP64, which holds any product, sum or
 * difference of two binary16 values exactly) -- then u +- wv in FP32. */
static void fp16_butterflies(int nb, const float *U, const float *V, const double *Wr,
                             const double *Wi, float *Y0, float *Y1)
{
    for (int b = 0; b < nb; b++) {
        double wr = q_fp16(Wr[b]), wi = q_fp16(Wi[b]);
        double vr = q_fp16(V[2 * b]), vi = q_fp16(V[2 * b + 1]);
        double pr = q_fp16(q_fp16(wr * vr) - q_fp16(wi * vi));
        double pi = q_fp16(q_fp16(wr * vi) + q_fp16(wi * vr));
        float fr = (float)pr, fi = (float)pi;   /* exact */
        Y0[2 * b] = U[2 * b] + fr;
        Y0[2 * b + 1] = U[2 * b + 1] + fi;
        Y1[2 * b] = U[2 * b] - fr;
        Y1[2 * b + 1] = U[2 * b + 1] - fi;
    }
}

/* exp(i sgn pi j / h), 0 <= j < h: the exact values 0, +-1, +-sqrt(1/2) at
 * the multiples of pi/4 (where cos / sin of the rounded angle would leave a
 * residue such as 6e-17 that FP32 keeps), cos / sin of pi j / h elsewhere. */
static void exact_twiddle(int j, int h, double sgn, double *c, double *s)
{
    if ((4L * j) % h == 0) {
        const double r = sqrt(0.5);
        const double cs[4] = {1.0, r, 0.0, -r}, sn[4] = {0.0, r, 1.0, r};
        int o = (int)(4L * j / h);      /* angle = o pi / 4, o = 0..3 */
        *c = cs[o];
        *s = sgn * sn[o];
        return;
    }
    double ang = M_PI * (double)j / (double)h;
    *c = cos(ang);
    *s = sgn * sin(ang);
}

/* FP32 reference ablation (reading C18): the twiddle rounded once to FP32,
 * the complex product and u +- wv in FP32, every operation rounded once. */
static void fp32_butterflies(int nb, const float *U, const float *V, const double *Wr,
                             const double *Wi, float *Y0, float *Y1)
{
    for (int b = 0; b < nb; b++) {
        float wr = (float)Wr[b], wi = (float)Wi[b];
        float vr = V[2 * b], vi = V[2 * b + 1];
        float a = wr * vr, bb = wi * vi, c = wr * vi, d = wi * vr;
        float pr = a - bb, pi = c + d;
        Y0[2 * b] = U[2 * b] + pr;
        Y0[2 * b + 1] = U[2 * b + 1] + pi;
        Y1[2 * b] = U[2 * b] - pr;
        Y1[2 * b + 1] = U[2 * b + 1] - pi;
    }
}

/* A: n complex values (interleaved FP32), transformed in place. */
static void fft1d_mx(float *A, int n, int kblk, int inverse, const elem_fmt *f,
                     const bf_opts *o, fft_ws *ws)
{
    int L = ilog2i(n);
    /* bit-reversed input order for decimation in time */
    memcpy(ws->tmp, A, sizeof(float) * 2 * n);
    for (int i = 0; i < n; i++) {
        int r = bitrev(i, L);
        A[2 * r] = ws->tmp[2 * i];
        A[2 * r + 1] = ws->tmp[2 * i + 1];
    }
    int nbf = n / 2;
    int m = kblk / 2;              /* complex values per MX block */
    if (m > nbf) m = nbf;
    double sgn = inverse ? 1.0 : -1.0;
    for (int h = 1; h < n; h <<= 1) {
        /* canonical butterfly order b = g*h + j */
        for (int b = 0; b < nbf; b++) {
            int g = b / h, j = b % h;
            int iu = 2 * h * g + j, iv = iu + h;
            ws->U[2 * b] = A[2 * iu];
            ws->U[2 * b + 1] = A[2 * iu + 1];
            ws->V[2 * b] = A[2 * iv];
            ws->V[2 * b + 1] = A[2 * iv + 1];
            if (f->fp32) {
                exact_twiddle(j, h, sgn, &ws->Wr[b], &ws->Wi[b]);
            } else {
                double ang = M_PI * (double)j / (double)h;   /* 2 pi j / (2h) */
                ws->Wr[b] = cos(ang);
                ws->Wi[b] = sgn * sin(ang);
            }
        }
        if (f->fp16) {
            fp16_butterflies(nbf, ws->U, ws->V, ws->Wr, ws->Wi, ws->Y0, ws->Y1);
        } else if (f->fp32) {
            fp32_butterflies(nbf, ws->U, ws->V, ws->Wr, ws->Wi, ws->Y0, ws->Y1);
        } else {
            for (int beta = 0; beta < nbf / m; beta++) {
                int b0 = beta * m;
                mx_butterfly_block(m, ws->U + 2 * b0, ws->V + 2 * b0, ws->Wr + b0,
                                   ws->Wi + b0, ws->Y0 + 2 * b0, ws->Y1 + 2 * b0,
                                   f, o, ws->scr);
            }
        }
        for (int b = 0; b < nbf; b++) {
            int g = b / h, j = b % h;
            int iu = 2 * h * g + j, iv = iu + h;
            A[2 * iu] = ws->Y0[2 * b];
            A[2 * iu + 1] = ws->Y0[2 * b + 1];
            A[2 * iv] = ws->Y1[2 * b];
            A[2 * iv + 1] = ws->Y1[2 * b + 1];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: global power-of-two prescale.                                      */
/* ------------------------------------------------------------------------- */

/* |x| per reading C3: scale both components by 2^-e (e the larger frexp
 * exponent of the nonzero components), take the FP32 sqrt of the FP32 sum of
 * squares, scale back by 2^e. */
static float mag_c3(float re, float im)
{
    if (isnan(re) || isnan(im)) return NAN;
    if (isinf(re) || isinf(im)) return INFINITY;
    if (re == 0.0f && im == 0.0f) return 0.0f;
    int e = -100000, t;
    if (re != 0.0f) { frexpf(re, &t); if (t > e) e = t; }
    if (im != 0.0f) { frexpf(im, &t); if (t > e) e = t; }
    float a = ldexpf(re, -e);
    float b = ldexpf(im, -e);
    float aa = a * a;
    float bb = b * b;
    float s = aa + bb;
    return ldexpf(sqrtf(s), e);
}

static int cmp_float(const void *p, const void *q)
{
    float a = *(const float *)p, b = *(const float *)q;
    return (a > b) - (a < b);
}

typedef struct {
    float tau;
    double target;
    double tau_min;
    int kmin, kmax;
} prescale_params;

/* Returns k; sets *nonfinite when a_max is not finite (then k = 0). */
static int prescale_k(const float *x, long cnt, const prescale_params *p,
                      int *nonfinite, float *magbuf)
{
    *nonfinite = 0;
    float amax = 0.0f;
    long nnz = 0;
    for (long i = 0; i < cnt; i++) {
        float m = mag_c3(x[2 * i], x[2 * i + 1]);
        if (!isfinite(m)) { *nonfinite = 1; continue; }
        if (m > amax) amax = m;
        if (m > 0.0f) magbuf[nnz++] = m;
    }
    if (*nonfinite) return 0;
    if (amax == 0.0f) return 0;
    /* tau-percentile of the nonzero magnitudes ("lower" order statistic) */
    qsort(magbuf, (size_t)nnz, sizeof(float), cmp_float);
    float rf = p->tau * (float)(nnz - 1);
    long r = (long)floorf(rf);
    if (r < 0) r = 0;
    if (r > nnz - 1) r = nnz - 1;
    float ptau = magbuf[r];
    const double eps = 1e-30;
    int k1 = (int)lround(log2(p->target / fmax((double)amax, eps)));
    int k2 = (int)ceil(log2(p->tau_min / fmax((double)ptau, eps)));
    int k = k1 > k2 ? k1 : k2;
    if (k < p->kmin) k = p->kmin;
    if (k > p->kmax) k = p->kmax;
    return k;
}

/* ------------------------------------------------------------------------- */
/* 2D driver.                                                                 */
/* ------------------------------------------------------------------------- */

static void rows_mx(float *S, int n0, int n1, int kblk, int inverse,
                    const elem_fmt *f, const bf_opts *o, fft_ws *ws)
{
    for (int r = 0; r < n0; r++)
        fft1d_mx(S + 2L * r * n1, n1, kblk, inverse, f, o, ws);
}

static void cols_mx(float *S, int n0, int n1, int kblk, int inverse,
                    const elem_fmt *f, const bf_opts *o, fft_ws *ws)
{
    float *col = malloc(sizeof(float) * 2 * n0);
    for (int c = 0; c < n1; c++) {
        for (int r = 0; r < n0; r++) {
            col[2 * r] = S[2L * ((long)r * n1 + c)];
            col[2 * r + 1] = S[2L * ((long)r * n1 + c) + 1];
        }
        fft1d_mx(col, n0, kblk, inverse, f, o, ws);
        for (int r = 0; r < n0; r++) {
            S[2L * ((long)r * n1 + c)] = col[2 * r];
            S[2L * ((long)r * n1 + c) + 1] = col[2 * r + 1];
        }
    }
    free(col);
}

/* One 2D transform: rows (length n1) first, then columns (reading C12). */
static void transform_slice(float *S, int n0, int n1, int kblk, int inverse,
                            const elem_fmt *f, const bf_opts *o, fft_ws *ws)
{
    rows_mx(S, n0, n1, kblk, inverse, f, o, ws);
    cols_mx(S, n0, n1, kblk, inverse, f, o, ws);
}

static int valid_pow2(int n) { return n >= 2 && n <= 4096 && (n & (n - 1)) == 0; }

/* op: 0 forward, 1 inverse, 2 round trip, 3 fused round trip (reading C17).
 * in/out: [batch][n0][n1] complex64 interleaved (in == out allowed).  k_out:
 * [batch] prescale exponents (for the round trip, k_out[2b] = forward k and
 * k_out[2b+1] = inverse k), flags_out: [batch] nonzero when a prescale saw a
 * non-finite magnitude.  Returns 0, or -1 on bad arguments (op 3 with the FP16
 * control) / allocation failure. */
int oracle_mxfft2d(const float *in, float *out, int batch, int n0, int n1,
                   int fmt, int kblk, float tau, double target, double tau_min,
                   int kmin, int kmax, int op, int renorm, int direct_enc,
                   int32_t *k_out, int32_t *flags_out)
{
    elem_fmt f;
    if (get_fmt(fmt, &f) || !valid_pow2(n0) || !valid_pow2(n1) || batch < 0 ||
        kblk < 2 || (kblk & (kblk - 1)) || op < 0 || op > 3 || (op == 3 && f.fp16))
        return -1;
    bf_opts o = {renorm, direct_enc};
    prescale_params pp = {tau, target, tau_min, kmin, kmax};
    long npts = (long)n0 * n1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int s = 0; s < batch; s++) {
        fft_ws ws;
        int nmax = n0 > n1 ? n0 : n1;
        float *S = malloc(sizeof(float) * 2 * npts);
        float *mag = malloc(sizeof(float) * npts);
        if (ws_init(&ws, nmax) || !S || !mag) { bad |= 1; ws_free(&ws); free(S); free(mag); continue; }
        memcpy(S, in + 2 * npts * s, sizeof(float) * 2 * npts);
        int nf = 0, k;
        int inv0 = (op == 1);
        /* first transform: forward (op 0, 2) or inverse (op 1) */
        /* the FP16 control rounds each transform's input (after the
         * prescale) and output (before the exact unscale) to binary16: it runs
         * in the prescaled domain */
        const int q16 = f.fp16;
        k = prescale_k(S, npts, &pp, &nf, mag);
        int flag = nf;
        for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], k);
        if (q16) for (long i = 0; i < 2 * npts; i++) S[i] = (float)q_fp16(S[i]);
        transform_slice(S, n0, n1, kblk, inv0, &f, &o, &ws);
        if (op == 2) {
            if (k_out) k_out[2 * s] = k;
            /* forward output y = ldexp(A, -k), then the inverse with its own
             * prescale, and one combined scaling by 2^(-k_inv - log2(n0 n1)) */
            if (q16) for (long i = 0; i < 2 * npts; i++) S[i] = (float)q_fp16(S[i]);
            for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], -k);
            int nf2 = 0;
            int kinv = prescale_k(S, npts, &pp, &nf2, mag);
            flag |= nf2;
            for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], kinv);
            if (q16) for (long i = 0; i < 2 * npts; i++) S[i] = (float)q_fp16(S[i]);
            transform_slice(S, n0, n1, kblk, 1, &f, &o, &ws);
            int lg = ilog2i(n0) + ilog2i(n1);
            if (q16) for (long i = 0; i < 2 * npts; i++) S[i] = (float)q_fp16(S[i]);
            for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], -kinv - lg);
            if (k_out) k_out[2 * s + 1] = kinv;
        } else if (op == 3) {
            /* fused round trip: the forward result A stays at the input's
             * scale (no unscale, no second prescale); the inverse runs
             * columns first, then rows; one combined decode by
             * 2^(-k - log2(n0 n1)) */
            cols_mx(S, n0, n1, kblk, 1, &f, &o, &ws);
            rows_mx(S, n0, n1, kblk, 1, &f, &o, &ws);
            int lg = ilog2i(n0) + ilog2i(n1);
            for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], -k - lg);
            if (k_out) k_out[s] = k;
        } else {
            if (q16) for (long i = 0; i < 2 * npts; i++) S[i] = (float)q_fp16(S[i]);
            for (long i = 0; i < 2 * npts; i++) S[i] = ldexpf(S[i], -k);
            if (k_out) k_out[s] = k;
        }
        if (flags_out) flags_out[s] = flag;
        memcpy(out + 2 * npts * s, S, sizeof(float) * 2 * npts);
        ws_free(&ws);
        free(S);
        free(mag);
    }
    return bad ? -1 : 0;
}

/* Alg. 1 alone on one slice (count complex values): returns k. */
int oracle_prescale_k(const float *x, long count, float tau, double target,
                      double tau_min, int kmin, int kmax, int32_t *nonfinite)
{
    prescale_params pp = {tau, target, tau_min, kmin, kmax};
    float *mag = malloc(sizeof(float) * (count > 0 ? count : 1));
    int nf = 0;
    int k = prescale_k(x, count, &pp, &nf, mag);
    free(mag);
    if (nonfinite) *nonfinite = nf;
    return k;
}

/* |x| per reading C3, elementwise (count complex values). */
void oracle_magnitude(const float *x, float *m, long count)
{
    for (long i = 0; i < count; i++) m[i] = mag_c3(x[2 * i], x[2 * i + 1]);
}

/* Element quantiser on FP32 values that are already divided by the block
 * scale (no block scale applied here). */
int oracle_quantize(const float *in, float *out, long count, int fmt)
{
    elem_fmt f;
    if (get_fmt(fmt, &f)) return -1;
    for (long i = 0; i < count; i++)
        out[i] = (float)(f.fp16 ? q_fp16((double)in[i]) : q_elem((double)in[i], &f));
    return 0;
}

/* Same quantiser on FP64 values (used for twiddles). */
int oracle_quantize_f64(const double *in, double *out, long count, int fmt)
{
    elem_fmt f;
    if (get_fmt(fmt, &f)) return -1;
    for (long i = 0; i < count; i++) out[i] = (f.fp16 ? q_fp16(in[i]) : q_elem(in[i], &f));
    return 0;
}

/* One Alg. 2 block on nb complex values: returns y0, y1 (FP32 interleaved). */
int oracle_butterfly_block(int nb, const float *u, const float *v,
                           const double *wre, const double *wim, float *y0,
                           float *y1, int fmt, int renorm, int direct_enc)
{
    elem_fmt f;
    if (get_fmt(fmt, &f) || nb < 1) return -1;
    if (f.fp16) {
        fp16_butterflies(nb, u, v, wre, wim, y0, y1);
        return 0;
    }
    bf_opts o = {renorm, direct_enc};
    float *scr = malloc(sizeof(float) * 6 * nb);
    mx_butterfly_block(nb, u, v, wre, wim, y0, y1, &f, &o, scr);
    free(scr);
    return 0;
}

/* Format constants, for tests: emax, emin, mbits, maxnorm. */
int oracle_format_info(int fmt, int32_t *emax, int32_t *emin, int32_t *mbits,
                       double *maxnorm)
{
    elem_fmt f;
    if (get_fmt(fmt, &f)) return -1;
    *emax = f.emax; *emin = f.emin; *mbits = f.mbits; *maxnorm = f.maxnorm;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* FP64 exact mode: same bit reversal, stage order and butterfly indexing,    */
/* double arithmetic, no quantisation, no prescale.                           */
/* ------------------------------------------------------------------------- */

static void fft1d_f64(double *A, int n, int inverse, double *tmp)
{
    int L = ilog2i(n);
    memcpy(tmp, A, sizeof(double) * 2 * n);
    for (int i = 0; i < n; i++) {
        int r = bitrev(i, L);
        A[2 * r] = tmp[2 * i];
        A[2 * r + 1] = tmp[2 * i + 1];
    }
    double sgn = inverse ? 1.0 : -1.0;
    for (int h = 1; h < n; h <<= 1) {
        for (int b = 0; b < n / 2; b++) {
            int g = b / h, j = b % h;
            int iu = 2 * h * g + j, iv = iu + h;
            double ang = M_PI * (double)j / (double)h;
            double wr = cos(ang), wi = sgn * sin(ang);
            double vr = A[2 * iv], vi = A[2 * iv + 1];
            double pr = wr * vr - wi * vi, pi = wr * vi + wi * vr;
            double ur = A[2 * iu], ui = A[2 * iu + 1];
            A[2 * iu] = ur + pr; A[2 * iu + 1] = ui + pi;
            A[2 * iv] = ur - pr; A[2 * iv + 1] = ui - pi;
        }
    }
}

static void rows_f64(double *S, int n0, int n1, int inv, double *tmp)
{
    for (int r = 0; r < n0; r++) fft1d_f64(S + 2L * r * n1, n1, inv, tmp);
}

static void cols_f64(double *S, int n0, int n1, int inv, double *tmp, double *col)
{
    for (int c = 0; c < n1; c++) {
        for (int r = 0; r < n0; r++) {
            col[2 * r] = S[2L * ((long)r * n1 + c)];
            col[2 * r + 1] = S[2L * ((long)r * n1 + c) + 1];
        }
        fft1d_f64(col, n0, inv, tmp);
        for (int r = 0; r < n0; r++) {
            S[2L * ((long)r * n1 + c)] = col[2 * r];
            S[2L * ((long)r * n1 + c) + 1] = col[2 * r + 1];
        }
    }
}

/* op: 0 forward, 1 inverse (unnormalised), 2 round trip (with 1/(n0 n1)),
 * 3 fused round trip (inverse columns first, then rows; with 1/(n0 n1)). */
int oracle_fft2d_exact(const double *in, double *out, int batch, int n0, int n1, int op)
{
    if (!valid_pow2(n0) || !valid_pow2(n1) || batch < 0 || op < 0 || op > 3) return -1;
    long npts = (long)n0 * n1;
    int nmax = n0 > n1 ? n0 : n1;
    double *tmp = malloc(sizeof(double) * 2 * nmax);
    double *col = malloc(sizeof(double) * 2 * n0);
    for (int s = 0; s < batch; s++) {
        double *S = out + 2 * npts * s;
        memmove(S, in + 2 * npts * s, sizeof(double) * 2 * npts);
        rows_f64(S, n0, n1, op == 1, tmp);
        cols_f64(S, n0, n1, op == 1, tmp, col);
        if (op == 2) {
            rows_f64(S, n0, n1, 1, tmp);
            cols_f64(S, n0, n1, 1, tmp, col);
        } else if (op == 3) {
            cols_f64(S, n0, n1, 1, tmp, col);
            rows_f64(S, n0, n1, 1, tmp);
        }
        if (op >= 2)
            for (long i = 0; i < 2 * npts; i++) S[i] /= (double)npts;
    }
    free(tmp);
    free(col);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. (1): root-sum-of-squares coil combine.                                 */
/* ------------------------------------------------------------------------- */

/* x_RSS = (sum over coils c of |T_c|^2)^(1/2) per point.  z holds images * coils
 * slices of npts interleaved complex points, slice i * coils + c being coil c
 * of image i; out[i * npts + p] (FP32).  Coils are added in the order
 * c = 0, 1, ...: acc = fl(acc + fl(fl(re*re) + fl(im*im))), then one correctly
 * rounded square root. */
void oracle_rss(const float *z, float *out, long images, int coils, long npts)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < images; i++) {
        for (long p = 0; p < npts; p++) {
            float acc = 0.0f;
            for (int c = 0; c < coils; c++) {
                const float *v = z + 2 * (((long)i * coils + c) * npts + p);
                float re2 = v[0] * v[0];
                float im2 = v[1] * v[1];
                float m2 = re2 + im2;
                acc = acc + m2;
            }
            out[i * npts + p] = sqrtf(acc);
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
