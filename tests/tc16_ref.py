"""numpy emulation of the tensor-core radix-16 variant (MXFFT_OPT_PATH = 1),
written from its description: four-step n = 16 x 16 r (n = 128: 16 x 8, the
second round 8-point DFTs of pairs of vectors), each 16-point input
vector one MX block (k = 32; for k = 64 / 128 a block is 2 / 4 consecutive
vectors of a transform), the real 32 x 32 DFT matrix quantised with one shared
scale per output row, products exact and accumulated in FP64 (the hardware
accumulates 32 exact products in FP32, so results agree to ~1e-7 relative),
MX-quantised twiddles multiplied in FP32.  Uses the oracle's element rounding
and Alg. 1 (test infrastructure only)."""
import numpy as np

import oracle

EMAX = {"e4m3": 8, "e5m2": 15}


def _scale_exp(amax, emax):
    s = np.zeros(amax.shape, np.int64)
    nz = amax > 0
    s[nz] = np.floor(np.log2(amax[nz].astype(np.float64))).astype(np.int64) - emax
    return np.clip(s, -127, 127)


def _q(x, fmt):
    return oracle.quantize(np.ascontiguousarray(x, np.float32), fmt).astype(np.float64)


def twiddle_block(m, N, sgn, fmt):
    """16 MX-quantised twiddles exp(sgn 2 pi i m idx / N), back-scaled."""
    idx = np.arange(16)
    ang = 2 * np.pi * ((m * idx) % N) / N
    c, s = np.cos(ang), sgn * np.sin(ang)
    c[np.abs(c) < 1e-12] = 0.0
    s[np.abs(s) < 1e-12] = 0.0
    amax = max(np.abs(c).max(), np.abs(s).max())
    sc = int(np.floor(np.log2(amax))) - EMAX[fmt]
    qc = oracle.quantize(np.ldexp(c, -sc), fmt) * 2.0 ** sc
    qs = oracle.quantize(np.ldexp(s, -sc), fmt) * 2.0 ** sc
    return qc.astype(np.float32) + 1j * qs.astype(np.float32)


def dft16_matrix(sgn, fmt):
    """(element values [32, 32], row scale exponents [32])."""
    F = np.zeros((32, 32))
    for m in range(16):
        for j in range(16):
            ang = 2 * np.pi * ((j * m) % 16) / 16
            c, s = np.cos(ang), sgn * np.sin(ang)
            c = 0.0 if abs(c) < 1e-12 else c
            s = 0.0 if abs(s) < 1e-12 else s
            F[2 * m, 2 * j], F[2 * m, 2 * j + 1] = c, -s
            F[2 * m + 1, 2 * j], F[2 * m + 1, 2 * j + 1] = s, c
    sF = _scale_exp(np.abs(F).max(axis=1), EMAX[fmt])
    Fq = oracle.quantize(np.ldexp(F, -sF[:, None]), fmt)
    return Fq, sF


def dft8pair_matrix(sgn, fmt):
    """The 8-point DFT twice on the diagonal of the real 32 x 32 matrix (a row
    of 16 complex elements = two 8-point vectors), quantised like the
    16-point matrix: (element values, row scale exponents)."""
    F = np.zeros((32, 32))
    for b in range(2):
        for m in range(8):
            for j in range(8):
                ang = 2 * np.pi * ((j * m) % 8) / 8
                c, s = np.cos(ang), sgn * np.sin(ang)
                c = 0.0 if abs(c) < 1e-12 else c
                s = 0.0 if abs(s) < 1e-12 else s
                r0, c0 = 2 * (8 * b + m), 2 * (8 * b + j)
                F[r0, c0], F[r0, c0 + 1] = c, -s
                F[r0 + 1, c0], F[r0 + 1, c0 + 1] = s, c
    sF = _scale_exp(np.abs(F).max(axis=1), EMAX[fmt])
    Fq = oracle.quantize(np.ldexp(F, -sF[:, None]), fmt)
    return Fq, sF


def dft16_mx(V, fmt, sgn, g=1, vec_axes=1, matrix=None):
    """V: complex64 [..., vectors, 16] -> complex64 [..., vectors, 16].  With
    k = 32 g one MX block is g consecutive vectors of a transform (the last
    vec_axes axes before the element axis, flattened in order).  matrix:
    (element values, row scale exponents) of another 32 x 32 real matrix than
    the 16-point DFT's."""
    r = np.stack([V.real, V.imag], -1).reshape(V.shape[:-1] + (32,)).astype(np.float32)
    amax = np.abs(r).max(-1)
    if g > 1:
        lead = amax.shape[:amax.ndim - vec_axes]
        a = amax.reshape(lead + (-1, g)).max(-1, keepdims=True)
        amax = np.broadcast_to(a, lead + (a.shape[-2], g)).reshape(amax.shape)
    sv = _scale_exp(amax, EMAX[fmt])
    q = _q(r * np.exp2(-sv)[..., None].astype(np.float32), fmt)
    Fq, sF = dft16_matrix(sgn, fmt) if matrix is None else matrix
    D = (q @ Fq.T).astype(np.float32)                    # exact products, FP32 result
    y = (D * np.exp2(sF).astype(np.float32)) * np.exp2(sv)[..., None].astype(np.float32)
    return (y[..., 0::2] + 1j * y[..., 1::2]).astype(np.complex64)


def cmul32(w, y):
    w = w.astype(np.complex64)
    y = y.astype(np.complex64)
    wr, wi, yr, yi = (np.float32(0) + a for a in (w.real, w.imag, y.real, y.imag))
    return ((wr * yr - wi * yi) + 1j * (wr * yi + wi * yr)).astype(np.complex64)


def fft1d(x, fmt, sgn, g=1):
    """x: complex64 [..., n], n in {128, 256, 512, 1024, 2048}; transforms the last axis."""
    n = x.shape[-1]
    r = n // 256
    M = n // 16
    X = x.reshape(x.shape[:-1] + (16, M))                # [j1][j2]
    V = np.swapaxes(X, -1, -2)                          # [j2][j1]
    Y = dft16_mx(V, fmt, sgn, g)                        # [j2][k1]
    TA = np.stack([twiddle_block(j2, n, sgn, fmt) for j2 in range(M)])  # [j2][k1]
    Y = cmul32(TA, Y)
    Y = np.swapaxes(Y, -1, -2)                          # [k1][j2]
    if n == 128:
        # pairs (k1 = 2 p, 2 p + 1) of 8-point vectors over j2, one MMA row each
        P = Y.reshape(Y.shape[:-2] + (8, 16))           # [p][(k1 parity, j2)]
        Z = dft16_mx(P, fmt, sgn, g, matrix=dft8pair_matrix(sgn, fmt))   # [p][(parity, k2)]
        Z = Z.reshape(Y.shape[:-2] + (16, 8))           # [k1][k2]
        return np.swapaxes(Z, -1, -2).reshape(x.shape)  # X[k1 + 16 k2]
    if r == 1:
        Z = dft16_mx(Y, fmt, sgn, g)                    # [k1][k2]
        return np.swapaxes(Z, -1, -2).reshape(x.shape)  # X[k1 + 16 k2]
    Yr = Y.reshape(Y.shape[:-1] + (16, r))              # [k1][j21][j22]
    U = dft16_mx(np.swapaxes(Yr, -1, -2), fmt, sgn, g, 2)   # [k1][j22][k21]
    TC = np.stack([twiddle_block(j22, M, sgn, fmt) for j22 in range(r)])   # [j22][k21]
    U = cmul32(TC, U)
    if r == 8:
        # radix 4 on the even and the odd j22, then the odd half times W_8^k
        # (sqrt(1/2) rounded to FP32); the same operations as the kernel
        f32 = np.float32
        sg = f32(sgn)

        def radix4(x0, x1, x2, x3):
            a0, a1 = (x0 + x2).astype(np.complex64), (x0 - x2).astype(np.complex64)
            b0, b1 = (x1 + x3).astype(np.complex64), (x1 - x3).astype(np.complex64)
            wb = (-sg * b1.imag + 1j * (sg * b1.real)).astype(np.complex64)
            return [(a0 + b0).astype(np.complex64), (a1 + wb).astype(np.complex64),
                    (a0 - b0).astype(np.complex64), (a1 - wb).astype(np.complex64)]
        Uj = [U[..., j, :] for j in range(8)]
        E = radix4(Uj[0], Uj[2], Uj[4], Uj[6])
        O = radix4(Uj[1], Uj[3], Uj[5], Uj[7])
        c8 = f32(0.70710678118654752)
        o1r, o1i, o3r, o3i = O[1].real, O[1].imag, O[3].real, O[3].imag
        P = [O[0],
             ((o1r - sg * o1i) * c8 + 1j * ((o1i + sg * o1r) * c8)).astype(np.complex64),
             (-sg * O[2].imag + 1j * (sg * O[2].real)).astype(np.complex64),
             (-((o3r + sg * o3i) * c8) + 1j * ((sg * o3r - o3i) * c8)).astype(np.complex64)]
        X = [(E[k] + P[k]).astype(np.complex64) for k in range(4)] + \
            [(E[k] - P[k]).astype(np.complex64) for k in range(4)]
        out = np.stack(X, -1)                           # [k1][k21][k22]
        return np.swapaxes(out, -1, -3).reshape(x.shape)
    if r == 2:
        a, b = U[..., 0, :], U[..., 1, :]               # [k1][k21]
        s0 = (a + b).astype(np.complex64)
        s1 = (a - b).astype(np.complex64)
        out = np.stack([s0, s1], -1)                    # [k1][k21][k22]
    else:
        # radix 4 in FP32 with W_4 = sgn i (exact): the same additions in the
        # same order as the kernel
        U0, U1, U2, U3 = (U[..., j, :] for j in range(4))
        a0, a1 = (U0 + U2).astype(np.complex64), (U0 - U2).astype(np.complex64)
        b0, b1 = (U1 + U3).astype(np.complex64), (U1 - U3).astype(np.complex64)
        wb = (np.float32(-sgn) * b1.imag + 1j * (np.float32(sgn) * b1.real)).astype(np.complex64)
        out = np.stack([a0 + b0, a1 + wb, a0 - b0, a1 - wb], -1).astype(np.complex64)
    return np.swapaxes(out, -1, -3).reshape(x.shape)    # [k22][k21][k1]: k = k1 + 16 (k21 + 16 k22)


def mxfft2d(x, fmt="e4m3", op="forward", k=32):
    """Batch [..., n0, n1] complex64; same prescale (Alg. 1) as the library;
    k in {32, 64, 128} (blocks of k / 32 consecutive vectors)."""
    g = k // 32
    x = np.asarray(x, np.complex64)
    out = np.empty_like(x)
    flat = x.reshape((-1,) + x.shape[-2:])
    res = out.reshape(flat.shape)
    for i, s in enumerate(flat):
        def transform(z, sgn):
            ke, _ = oracle.prescale_k(z, fmt)
            zs = (z * np.float32(2.0 ** ke)).astype(np.complex64)
            zs = fft1d(zs, fmt, sgn, g)                                      # rows
            zs = np.swapaxes(fft1d(np.swapaxes(zs, 0, 1).copy(), fmt, sgn, g), 0, 1)   # columns
            return zs, ke
        if op == "forward":
            y, ke = transform(s, -1)
            res[i] = y * np.float32(2.0 ** -ke)
        elif op == "inverse":
            y, ke = transform(s, +1)
            res[i] = y * np.float32(2.0 ** -ke)
        elif op == "roundtrip_fused":
            # one prescale; the inverse on the undecoded forward result,
            # columns first, then rows; one decode
            y, ke = transform(s, -1)
            z = np.swapaxes(fft1d(np.swapaxes(y, 0, 1).copy(), fmt, +1, g), 0, 1)
            z = fft1d(z, fmt, +1, g)
            lg = int(np.log2(s.shape[0] * s.shape[1]))
            res[i] = z * np.float32(2.0 ** (-ke - lg))
        else:
            y, ke = transform(s, -1)
            y = (y * np.float32(2.0 ** -ke)).astype(np.complex64)
            z, ki = transform(y, +1)
            lg = int(np.log2(s.shape[0] * s.shape[1]))
            res[i] = z * np.float32(2.0 ** (-ki - lg))
    return out
