"""Independent numpy emulation of the FP16 positive control (Sec. 2.2) for
small transforms: the radix-2 decimation-in-time dataflow written directly,
with every binary16 operation formed exactly in float64 and rounded once by
numpy's IEEE float64 -> float16 conversion, FP32 additions by numpy float32.
Shares nothing with the oracle but the prescale exponent it is handed."""
import numpy as np


def h16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def _bitrev(i, bits):
    r = 0
    for b in range(bits):
        r |= ((i >> b) & 1) << (bits - 1 - b)
    return r


def fft1d(re, im, inverse):
    """re, im: float32 arrays of length n (power of two), transformed in place."""
    n = len(re)
    bits = n.bit_length() - 1
    perm = [_bitrev(i, bits) for i in range(n)]
    R = np.empty(n, np.float32)
    I = np.empty(n, np.float32)
    R[perm] = re
    I[perm] = im
    sgn = 1.0 if inverse else -1.0
    h = 1
    while h < n:
        for b in range(n // 2):
            g, j = divmod(b, h)
            iu = 2 * h * g + j
            iv = iu + h
            wr = h16(np.cos(np.pi * j / h))
            wi = h16(sgn * np.sin(np.pi * j / h))
            vr, vi = h16(R[iv]), h16(I[iv])
            pr = np.float32(h16(h16(wr * vr) - h16(wi * vi)))
            pi = np.float32(h16(h16(wr * vi) + h16(wi * vr)))
            ur, ui = R[iu], I[iu]
            R[iu], I[iu] = ur + pr, ui + pi
            R[iv], I[iv] = ur - pr, ui - pi
        h *= 2
    return R, I


def fft2d(x, k, inverse):
    """One prescaled 2D transform of a complex64 slice, rows then columns."""
    re = np.ldexp(x.real.astype(np.float32), k).astype(np.float32)
    im = np.ldexp(x.imag.astype(np.float32), k).astype(np.float32)
    re, im = h16(re).astype(np.float32), h16(im).astype(np.float32)
    n0, n1 = x.shape
    for r in range(n0):
        re[r], im[r] = fft1d(re[r].copy(), im[r].copy(), inverse)
    for c in range(n1):
        cr, ci = fft1d(re[:, c].copy(), im[:, c].copy(), inverse)
        re[:, c], im[:, c] = cr, ci
    return re, im


def mxfft2d_fp16(x, k, op, k_inv=None):
    """x: complex64 [n0, n1]; k (and k_inv for the round trip) from Alg. 1."""
    # outputs rounded to binary16 in the prescaled domain, then unscaled exactly
    inv0 = op == "inverse"
    re, im = fft2d(x, k, inv0)
    re, im = h16(re).astype(np.float32), h16(im).astype(np.float32)
    re = np.ldexp(re, -k).astype(np.float32)
    im = np.ldexp(im, -k).astype(np.float32)
    if op == "roundtrip":
        y = (re + 1j * im).astype(np.complex64)
        re, im = fft2d(y, k_inv, True)
        lg = (x.shape[0].bit_length() - 1) + (x.shape[1].bit_length() - 1)
        re, im = h16(re).astype(np.float32), h16(im).astype(np.float32)
        re = np.ldexp(re, -k_inv - lg).astype(np.float32)
        im = np.ldexp(im, -k_inv - lg).astype(np.float32)
    return (re + 1j * im).astype(np.complex64)
