"""The oracle's FP32 reference ablation (format "fp32"): the method's prescale
and radix-2 dataflow with no quantisation, so that an MX format's distance to
it is its quantisation error.  Pinned (1) to a plain float32 radix-2 FFT
written here for sizes whose twiddles are all exact (n <= 8: multiples of pi/4),
bit for bit, (2) to the exact DFT within FP32 rounding at larger sizes, and
(3) as the floor of the MX formats' error."""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

f32 = np.float32


def fft1d_f32(x, sgn):
    """Decimation-in-time radix-2 FFT of a complex64 vector in float32, every
    product, sum and difference rounded once; twiddles exp(sgn i pi j / h) for
    n <= 8 are exact (0, +-1, +-sqrt(1/2) rounded to float32)."""
    n = len(x)
    L = n.bit_length() - 1
    rev = [int(format(i, f"0{L}b")[::-1], 2) if L else 0 for i in range(n)]
    re = np.array([x[r].real for r in rev], f32)
    im = np.array([x[r].imag for r in rev], f32)
    h = 1
    r2 = f32(np.sqrt(0.5))
    table = {0: (f32(1), f32(0)), 1: (r2, r2), 2: (f32(0), f32(1)), 3: (-r2, r2)}
    while h < n:
        for g in range(n // (2 * h)):
            for j in range(h):
                o = 4 * j // h                     # angle = o pi / 4 (exact for n <= 8)
                assert (4 * j) % h == 0
                wr, wi = table[o]
                wi = f32(sgn) * wi
                iu, iv = 2 * h * g + j, 2 * h * g + j + h
                pr = f32(f32(wr * re[iv]) - f32(wi * im[iv]))
                pi = f32(f32(wr * im[iv]) + f32(wi * re[iv]))
                ur, ui = re[iu], im[iu]
                re[iu], im[iu] = f32(ur + pr), f32(ui + pi)
                re[iv], im[iv] = f32(ur - pr), f32(ui - pi)
        h *= 2
    return (re + 1j * im).astype(np.complex64)


def fft2d_f32(x, sgn):
    y = np.array([fft1d_f32(r, sgn) for r in x])
    return np.array([fft1d_f32(c, sgn) for c in y.T]).T


@pytest.mark.parametrize("n0,n1", [(2, 2), (4, 8), (8, 2), (8, 8)])
@pytest.mark.parametrize("op", ["forward", "inverse"])
def test_small_sizes_equal_plain_float32_fft(n0, n1, op):
    x = phantom.random_complex((3, n0, n1), seed=n0 * 10 + n1, scale=5.0)
    # k = 0 (prescale and unscale are the identity) so that the plain FFT
    # needs no prescale of its own
    got, kexp, _ = oracle.mxfft2d(x, "fp32", 32, op=op, kmin=0, kmax=0)
    assert np.all(kexp == 0)
    want = np.array([fft2d_f32(s, -1 if op == "forward" else 1) for s in x])
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_prescale_is_exact_scaling():
    # a power-of-two prescale and unscale commute with float32 rounding
    # (no overflow or underflow here), so the result does not depend on k
    x = phantom.random_complex((2, 8, 8), seed=5)
    a = oracle.mxfft2d(x, "fp32", 32, kmin=0, kmax=0)[0]
    b, kb, _ = oracle.mxfft2d(x, "fp32", 32)
    assert np.all(kb != 0)
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("n0,n1", [(64, 64), (256, 256), (128, 1024), (2048, 16)])
def test_close_to_exact_dft(n0, n1):
    x = phantom.random_complex((2, n0, n1), seed=n0 + n1, scale=3.0)
    xd = x.astype(np.complex128)
    fwd = oracle.mxfft2d(x, "fp32", 32)[0].astype(np.complex128)
    ref = np.fft.fft2(xd)
    # FP32 radix-2: error grows like log2(n0 n1) x 2^-24
    bound = 2.0 * np.log2(n0 * n1) * 2.0**-24
    assert np.linalg.norm(fwd - ref) / np.linalg.norm(ref) < bound
    rt = oracle.mxfft2d(x, "fp32", 32, op="roundtrip")[0].astype(np.complex128)
    assert np.linalg.norm(rt - xd) / np.linalg.norm(xd) < 2 * bound
    rtf = oracle.mxfft2d(x, "fp32", 32, op="roundtrip_fused")[0].astype(np.complex128)
    assert np.linalg.norm(rtf - xd) / np.linalg.norm(xd) < 2 * bound


def test_is_the_floor_of_the_mx_error():
    x = phantom.mri_batch(64, 64, 2, 1, config_id=94)
    ref = np.fft.fft2(x.astype(np.complex128))
    err = {}
    for fmt in ("fp32", "fp16", "e4m3"):
        y = oracle.mxfft2d(x, fmt, 32)[0].astype(np.complex128)
        err[fmt] = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err["fp32"] < 1e-6 < err["fp16"] < err["e4m3"], err
