"""Pins for the fused round trip of Sec. 4.3 (encode -> F -> F^-1 -> decode),
the declared variant of reading C17: one prescale of the input, the forward
transform (rows, then columns), the inverse applied to the forward result
without unscale or second prescale (columns, then rows), one decode by
2^(-k - log2(n0 n1)).

* the exact-rational brute-force model (tests/bruteforce_mx.py) on every
  format and block size for n0, n1 <= 8;
* the FP64 dataflow of the variant against numpy's ifft2(fft2(x));
* closed forms: a delta comes back bit for bit, zero stays zero;
* its relation to the separate transforms: the forward result re-scaled by
  2^k, then the inverse with its prescale pinned to k = 0 along the transposed
  axes, decoded by 2^(-k - log2(n0 n1));
* invariances under power-of-two scaling and multiplication by i;
* accuracy on the phantom beside the separate round trip.
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import bruteforce_mx as bf  # noqa: E402

FMTS = ["e4m3", "e5m2", "e2m3", "e3m2", "e2m1"]


def nrmse(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n0,n1", [(2, 2), (2, 8), (4, 4), (8, 2), (8, 8)])
@pytest.mark.parametrize("fmt", FMTS)
def test_bruteforce_exact_model(n0, n1, fmt):
    for kblk in (2, 4, 8, 16):
        x = phantom.random_complex((n0, n1), seed=7000 * n0 + 10 * n1 + kblk)
        got, kg, _ = oracle.mxfft2d(x[None], fmt, kblk, op="roundtrip_fused")
        want, kw = bf.mxfft2d(x, fmt, kblk, op="roundtrip_fused")
        assert np.array_equal(got[0].astype(np.complex128), want), (fmt, kblk)
        assert int(kg[0]) == kw


@pytest.mark.parametrize("n0,n1", [(4, 8), (64, 32), (256, 128)])
def test_exact_mode_is_the_identity(n0, n1):
    x = phantom.random_complex((2, n0, n1), seed=n0 + n1).astype(np.complex128)
    got = oracle.fft2d_exact(x, op="roundtrip_fused")
    np.testing.assert_allclose(got, np.fft.ifft2(np.fft.fft2(x)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("kblk", [2, 8, 32, 128])
def test_closed_form_delta(fmt, kblk):
    # F of a delta is the constant 2^k a (no v block is ever nonzero); the
    # inverse of that constant meets only unit twiddles and exactly
    # representable blocks, so n0 n1 2^k a lands at the origin and the decode
    # returns a, bit for bit
    for a in (1 + 0j, 1.5 + 0.75j, -3.0 + 0.5j):
        x = np.zeros((1, 16, 32), np.complex64)
        x[0, 0, 0] = a
        out, _, _ = oracle.mxfft2d(x, fmt, kblk, op="roundtrip_fused")
        assert np.array_equal(out, x), (fmt, kblk, a)


def test_closed_form_zero():
    x = np.zeros((2, 8, 16), np.complex64)
    out, k, flags = oracle.mxfft2d(x, "e4m3", 32, op="roundtrip_fused")
    assert np.array_equal(out, x) and not np.signbit(out.real).any()
    assert (k == 0).all() and not flags.any()


@pytest.mark.parametrize("fmt", ["e4m3", "e5m2", "e2m1"])
@pytest.mark.parametrize("kblk", [8, 32])
def test_composition_of_the_separate_transforms(fmt, kblk):
    # non-square slices, so a wrong axis order or transposition fails
    x = phantom.mri_batch(64, 32, 2, 1, config_id=3, domain="image")
    fused, kf, _ = oracle.mxfft2d(x, fmt, kblk, op="roundtrip_fused")
    fwd, k, _ = oracle.mxfft2d(x, fmt, kblk)
    assert np.array_equal(kf, k)
    lg = 6 + 5
    for s in range(x.shape[0]):
        A = np.ldexp(fwd[s].real, k[s]) + 1j * np.ldexp(fwd[s].imag, k[s])
        A = A.astype(np.complex64)
        # the inverse, columns first = the library's rows-first inverse on the
        # transposed slice; its prescale pinned to 2^0
        z, kz, _ = oracle.mxfft2d(np.ascontiguousarray(A.T)[None], fmt, kblk, op="inverse",
                                  kmin=0, kmax=0)
        assert int(kz[0]) == 0
        z = z[0].T
        want = (np.ldexp(z.real, -int(k[s]) - lg) + 1j * np.ldexp(z.imag, -int(k[s]) - lg))
        assert np.array_equal(fused[s], want.astype(np.complex64)), (fmt, kblk, s)


@pytest.mark.parametrize("fmt", ["e4m3", "e3m2"])
def test_invariances(fmt):
    x = phantom.random_complex((2, 32, 64), seed=31)
    base, k0, _ = oracle.mxfft2d(x, fmt, 32, op="roundtrip_fused")
    for j in (-7, 5):
        s = np.float32(2.0 ** j)
        out, k, _ = oracle.mxfft2d(x * s, fmt, 32, op="roundtrip_fused")
        assert np.array_equal(k, k0 - j)
        assert np.array_equal(out, base * s)
    b, _, _ = oracle.mxfft2d((1j * x).astype(np.complex64), fmt, 32, op="roundtrip_fused")
    assert np.array_equal(b, (1j * base).astype(np.complex64))


def test_accuracy_beside_the_separate_round_trip():
    img = phantom.mri_batch(128, 128, 2, 2, config_id=1, domain="image")
    for fmt in ("e4m3", "e5m2"):
        sep = nrmse(oracle.mxfft2d(img, fmt, 32, op="roundtrip")[0], img)
        fus = nrmse(oracle.mxfft2d(img, fmt, 32, op="roundtrip_fused")[0], img)
        # the same MX blocks in another inverse axis order: the same error
        # level, not a different method
        assert 0.8 * sep < fus < 1.25 * sep, (fmt, sep, fus)
    fw = nrmse(oracle.mxfft2d(img, "e4m3", 32)[0], np.fft.fft2(img.astype(np.complex128)))
    assert fus > fw


def test_fp16_control_rejects_the_variant():
    x = np.zeros((1, 8, 8), np.complex64)
    with pytest.raises(ValueError):
        oracle.mxfft2d(x, "fp16", 32, op="roundtrip_fused")
