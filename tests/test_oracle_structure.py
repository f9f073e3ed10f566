"""Pins for the oracle's dataflow (bit reversal, stage indexing, twiddles,
row/column order, inverse, 1/(n0 n1) of the round trip; Eq. 1, Fig. 1B).

The FP64 mode runs the same loops as the MX mode with the quantisation removed,
so it must reproduce the discrete Fourier transform: a direct O(n^2) DFT written
from its definition, numpy's FFT, Parseval and linearity.
"""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom


def direct_dft2(x, sign=-1):
    n0, n1 = x.shape[-2:]
    F0 = np.exp(sign * 2j * np.pi * np.outer(np.arange(n0), np.arange(n0)) / n0)
    F1 = np.exp(sign * 2j * np.pi * np.outer(np.arange(n1), np.arange(n1)) / n1)
    return F0 @ x @ F1.T


SIZES_SMALL = [(2, 2), (2, 8), (4, 4), (8, 2), (8, 16), (16, 16), (32, 4), (32, 32)]


@pytest.mark.parametrize("n0,n1", SIZES_SMALL)
def test_exact_mode_equals_direct_dft(n0, n1):
    x = phantom.random_complex((n0, n1), seed=n0 * 31 + n1).astype(np.complex128)
    f = oracle.fft2d_exact(x, "forward")
    assert np.abs(f - direct_dft2(x)).max() <= 1e-13 * np.abs(x).sum()
    i = oracle.fft2d_exact(x, "inverse")
    assert np.abs(i - direct_dft2(x, +1)).max() <= 1e-13 * np.abs(x).sum()


@pytest.mark.parametrize("n0,n1", [(64, 64), (128, 32), (256, 256), (2048, 4), (4, 2048),
                                   (512, 512)])
def test_exact_mode_equals_numpy_fft(n0, n1):
    x = phantom.random_complex((2, n0, n1), seed=n0 + 7 * n1).astype(np.complex128)
    f = oracle.fft2d_exact(x, "forward")
    ref = np.fft.fft2(x)
    assert np.abs(f - ref).max() / np.abs(ref).max() < 1e-12
    inv = oracle.fft2d_exact(x, "inverse")
    ref_i = np.fft.ifft2(x) * (n0 * n1)
    assert np.abs(inv - ref_i).max() / np.abs(ref_i).max() < 1e-12
    rt = oracle.fft2d_exact(x, "roundtrip")
    assert np.abs(rt - x).max() / np.abs(x).max() < 1e-13


def test_exact_mode_parseval_and_linearity():
    n0, n1 = 64, 128
    x = phantom.random_complex((n0, n1), seed=11).astype(np.complex128)
    y = phantom.random_complex((n0, n1), seed=12).astype(np.complex128)
    fx, fy = oracle.fft2d_exact(x), oracle.fft2d_exact(y)
    assert abs(np.sum(np.abs(fx) ** 2) / (n0 * n1) - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    a, b = 0.75 - 2j, 3 + 0.5j
    fxy = oracle.fft2d_exact(a * x + b * y)
    assert np.abs(fxy - (a * fx + b * fy)).max() < 1e-11 * np.abs(fxy).max()


def test_exact_mode_delta_and_constant_closed_forms():
    n0, n1 = 16, 32
    d = np.zeros((n0, n1), np.complex128)
    d[0, 0] = 2 - 1j
    assert np.allclose(oracle.fft2d_exact(d), 2 - 1j, atol=0, rtol=1e-15)
    c = np.full((n0, n1), 0.5 + 0.25j)
    f = oracle.fft2d_exact(c)
    want = np.zeros_like(c)
    want[0, 0] = n0 * n1 * (0.5 + 0.25j)
    assert np.abs(f - want).max() < 1e-12


def test_exact_mode_row_then_column_axis_convention():
    # a signal varying along n1 only must land on row 0 of the spectrum
    n0, n1 = 8, 16
    x = np.tile(np.exp(2j * np.pi * 3 * np.arange(n1) / n1), (n0, 1))
    f = oracle.fft2d_exact(x)
    want = np.zeros((n0, n1), complex)
    want[0, 3] = n0 * n1
    assert np.abs(f - want).max() < 1e-11
