"""Pins of the oracle's FP16 positive control (Sec. 2.2): its binary16
rounding against numpy's IEEE conversion, the whole transform against an
independent emulation on small sizes bit for bit, closed forms, and its role
as a positive control (far more accurate than MXFP8 on the phantom)."""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

from bruteforce_fp16 import mxfft2d_fp16


def test_binary16_rounding_matches_ieee_conversion():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200000) * 2.0 ** rng.uniform(-30, 18, 200000)).astype(np.float32)
    ties = (np.arange(-3000, 3000) + 0.5).astype(np.float32) * np.float32(2.0 ** -24)   # subnormal ties
    big = np.array([65504, 65519.99, 65520, 65536, 1e30, -65520, 3.4e38], np.float32)
    for v in (x, ties, big, np.array([0.0, -0.0, np.inf, -np.inf], np.float32)):
        got = oracle.quantize(v, "fp16")
        with np.errstate(over="ignore"):
            want = v.astype(np.float16).astype(np.float32)
        np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    d = rng.standard_normal(100000) * 2.0 ** rng.uniform(-30, 18, 100000)
    with np.errstate(over="ignore"):
        want = d.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(oracle.quantize(d, "fp16"), want)


@pytest.mark.parametrize("n0,n1", [(2, 2), (4, 8), (8, 4), (16, 16)])
@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip"])
def test_transform_equals_independent_emulation(n0, n1, op):
    x = phantom.random_complex((3, n0, n1), seed=n0 * 100 + n1, scale=7.0)
    got, ks, _ = oracle.mxfft2d(x, "fp16", 32, op=op)
    for s in range(3):
        k = int(ks[s][0] if op == "roundtrip" else ks[s])
        kinv = int(ks[s][1]) if op == "roundtrip" else None
        want = mxfft2d_fp16(x[s], k, op, kinv)
        np.testing.assert_array_equal(got[s].view(np.uint32), want.view(np.uint32))


def test_closed_forms():
    # delta: every output equals the value; constant: n0 n1 c at DC, exact zeros elsewhere
    x = np.zeros((1, 16, 8), np.complex64)
    x[0, 0, 0] = 3.0 - 1.5j
    y, _, _ = oracle.mxfft2d(x, "fp16", 32)
    assert np.all(y == np.complex64(3.0 - 1.5j))
    c = np.full((1, 16, 8), 0.75 + 0.25j, np.complex64)
    y, _, _ = oracle.mxfft2d(c, "fp16", 32)
    want = np.zeros_like(c)
    want[0, 0, 0] = 128 * (0.75 + 0.25j)
    np.testing.assert_array_equal(y, want)


def test_positive_control_accuracy():
    # at 256 x 256 with the default tail floor no stage value can overflow
    ksp = phantom.mri_batch(256, 256, 2, 1, config_id=1)
    ref = np.fft.fft2(ksp.astype(np.complex128))
    def nrmse(a):
        return np.linalg.norm(a - ref) / np.linalg.norm(ref)
    e16 = nrmse(oracle.mxfft2d(ksp, "fp16", 32)[0])
    e8 = nrmse(oracle.mxfft2d(ksp, "e4m3", 32)[0])
    assert e16 < 0.01 and e16 < e8 / 20


def test_fp16_twiddles_are_far_from_rounding_ties():
    # as for the MX formats: no twiddle cos / sin(pi j / h), h <= 1024, lies near
    # a binary16 rounding midpoint, so any accurate FP64 source rounds them alike
    worst = 1.0
    for h in (2 ** p for p in range(1, 11)):
        ang = np.pi * np.arange(h) / h
        for t in np.abs(np.concatenate([np.cos(ang), np.sin(ang)])):
            if t == 0 or t == 1 or t == 0.5:
                continue
            E = max(int(np.floor(np.log2(t))), -14)
            q = 2.0 ** (E - 10)
            frac = t / q - np.floor(t / q)
            if frac == 0:
                continue
            worst = min(worst, abs(frac - 0.5))
    assert worst > 1e-9, worst


def test_default_prescale_keeps_binary16_in_range():
    # tau_min = 2^-24: k = k1, the peak lands on the target 0.5, and every
    # output of a 256 x 256 forward stays finite
    ksp = phantom.mri_batch(256, 256, 3, 2, config_id=2)
    y, ks, _ = oracle.mxfft2d(ksp, "fp16", 32)
    assert np.isfinite(y).all()
    for s in range(ksp.shape[0]):
        peak = np.abs(ksp[s]).max()
        assert 0.25 < peak * 2.0 ** int(ks[s]) <= 0.5 * 2 ** 0.5
