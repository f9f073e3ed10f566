"""Pins for the oracle's MX arithmetic (Alg. 1, Alg. 2, Eq. 1).

* a hand-traced 2x2 example (tests/golden/mx_2x2_e4m3_k2.txt);
* an exact-rational brute-force model (tests/bruteforce_mx.py) on every
  format, block size and operation for n0, n1 <= 8;
* closed forms that hold bit for bit under MX: a delta, a representable
  constant, zero;
* invariances: power-of-two scaling, multiplication by i, conjugation between
  forward and inverse, the renormalisation of Alg. 2 being a no-op;
* the accuracy trends the paper reports (Sec. 3, 4.1, 4.2).
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
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def nrmse(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def test_golden_hand_traced_2x2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "mx_2x2_e4m3_k2.txt"))
            if l.strip() and not l.startswith("#")]
    x = np.zeros((2, 2), np.complex64)
    want = np.zeros((2, 2), np.complex64)
    for r, c, xr, xi, yr, yi in rows:
        x[int(r), int(c)] = complex(float(xr), float(xi))
        want[int(r), int(c)] = complex(float(yr), float(yi))
    out, k, _ = oracle.mxfft2d(x[None], "e4m3", 2)
    assert k.tolist() == [-1]
    assert np.array_equal(out[0], want)


@pytest.mark.parametrize("n0,n1", [(2, 2), (2, 8), (4, 4), (8, 2), (8, 8)])
@pytest.mark.parametrize("fmt", FMTS)
def test_bruteforce_exact_model(n0, n1, fmt):
    for kblk in (2, 4, 8, 16):
        for op in ("forward", "inverse", "roundtrip"):
            x = phantom.random_complex((n0, n1), seed=1000 * n0 + 10 * n1 + kblk)
            got, kg, _ = oracle.mxfft2d(x[None], fmt, kblk, op=op)
            want, kw = bf.mxfft2d(x, fmt, kblk, op=op)
            assert np.array_equal(got[0].astype(np.complex128), want), (fmt, kblk, op)
            assert (kg[0].tolist() if op == "roundtrip" else int(kg[0])) == (
                list(kw) if op == "roundtrip" else kw)


def test_bruteforce_exact_model_wide_range():
    # values spanning many binades, so blocks carry elements in the element
    # format's subnormal range and some underflow to zero
    rng = np.random.default_rng(5)
    for fmt in FMTS:
        x = (rng.standard_normal((4, 8)) * np.exp2(rng.uniform(-30, 10, (4, 8)))
             + 1j * rng.standard_normal((4, 8)) * np.exp2(rng.uniform(-30, 10, (4, 8))))
        x = x.astype(np.complex64)
        got, _, _ = oracle.mxfft2d(x[None], fmt, 8)
        want, _ = bf.mxfft2d(x, fmt, 8)
        assert np.array_equal(got[0].astype(np.complex128), want), fmt


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("kblk", [2, 8, 32, 128])
def test_closed_form_delta(fmt, kblk):
    # a delta at the origin: every v block is zero, so u passes unchanged and
    # every output equals the delta's value, bit for bit
    for a in (1 + 0j, 2.5 - 0.375j, 3.0e-20 + 1.0e-21j, -7.0e12 + 1j):
        x = np.zeros((1, 16, 32), np.complex64)
        x[0, 0, 0] = a
        out, _, _ = oracle.mxfft2d(x, fmt, kblk)
        assert np.array_equal(out[0], np.full((16, 32), np.complex64(a)))


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("kblk", [2, 4, 16, 64])
def test_closed_form_constant(fmt, kblk):
    # a constant whose components are exact in the element format: every
    # butterfly's v block holds the running constant (exact) or zeros, every
    # twiddle that meets a nonzero v is 1, so the spectrum is n0 n1 c at the
    # origin and zero elsewhere
    n0, n1 = 32, 16
    c = np.complex64(1.5 + 0.75j)       # 1.1b and 1.1b * 2^-1: two significant bits
    x = np.full((1, n0, n1), c)
    out, _, _ = oracle.mxfft2d(x, fmt, kblk)
    want = np.zeros((n0, n1), np.complex64)
    want[0, 0] = n0 * n1 * c
    assert np.array_equal(out[0], want)


@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip"])
def test_closed_form_zero(op):
    x = np.zeros((2, 8, 16), np.complex64)
    out, k, flags = oracle.mxfft2d(x, "e4m3", 32, op=op)
    assert np.array_equal(out, x) and not np.signbit(out.real).any()
    assert (np.asarray(k) == 0).all() and not flags.any()


@pytest.mark.parametrize("fmt", FMTS)
def test_invariance_power_of_two_scaling(fmt):
    # with the prescale pinned to k = 0 the MX blocks still rescale themselves,
    # so MXFFT(2^j x) = 2^j MXFFT(x) away from the range edges
    x = phantom.random_complex((2, 32, 64), seed=21)
    base, _, _ = oracle.mxfft2d(x, fmt, 32, kmin=0, kmax=0)
    for j in (-9, 3, 17):
        s = np.float32(2.0 ** j)
        out, _, _ = oracle.mxfft2d(x * s, fmt, 32, kmin=0, kmax=0)
        assert np.array_equal(out, base * s)
    # and the computed prescale gives the same bits as k = 0 here
    out, k, _ = oracle.mxfft2d(x, fmt, 32)
    assert (k != 0).all() and np.array_equal(out, base)


@pytest.mark.parametrize("fmt", FMTS)
def test_invariance_multiply_by_i(fmt):
    # joint re/im block maximum and sign-symmetric rounding: MXFFT(i x) = i MXFFT(x)
    x = phantom.random_complex((2, 16, 32), seed=22)
    a, _, _ = oracle.mxfft2d(x, fmt, 16)
    b, _, _ = oracle.mxfft2d((1j * x).astype(np.complex64), fmt, 16)
    assert np.array_equal(b, (1j * a).astype(np.complex64))


@pytest.mark.parametrize("fmt", FMTS)
def test_invariance_conjugation(fmt):
    # the inverse uses conjugate twiddles: MXiFFT(conj x) = conj(MXFFT(x))
    x = phantom.random_complex((2, 32, 16), seed=23)
    a, _, _ = oracle.mxfft2d(x, fmt, 32)
    b, _, _ = oracle.mxfft2d(np.conj(x), fmt, 32, op="inverse")
    assert np.array_equal(b, np.conj(a))


@pytest.mark.parametrize("fmt", FMTS)
def test_renormalisation_is_a_noop_under_fresh_encode(fmt):
    x = phantom.mri_batch(32, 64, 2, 1, config_id=3)
    a, _, _ = oracle.mxfft2d(x, fmt, 32, renorm=True)
    b, _, _ = oracle.mxfft2d(x, fmt, 32, renorm=False)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_twiddles_are_far_from_rounding_ties():
    # cos/sin(pi j / h) are irrational except at 0, 1/2, 1, so no FP64 rounding
    # of a twiddle can move it across an element-grid midpoint; check the margin
    for fmt in FMTS:
        emax, emin, mbits, maxn = oracle.format_info(fmt)
        worst = 1.0
        for h in (2 ** p for p in range(1, 11)):
            ang = np.pi * np.arange(h) / h
            for v in np.abs(np.concatenate([np.cos(ang), np.sin(ang)])):
                for sw in (-emax, -emax - 1):
                    t = v * 2.0 ** -sw
                    if t == 0 or t >= maxn or t == round(t):
                        continue
                    E = max(int(np.floor(np.log2(t))), emin)
                    q = 2.0 ** (E - mbits)
                    frac = t / q - np.floor(t / q)
                    if abs(frac - 0.5) < 1e-15 or frac == 0:
                        continue   # exact values (1/2, dyadics) are not perturbed
                    worst = min(worst, abs(frac - 0.5))
        assert worst > 1e-9, (fmt, worst)


def test_paper_trends_on_phantom():
    # Sec. 3 and 4: e4m3 beats e5m2, e2m3 tracks e4m3, B = 2 is worst,
    # and the round trip loses more than the forward transform
    x = phantom.mri_batch(64, 64, 2, 1, config_id=1)
    ref = np.fft.fft2(x.astype(np.complex128))
    e = {(f, k): nrmse(oracle.mxfft2d(x, f, k)[0], ref)
         for f in ("e4m3", "e5m2", "e2m3") for k in (2, 8, 32)}
    for k in (2, 8, 32):
        assert e["e4m3", k] < e["e5m2", k]
        assert e["e2m3", k] < 1.5 * e["e4m3", k]
    for f in ("e4m3", "e5m2"):
        assert e[f, 2] > e[f, 8] and e[f, 2] > e[f, 32]
    img = phantom.mri_batch(64, 64, 2, 1, config_id=1, domain="image")
    rt = nrmse(oracle.mxfft2d(img, "e4m3", 32, op="roundtrip")[0], img)
    fw = nrmse(oracle.mxfft2d(img, "e4m3", 32)[0], np.fft.fft2(img.astype(np.complex128)))
    assert rt > fw
    # quantisation is real but bounded
    assert 0.01 < e["e4m3", 32] < 0.3


def test_direct_encode_reading_differs_but_is_close():
    x = phantom.mri_batch(32, 32, 1, 1, config_id=4)
    ref = np.fft.fft2(x.astype(np.complex128))
    a = nrmse(oracle.mxfft2d(x, "e4m3", 32)[0], ref)
    b = nrmse(oracle.mxfft2d(x, "e4m3", 32, direct_enc=True)[0], ref)
    assert a != b and abs(a - b) < 0.5 * a


def test_nonfinite_flag_and_k_zero():
    x = phantom.random_complex((3, 8, 8), seed=2)
    x[1, 3, 4] = np.nan
    x[2, 0, 0] = np.float32(3e38) * (1 + 1j)   # finite input, |x| overflows
    _, k, flags = oracle.mxfft2d(x, "e4m3", 8)
    assert flags.tolist() == [0, 1, 1]
    assert k[1] == 0 and k[2] == 0 and k[0] != 0


def test_nonfinite_block_decodes_to_nan():
    # OCP MX: a block holding Inf/NaN has a NaN shared scale; every element of
    # the block decodes to NaN, so both butterfly outputs are NaN for that block
    u = np.array([1 + 1j, 2 - 1j], np.complex64)
    v = np.array([np.inf + 0j, 0.5 + 0.25j], np.complex64)
    w = np.array([1.0, np.exp(-0.25j * np.pi)])
    y0, y1 = oracle.butterfly_block(u, v, w, "e4m3")
    assert np.isnan(y0.real).all() and np.isnan(y1.imag).all()
    # a finite block next to it is untouched
    y0f, _ = oracle.butterfly_block(u, np.array([1 + 0j, 0.5 + 0.25j], np.complex64), w, "e4m3")
    assert np.isfinite(y0f).all()
    # a prescale that overflows the peak (k2 ruled by a 1e-45 tail) yields
    # non-finite outputs without the non-finite input flag
    x = np.full((1, 8, 8), 1e-45, np.complex64)
    x[0, 0, 0] = 1e36
    out, k, flags = oracle.mxfft2d(x, "e4m3", 8)
    assert k[0] == 90 and flags[0] == 0 and not np.isfinite(out).all()
