"""Pins for the oracle's Alg. 1 (global power-of-two prescale, Sec. 2.1) and for
its magnitude |x| (reading C3), using hand-computed cases and the exact-rational
model."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import bruteforce_mx as bf  # noqa: E402
from fractions import Fraction as Fr  # noqa: E402


def test_hand_case_peak_three():
    # a_max = 3: k1 = round(log2(0.5 / 3)) = round(-2.585) = -3;
    # p_tau = 3: k2 = ceil(log2(2^-10 / 3)) = ceil(-11.585) = -11; k = -3
    x = np.zeros((4, 4), np.complex64)
    x[1, 2] = 3
    assert oracle.prescale_k(x, "e4m3") == (-3, False)


def test_hand_case_tail_dominates():
    # 1000 magnitudes 2^-20 and one 1: n_nz = 1001, rank floor(1e-3 * 1000) = 1
    # picks 2^-20, so k2 = ceil(log2(2^-10 / 2^-20)) = 10 > k1 = -1
    x = np.full(1001, 2.0 ** -20, np.complex64)
    x[0] = 1
    assert oracle.prescale_k(x, "e4m3") == (10, False)
    # e5m2's floor 2^-12 gives 8
    assert oracle.prescale_k(x, "e5m2") == (8, False)
    # with tau = 0.5 the median 2^-20 still rules; k_max clips it
    assert oracle.prescale_k(x, "e4m3", tau=0.5, kmax=4) == (4, False)


def test_hand_case_rounding_of_k1_at_sqrt2():
    # round(log2(0.5 / a)) flips where a's significand crosses sqrt(2):
    # sqrt(2) * 2^23 = 11863283.2, so significands 11863283 and 11863284 sit on
    # either side of it
    lo = np.float32(11863283 * 2.0 ** -23)   # just below sqrt(2): log2 a = 0.4999999753
    hi = np.float32(11863284 * 2.0 ** -23)   # just above: log2 a = 0.5000000969
    kl, _ = oracle.prescale_k(np.array([lo], np.complex64), "e4m3", tau_min=2.0 ** -40)
    kh, _ = oracle.prescale_k(np.array([hi], np.complex64), "e4m3", tau_min=2.0 ** -40)
    assert (kl, kh) == (-1, -2)


def test_hand_case_epsilon_floor():
    # a_max below 1e-30: max(a_max, 1e-30) = 1e-30 and log2(1e-30) = -99.658,
    # so k1 = round(-1 + 99.658) = 99 and k2 = ceil(-10 + 99.658) = 90
    x = np.full(16, 1e-40, np.complex64)
    assert oracle.prescale_k(x, "e4m3") == (99, False)
    assert oracle.prescale_k(x, "e4m3", kmax=126) == (99, False)
    assert oracle.prescale_k(x, "e4m3", kmax=50) == (50, False)


def test_zero_and_nonfinite():
    assert oracle.prescale_k(np.zeros(64, np.complex64), "e4m3") == (0, False)
    x = np.ones(64, np.complex64)
    x[5] = complex(np.inf, 0)
    assert oracle.prescale_k(x, "e4m3") == (0, True)
    x[5] = complex(0, np.nan)
    assert oracle.prescale_k(x, "e4m3") == (0, True)


def test_percentile_is_lower_order_statistic():
    # magnitudes 1..1000 (exact integers): tau = 0.25 gives rank
    # floor(0.25 * 999) = 249 -> p = 250, k2 = ceil(log2(2^-10/250)) = -17
    # while k1 = round(log2(0.5/1000)) = -11; choose tau_min so k2 rules
    x = np.arange(1, 1001).astype(np.complex64)
    rng = np.random.default_rng(0)
    rng.shuffle(x)
    # tau_min = 2^-2: k2 = ceil(log2(0.25/250)) = ceil(-9.97) = -9 > -11
    assert oracle.prescale_k(x, "e4m3", tau=0.25, tau_min=0.25) == (-9, False)
    # p = 250 for tau = 0.25; p = 251 would give the same k, so also check a
    # boundary: tau = 255/999 -> rank 255 -> p = 256 = 2^8 exactly,
    # k2 = ceil(log2(2^-2 / 2^8)) = -10 (exact power of two)
    assert oracle.prescale_k(x, "e4m3", tau=np.float32(255 / 999) + np.float32(1e-7),
                             tau_min=0.25) == (-10, False)


def test_magnitude_matches_exact_model():
    rng = np.random.default_rng(9)
    re = (rng.standard_normal(300) * np.exp2(rng.uniform(-140, 120, 300))).astype(np.float32)
    im = (rng.standard_normal(300) * np.exp2(rng.uniform(-140, 120, 300))).astype(np.float32)
    re[:20] = 0
    im[20:40] = 0
    x = (re + 1j * im).astype(np.complex64)
    got = oracle.magnitude(x)
    for g, a, b in zip(got, re, im):
        assert Fr(float(g)) == bf.magnitude(Fr(float(a)), Fr(float(b)))


def test_magnitude_close_to_hypot():
    x = phantom.random_complex(5000, seed=4, scale=1e3)
    m = oracle.magnitude(x).astype(np.float64)
    ref = np.abs(x.astype(np.complex128))
    assert np.max(np.abs(m - ref) / ref) < 2 * 2.0 ** -24


@pytest.mark.parametrize("seed", range(6))
def test_prescale_matches_exact_model(seed):
    rng = np.random.default_rng(100 + seed)
    shape = (8, 8)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.exp2(
        rng.uniform(-60, 60, shape))
    x[rng.random(shape) < 0.3] = 0
    x = x.astype(np.complex64)
    for fmt in ("e4m3", "e5m2"):
        for tau in (1e-3, 0.3, 0.9):
            k, _ = oracle.prescale_k(x, fmt, tau=tau)
            S = [[(Fr(float(z.real)), Fr(float(z.imag))) for z in row] for row in x]
            tmin = Fr(1, 4096) if fmt == "e5m2" else Fr(1, 1024)
            kb = bf.prescale_k(S, Fr(float(np.float32(tau))), Fr(1, 2), tmin)
            assert k == kb
