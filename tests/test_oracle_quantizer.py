"""Pins for the oracle's element quantiser (EncodeBlockMX's rounding, Sec. 2.2).

The code tables are rebuilt here from the OCP bit layouts (sign, exponent field,
mantissa field, bias, reserved NaN/Inf codes) and the expected result of
rounding is found by brute force: the nearest table value, a tie going to the
code whose mantissa field is even, values beyond the largest normal saturating.
"""
import numpy as np
import pytest

import oracle

# (exponent bits, mantissa bits, bias, reserved-code predicate)
LAYOUT = {
    "e4m3": (4, 3, 7, lambda E, M: E == 15 and M == 7),      # S.1111.111 is NaN
    "e5m2": (5, 2, 15, lambda E, M: E == 31),                  # Inf / NaN
    "e2m3": (2, 3, 1, lambda E, M: False),
    "e3m2": (3, 2, 3, lambda E, M: False),
    "e2m1": (2, 1, 1, lambda E, M: False),
}


def code_table(fmt):
    """Nonnegative finite values and the parity of their mantissa field."""
    eb, mb, bias, reserved = LAYOUT[fmt]
    vals, even = [], []
    for E in range(2 ** eb):
        for M in range(2 ** mb):
            if reserved(E, M):
                continue
            if E == 0:
                v = (M / 2 ** mb) * 2.0 ** (1 - bias)
            else:
                v = (1 + M / 2 ** mb) * 2.0 ** (E - bias)
            vals.append(v)
            even.append(M % 2 == 0)
    order = np.argsort(vals)
    return np.array(vals)[order], np.array(even)[order]


def brute_quantize(x, fmt):
    vals, even = code_table(fmt)
    out = np.empty_like(x, dtype=np.float64)
    for i, xv in enumerate(np.asarray(x, np.float64)):
        a = abs(xv)
        if a >= vals[-1]:
            r = vals[-1]
        else:
            j = np.searchsorted(vals, a)            # vals[j-1] < a <= vals[j]
            lo, hi = vals[j - 1], vals[j]
            if a == hi:
                r = hi
            elif a - lo < hi - a:
                r = lo
            elif a - lo > hi - a:
                r = hi
            else:
                r = lo if even[j - 1] else hi
        out[i] = np.copysign(r, xv)
    return out


@pytest.mark.parametrize("fmt", list(LAYOUT))
def test_format_constants_match_bit_layout(fmt):
    vals, _ = code_table(fmt)
    emax, emin, mbits, maxnorm = oracle.format_info(fmt)
    assert maxnorm == vals[-1]
    assert mbits == LAYOUT[fmt][1]
    assert emin == 1 - LAYOUT[fmt][2]
    assert 2.0 ** emax <= maxnorm < 2.0 ** (emax + 1)
    # the smallest subnormal is 2^(emin - mbits)
    assert vals[1] == 2.0 ** (emin - mbits)


@pytest.mark.parametrize("fmt", list(LAYOUT))
def test_quantizer_matches_nearest_code(fmt):
    vals, _ = code_table(fmt)
    rng = np.random.default_rng(7)
    mids = (vals[1:] + vals[:-1]) / 2                       # exact ties
    probes = np.concatenate([
        vals, mids,
        np.nextafter(mids.astype(np.float32), np.float32(np.inf)),
        np.nextafter(mids.astype(np.float32), np.float32(-np.inf)),
        vals[-1] * np.array([1.0001, 1.07, 1.14, 1.5, 1.99]),
        rng.uniform(0, vals[-1] * 1.1, 4000),
        np.exp2(rng.uniform(np.log2(vals[1]) - 8, np.log2(vals[-1]) + 1, 4000)),
        [1e-30, 1e-45, 0.0],
    ]).astype(np.float32)
    probes = np.concatenate([probes, -probes])
    got = oracle.quantize(probes, fmt).astype(np.float64)
    want = brute_quantize(probes, fmt)
    assert np.array_equal(got, want)
    # sign of zero is kept
    assert np.array_equal(np.signbit(got), np.signbit(want))


def test_quantizer_hand_cases_e4m3():
    # e4m3 around 448: spacing 32 in [256, 512); 464 is the 448/480 tie and 480
    # is not a code (S.1111.111 is NaN), so everything above 448 saturates.
    x = np.array([464, 470, 480, 500, 1e6, 447, 433, 432, 431, 0.0029296875, 0.0009765625,
                  0.001953125 * 0.75, -0.0], np.float32)
    # 432 = 13.5 * 32 is a tie between 416 (odd mantissa 101) and 448 (110);
    # 3 * 2^-10 = 1.5 * 2^-9 is a subnormal tie between codes 1 and 2.
    want = [448, 448, 448, 448, 448, 448, 448, 448, 416, 0.00390625, 0.0,
            0.001953125, -0.0]
    got = oracle.quantize(x, "e4m3")
    assert got.tolist() == want
    assert np.signbit(got[-1])


def test_quantizer_f64_agrees_with_f32_on_f32_values():
    x = np.random.default_rng(3).standard_normal(2000).astype(np.float32) * 100
    for fmt in LAYOUT:
        a = oracle.quantize(x, fmt).astype(np.float64)
        b = oracle.quantize(x.astype(np.float64), fmt)
        assert np.array_equal(a, b)
