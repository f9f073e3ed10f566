"""Pins of the oracle's root-sum-of-squares coil combine (Eq. (1)):
closed forms with exact answers, the correctly rounded square root of a
square, and the FP64 value within the error bound of C + 2 FP32 roundings."""
import numpy as np

import oracle


def test_pythagorean_closed_forms():
    # one coil (3 + 4i) -> 5; two coils 3 and 4i -> 5; (5, 12) -> 13; zeros -> 0
    z = np.array([[3 + 4j], [5 + 12j], [0j]], np.complex64).reshape(3, 1, 1)
    np.testing.assert_array_equal(oracle.rss(z, 1).ravel(), [5.0, 13.0, 0.0])
    z2 = np.array([3 + 0j, 4j, 5 + 0j, 12j], np.complex64).reshape(4, 1, 1)
    np.testing.assert_array_equal(oracle.rss(z2, 2).ravel(), [5.0, 13.0])
    # three coils: 2, 3, 6 -> 7; 1, 4, 8 -> 9
    z3 = np.array([2, 3j, 6, 1, 4, 8j], np.complex64).reshape(6, 1, 1)
    np.testing.assert_array_equal(oracle.rss(z3, 3).ravel(), [7.0, 9.0])


def test_single_coil_real_is_absolute_value():
    # sqrt of the correctly rounded square of a float is the float's magnitude
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(4096) * 10.0 ** rng.uniform(-15, 15, 4096)).astype(np.float32)
    z = x.astype(np.complex64).reshape(1, 64, 64)
    np.testing.assert_array_equal(oracle.rss(z, 1).ravel(), np.abs(x))


def test_within_the_fp32_error_bound_of_fp64():
    rng = np.random.default_rng(4)
    for coils in (1, 4, 16):
        z = (rng.standard_normal((3 * coils, 32, 32)) + 1j * rng.standard_normal((3 * coils, 32, 32)))
        z = z.astype(np.complex64)
        got = oracle.rss(z, coils).astype(np.float64)
        zz = z.astype(np.complex128).reshape(3, coils, 32, 32)
        want = np.sqrt((np.abs(zz) ** 2).sum(axis=1))
        bound = (coils + 3) * 2.0 ** -24
        assert np.all(np.abs(got - want) <= bound * want + 1e-38)
        assert got.shape == (3, 32, 32)


def test_coil_grouping_is_consecutive_slices():
    z = np.zeros((4, 2, 2), np.complex64)
    z[0, 0, 0] = 3
    z[1, 0, 0] = 4           # image 0, coil 1
    z[2, 1, 1] = 8           # image 1, coil 0
    z[3, 1, 1] = 6j          # image 1, coil 1
    out = oracle.rss(z, 2)
    assert out[0, 0, 0] == 5 and out[1, 1, 1] == 10
    assert np.count_nonzero(out) == 2
