"""The statistics kernel bins |x| = fl32(sqrt(s)), s = fl32(re^2 + im^2), by
floor(floor(log2 s) / 2) without taking the square root, and takes the
maximum |x| as fl32(sqrt(max s)).  Both rest on properties of the correctly
rounded float32 square root, checked here on every float near each power of
two (where a rounding could cross a binade) and on random floats."""
import numpy as np


def _bin_via_sqrt(s):
    m = np.sqrt(s)                      # float32, correctly rounded
    return (m.view(np.uint32) >> 23).astype(np.int64) - 127


def _bin_via_s(s):
    return ((s.view(np.uint32) >> 23).astype(np.int64) - 127) >> 1


def test_bin_identity_near_every_binade_edge():
    # s in [2^-124, 2^127): the range where s is normal and finite
    edges = np.arange(-124, 128, dtype=np.int64)
    base = ((edges + 127) << 23).astype(np.int64)
    offs = np.arange(-2000, 2000, dtype=np.int64)
    bits = (base[:, None] + offs[None, :]).ravel()
    lo, hi = (127 - 124) << 23, (127 + 127) << 23
    bits = bits[(bits >= lo) & (bits < hi)].astype(np.uint32)
    s = bits.view(np.float32)
    np.testing.assert_array_equal(_bin_via_sqrt(s), _bin_via_s(s))


def test_bin_identity_random():
    rng = np.random.default_rng(20251204)
    bits = rng.integers((127 - 124) << 23, (127 + 127) << 23, size=2_000_000, dtype=np.uint32)
    s = bits.view(np.float32)
    np.testing.assert_array_equal(_bin_via_sqrt(s), _bin_via_s(s))


def test_max_commutes_with_rounded_sqrt():
    rng = np.random.default_rng(7)
    bits = rng.integers((127 - 124) << 23, (127 + 127) << 23, size=(20000, 33), dtype=np.uint32)
    s = bits.view(np.float32)
    np.testing.assert_array_equal(np.sqrt(s).max(axis=1), np.sqrt(s.max(axis=1)))


def test_byte_offset_of_the_bin():
    # the statistics kernel's two-point body addresses the histogram word of
    # bin floor(floor(log2 s) / 2) + 149 as the byte offset
    # ((bits(s) >> 22) + 342) & ~3; every normal s (all biased exponents,
    # both values of the top significand bit, either end of the significand)
    e = np.arange(1, 255, dtype=np.uint32)
    top = np.array([0, 1 << 22, (1 << 23) - 1, 1], dtype=np.uint32)
    bits = ((e[:, None] << np.uint32(23)) | top[None, :]).ravel().astype(np.uint32)
    want = _bin_via_s(bits.view(np.float32)) + 149
    got = (((bits >> np.uint32(22)).astype(np.int64) + 342) & ~3) // 4
    np.testing.assert_array_equal(got, want)
    assert want.min() >= 0 and want.max() < 277
    # a shift by 23 instead of 22 fails
    assert not np.array_equal((((bits >> np.uint32(23)).astype(np.int64) + 342) & ~3) // 4, want)


def test_two_point_range_test_equals_both_point_tests():
    # the two-point body takes its fast path when min over the four
    # components of (|bits| - 1) (wrapping) is >= lo - 1 and their max is
    # < hi; that must hold exactly when each point passes its own test
    # (each component zero or of magnitude in [2^-62, 2^63))
    lo, hi = (127 - 62) << 23, (127 + 63) << 23
    edge = np.array([0, 1, lo - 1, lo, lo + 1, hi - 1, hi, hi + 1, 0x7f800000, 0x7fc00000,
                     127 << 23, 0x007fffff], dtype=np.uint32)
    rng = np.random.default_rng(11)
    comp = np.concatenate([edge, rng.integers(0, 0x7fffffff, 64, dtype=np.uint32)])
    q = rng.integers(0, len(comp), size=(200_000, 4))
    u = comp[q]                                           # |bits| of re0, im0, re1, im1
    um1 = u - np.uint32(1)

    def point_ok(a, b):
        return (np.minimum(um1[:, a], um1[:, b]) >= lo - 1) & (np.maximum(u[:, a], u[:, b]) < hi)

    def in_range(c):
        return (u[:, c] == 0) | ((u[:, c] >= lo) & (u[:, c] < hi))

    for a, b in ((0, 1), (2, 3)):
        np.testing.assert_array_equal(point_ok(a, b), in_range(a) & in_range(b))
    pair = (um1.min(axis=1) >= lo - 1) & (u.max(axis=1) < hi)
    np.testing.assert_array_equal(pair, point_ok(0, 1) & point_ok(2, 3))
    assert pair.any() and not pair.all()
