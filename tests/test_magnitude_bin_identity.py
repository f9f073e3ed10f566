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
