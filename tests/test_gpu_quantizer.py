"""The device element quantisers (mxfft_quantize: the register-resident pass's
hardware conversions and the generic pass's FP32 rounding) against the
oracle's quantiser, which the CPU tests pin to the OCP code tables and a
brute-force nearest-code search.  Every positive FP32 bit pattern from two
binades below each format's smallest subnormal to two binades above its
largest normal is compared bit for bit (ties to the even code, subnormal
targets, values between the largest normal and the next binade that saturate,
signed zeros), then a sampled set of negative values, values deep below the
grid (they round to zero) and far above it (they saturate)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

# unbiased exponents of the smallest subnormal and of the largest normal
GRID = {"e4m3": (-9, 8), "e5m2": (-16, 15), "e2m3": (-3, 2), "e3m2": (-4, 4), "e2m1": (-1, 2)}
CHUNK = 1 << 24


def oracle_q(x, fmt):
    """The oracle's quantiser over host cores (ctypes releases the GIL)."""
    parts = np.array_split(x, 16)
    with ThreadPoolExecutor(16) as ex:
        return np.concatenate(list(ex.map(lambda p: oracle.quantize(p, fmt), parts)))


def device_q(x, fmt):
    """(conversion path, generic path) results for x."""
    import torch

    from paper_2512_04317_gb300 import mxfft
    xd = torch.from_numpy(x).cuda()
    out = []
    for path in (0, 1):
        yd = torch.empty_like(xd)
        mxfft.mxfft_quantize(xd.data_ptr(), yd.data_ptr(), x.size, fmt, path,
                             torch.cuda.current_stream().cuda_stream)
        out.append(yd)
    torch.cuda.synchronize()
    return [y.cpu().numpy() for y in out]


def compare(x, fmt):
    want = oracle_q(x, fmt).view(np.uint32)
    for path, res in enumerate(device_q(x, fmt)):
        got = res.view(np.uint32)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (fmt, path, x[bad[:5]], got[bad[:5]].view(np.float32),
                               want[bad[:5]].view(np.float32))


@pytest.mark.parametrize("fmt", sorted(GRID))
def test_device_quantisers_equal_oracle_on_every_pattern(fmt, cuda_device):
    lo, hi = GRID[fmt]
    b0, b1 = (lo - 2 + 127) << 23, (hi + 3 + 127) << 23
    for start in range(b0, b1, CHUNK):
        bits = np.arange(start, min(start + CHUNK, b1), dtype=np.uint32)
        compare(bits.view(np.float32), fmt)


@pytest.mark.parametrize("fmt", sorted(GRID))
def test_device_quantisers_signs_extremes_and_zeros(fmt, cuda_device):
    rng = np.random.default_rng(7)
    lo, hi = GRID[fmt]
    inside = rng.integers((lo - 2 + 127) << 23, (hi + 3 + 127) << 23, 1 << 22, dtype=np.uint32)
    below = rng.integers(1, (lo - 2 + 127) << 23, 1 << 20, dtype=np.uint32)   # incl. FP32 subnormals
    above = rng.integers((hi + 3 + 127) << 23, 0x7f800000, 1 << 20, dtype=np.uint32)
    bits = np.concatenate([inside, inside | 0x80000000, below, below | 0x80000000,
                           above, above | 0x80000000, np.array([0, 0x80000000], np.uint32)])
    compare(bits.view(np.float32), fmt)
