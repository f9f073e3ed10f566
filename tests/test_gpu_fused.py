"""GPU parity of the fused encode -> F -> F^-1 -> decode round trip (Sec. 4.3,
reading C17): through the C ABI, bit for bit against the oracle (outputs and
the one prescale exponent per slice) on the register-resident kernel that runs
both column transforms of a tile in one launch, on the generic kernel, at long
axes and ragged batches, in place, on the phantom at the benchmark's shapes,
and through the tensor-core variant against its emulation."""
import os
import sys

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom
from parity_util import assert_bitwise, check, run_gpu, run_oracle, assert_close_to_emulation

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import tc16_ref  # noqa: E402

pytestmark = pytest.mark.gpu

OP = "roundtrip_fused"
FMTS = ["e4m3", "e5m2", "e2m3", "e3m2", "e2m1"]


@pytest.mark.parametrize("n0,n1", [(64, 64), (128, 256), (256, 64), (512, 32), (1024, 16),
                                   (2048, 16)])
@pytest.mark.parametrize("fmt", FMTS)
def test_fused_column_kernel(n0, n1, fmt, cuda_device):
    # n0 in [64, 2048] and m <= 16: both column transforms in one launch
    x = phantom.random_complex((3, n0, n1), seed=n0 + 7 * n1)
    for k in (2, 8, 32):
        check(x, fmt, k, OP)


@pytest.mark.parametrize("n0,n1", [(2, 2), (4, 8), (32, 16), (16, 128), (8, 2048)])
def test_small_and_generic_sizes(n0, n1, cuda_device):
    # columns shorter than 64 (generic kernel, two passes) and every k
    x = phantom.random_complex((2, n0, n1), seed=n0 * 31 + n1)
    for fmt in FMTS:
        for k in (2, 4, 16, 32, 64, 128):
            check(x, fmt, k, OP)


@pytest.mark.parametrize("k", [64, 128])
def test_large_blocks(k, cuda_device):
    # m = k / 2 = 32, 64: blocks over 4 / 8 lanes (groups of 8 / 4 transforms)
    x = phantom.random_complex((2, 256, 128), seed=k)
    check(x, "e4m3", k, OP)
    # columns of 64 with m = 32: the generic kernel's two column passes
    y = phantom.random_complex((2, 64, 128), seed=k + 1)
    check(y, "e5m2", 64, OP)


def test_generic_kernel_gives_the_same_bits(cuda_device):
    x = phantom.mri_batch(256, 256, 4, 1, config_id=2, domain="image")
    a, ka, _, _ = run_gpu(x, "e4m3", 32, OP)
    b, kb, _, _ = run_gpu(x, "e4m3", 32, OP, generic=True)
    assert_bitwise(a, b, "fused kernel vs generic")
    assert np.array_equal(ka, kb)


def test_in_place_and_ragged_batch(cuda_device):
    x = phantom.random_complex((5, 512, 256), seed=77)
    check(x, "e5m2", 16, OP, inplace=True)
    check(x[:1], "e2m1", 32, OP)


def test_phantom_batch_256_config(cuda_device):
    # the benchmark's image-domain batch, every slice
    img = phantom.mri_batch(256, 256, 64, 1, config_id=2, domain="image")
    for fmt in ("e4m3", "e5m2"):
        check(img, fmt, 32, OP)


def test_long_axes_2048(cuda_device):
    x = phantom.mri_batch(2048, 2048, 1, 1, config_id=5, domain="image")
    check(x, "e4m3", 32, OP)


def test_edge_inputs(cuda_device):
    z = np.zeros((2, 64, 64), np.complex64)
    check(z, "e4m3", 32, OP)
    d = z.copy()
    d[:, 0, 0] = 1.5 + 0.75j
    got, _, _, st = run_gpu(d, "e4m3", 32, OP)
    assert st == 0 and np.array_equal(got, d)
    tiny = phantom.random_complex((1, 128, 128), seed=3, scale=1e-40)
    check(tiny, "e4m3", 32, OP)
    big = phantom.random_complex((1, 128, 128), seed=4, scale=1e30)
    check(big, "e5m2", 32, OP)
    nf = phantom.random_complex((2, 64, 64), seed=5)
    nf[1, 3, 7] = np.inf
    check(nf, "e4m3", 32, OP)


def test_fp16_control_is_unsupported(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.zeros(1, 64, 64, dtype=torch.complex64, device="cuda")
    with mxfft.Plan(64, 64, "fp16", 32) as p:
        with pytest.raises(mxfft.MxfftError) as ei:
            p.roundtrip_fused(x)
    assert ei.value.status == mxfft.MXFFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("n0,n1,k", [(256, 256, 32), (512, 256, 64), (1024, 1024, 32)])
def test_tensor_core_variant_matches_emulation(n0, n1, k, cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(n0, n1, 2, 1, config_id=9, domain="image")
    with mxfft.Plan(n0, n1, "e4m3", k, path="tc16") as p:
        y = p.roundtrip_fused(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        st, flags, _ = p.status()
    assert st == 0 and flags == 0
    want = tc16_ref.mxfft2d(x, "e4m3", OP, k)
    assert_close_to_emulation(y.cpu().numpy(), want, (n0, n1, k))
    # and it is at least as accurate as the radix-2 fused round trip
    r2, _, _ = run_oracle(x, "e4m3", k, OP)
    e_tc = np.linalg.norm(y.cpu().numpy() - x) / np.linalg.norm(x)
    e_r2 = np.linalg.norm(r2 - x) / np.linalg.norm(x)
    assert e_tc <= 1.10 * e_r2, (e_tc, e_r2)
