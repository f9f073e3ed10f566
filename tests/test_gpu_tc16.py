"""Tensor-core radix-16 variant (MXFFT_OPT_PATH = 1): radix-16 sub-DFTs as
MXFP8 tcgen05 matrix products, n in {128, 256, 512, 1024, 2048} (n = 128:
16 x 8, the second round's 8-point DFTs in pairs per matrix row).  Not bit-exact
with the radix-2 oracle by design; checked (1) against a numpy emulation of
the same algorithm to FP32 accumulation-order level, and (2) against FP64 with the stated tolerance:
NRMSE <= 1.10 x the radix-2 oracle's NRMSE on the same input."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom
from parity_util import assert_close_to_emulation, run_gpu

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import tc16_ref  # noqa: E402

pytestmark = pytest.mark.gpu


def run_tc16(x, fmt, op, k=32):
    import torch

    from paper_2512_04317_gb300 import mxfft
    xt = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).cuda()
    with mxfft.Plan(x.shape[-2], x.shape[-1], fmt, k, path="tc16") as p:
        y = getattr(p, op)(xt)
        torch.cuda.synchronize()
        st, flags, _ = p.status()
    assert st == 0 and flags == 0, (st, flags)
    return y.cpu().numpy()


def nrmse(a, ref):
    return float(np.linalg.norm(a.astype(np.complex128) - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n0,n1", [(256, 256), (512, 512), (256, 512), (512, 256), (1024, 1024),
                                   (256, 1024), (1024, 512), (128, 128), (128, 256), (256, 128),
                                   (128, 1024), (2048, 128)])
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip"])
def test_tc16_matches_emulation(n0, n1, fmt, op, cuda_device):
    x = phantom.mri_batch(n0, n1, 2, 1, config_id=31, domain="image" if op == "roundtrip" else "kspace")
    got = run_tc16(x, fmt, op)
    want = tc16_ref.mxfft2d(x, fmt, op)
    assert_close_to_emulation(got, want, (n0, n1, fmt, op))


@pytest.mark.parametrize("n0,n1,fmt,op", [(2048, 2048, "e4m3", "forward"),
                                           (2048, 2048, "e5m2", "roundtrip"),
                                           (2048, 512, "e4m3", "inverse"),
                                           (256, 2048, "e5m2", "forward"),
                                           (2048, 256, "e4m3", "roundtrip_fused")])
def test_tc16_2048_matches_emulation(n0, n1, fmt, op, cuda_device):
    # n = 2048 = 16 x 16 x 8: the last stage is a radix-8 DFT in FP32
    img = op in ("roundtrip", "roundtrip_fused")
    x = phantom.mri_batch(n0, n1, 1, 1, config_id=36, domain="image" if img else "kspace")
    got = run_tc16(x, fmt, op)
    want = tc16_ref.mxfft2d(x, fmt, op)
    assert_close_to_emulation(got, want, (n0, n1, fmt, op))


@pytest.mark.parametrize("n0,n1", [(256, 256), (512, 512), (256, 512), (1024, 256), (2048, 256),
                                   (128, 128), (128, 512)])
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("k", [64, 128])
def test_tc16_shared_block_scales_match_emulation(n0, n1, fmt, k, cuda_device):
    # k = 64 / 128: one scale for 2 / 4 consecutive vectors, across warps on
    # the columns pass
    for op in ("forward", "roundtrip"):
        x = phantom.mri_batch(n0, n1, 2, 1, config_id=35, domain="image" if op == "roundtrip" else "kspace")
        got = run_tc16(x, fmt, op, k)
        want = tc16_ref.mxfft2d(x, fmt, op, k)
        assert_close_to_emulation(got, want, (n0, n1, fmt, k, op))


@pytest.mark.parametrize("n", [128, 256, 512, 1024])
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("k", [32, 64, 128])
def test_tc16_within_stated_tolerance(n, fmt, k, cuda_device):
    ksp = phantom.mri_batch(n, n, 4, 1, config_id=32)
    img = phantom.mri_batch(n, n, 4, 1, config_id=32, domain="image")
    ref = np.fft.fft2(ksp.astype(np.complex128))
    r2f = nrmse(oracle.mxfft2d(ksp, fmt, k)[0], ref)
    r2r = nrmse(oracle.mxfft2d(img, fmt, k, op="roundtrip")[0], img.astype(np.complex128))
    tcf = nrmse(run_tc16(ksp, fmt, "forward", k), ref)
    tcr = nrmse(run_tc16(img, fmt, "roundtrip", k), img.astype(np.complex128))
    assert tcf <= 1.10 * r2f, (tcf, r2f)
    assert tcr <= 1.10 * r2r, (tcr, r2r)


@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
def test_tc16_2048_within_stated_tolerance(fmt, cuda_device):
    ksp = phantom.mri_batch(2048, 2048, 1, 1, config_id=37)
    ref = np.fft.fft2(ksp.astype(np.complex128))
    r2f = nrmse(oracle.mxfft2d(ksp, fmt, 32)[0], ref)
    tcf = nrmse(run_tc16(ksp, fmt, "forward", 32), ref)
    assert tcf <= 1.10 * r2f, (tcf, r2f)


def test_tc16_option_validation(cuda_device):
    from paper_2512_04317_gb300 import mxfft
    for args in [(64, 256, "e4m3", 32), (256, 256, "e2m3", 32), (256, 256, "e4m3", 16)]:
        with pytest.raises(mxfft.MxfftError) as ei:
            mxfft.Plan(*args, path="tc16")
        assert ei.value.status == mxfft.MXFFT_ERR_UNSUPPORTED
    # same plan can switch back to the bit-exact path
    p = mxfft.Plan(256, 256, "e4m3", 32, path="tc16")
    mxfft.mxfft_set_option(p.handle, mxfft.OPT_PATH, 0)
    p.close()


@pytest.mark.parametrize("n0,n1,batch", [(256, 256, 40), (512, 512, 6), (512, 256, 11),
                                         (1024, 1024, 3), (1024, 256, 5), (2048, 2048, 2),
                                         (2048, 256, 9), (128, 128, 97), (128, 512, 7),
                                         (512, 128, 13)])
def test_tc16_many_tiles_per_cta(n0, n1, batch, cuda_device):
    # more 4096-point tiles than resident CTAs: every CTA walks several tiles,
    # an uneven number each, through both shared buffers
    x = phantom.random_complex((batch, n0, n1), seed=77, scale=3.0)
    got = run_tc16(x, "e4m3", "forward")
    want = tc16_ref.mxfft2d(x, "e4m3", "forward")
    assert_close_to_emulation(got, want, (n0, n1, batch))


def test_tc16_in_place(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(512, 512, 3, 1, config_id=33, domain="image")
    want = run_tc16(x, "e4m3", "roundtrip")
    xt = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).cuda()
    with mxfft.Plan(512, 512, "e4m3", 32, path="tc16") as p:
        p.roundtrip(xt, out=xt)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(xt.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_bounded_wait_times_out_and_the_context_stays_usable(cuda_device):
    # the products are withheld, so the completion mbarrier is never arrived
    # on: every CTA's wait must run out (100 ms), set the timeout flag and let
    # the kernel finish; afterwards the same plan computes correctly
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(256, 256, 2, 1, config_id=34)).cuda()
    with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as ref:
        want = ref.forward(x).cpu().numpy()
    with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as p:
        mxfft.mxfft_set_option(p.handle, mxfft.OPT_TEST_STALL, 1)
        p.forward(x)
        torch.cuda.synchronize()
        st, flags, _ = p.status()
        assert st == mxfft.MXFFT_ERR_TIMEOUT and flags & 2
        mxfft.mxfft_set_option(p.handle, mxfft.OPT_TEST_STALL, 0)
        got = p.forward(x)
        torch.cuda.synchronize()
        st, flags, _ = p.status()
        assert st == 0 and flags == 0
        np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
