"""Fused 2D tensor-core transform (MXFFT_OPT_FUSED2D, n0, n1 in {256, 512}):
each slice on one thread-block cluster, statistics, rows and columns in one
launch.  Its arithmetic per element is that of the per-axis tensor-core passes,
so on finite inputs its results equal theirs bit for bit (the packed twiddle
product rounds like the passes' scale-then-multiply order whenever no
intermediate is subnormal); it is also compared element by element with the
numpy emulation of the variant and with FP64 under the stated tolerance."""
import os
import sys

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import tc16_ref  # noqa: E402
from parity_util import assert_close_to_emulation  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256), (256, 512), (512, 256), (512, 512)]


def run(x, fmt, op, fused2d, k=32):
    import torch

    from paper_2512_04317_gb300 import mxfft
    xt = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).cuda()
    with mxfft.Plan(x.shape[-2], x.shape[-1], fmt, k, path="tc16", fused2d=fused2d) as p:
        mxfft.mxfft_profile(p.handle, True)
        y = getattr(p, op)(xt)
        torch.cuda.synchronize()
        prof = mxfft.mxfft_profile_read(p.handle)
        st, flags, kk = p.status()
    return y.cpu().numpy(), st, flags, kk, prof


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("n0,n1", SHAPES)
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip"])
def test_fused2d_equals_per_axis_passes(n0, n1, fmt, op, cuda_device):
    dom = "image" if op == "roundtrip" else "kspace"
    x = phantom.mri_batch(n0, n1, 3, 1, config_id=41, domain=dom)
    got, st, flags, kf, prof = run(x, fmt, op, True)
    want, st2, flags2, kp, prof2 = run(x, fmt, op, False)
    assert st == 0 and flags == 0 and st2 == 0 and flags2 == 0
    # the fused kernel ran (one launch per transform) and the passes did not
    assert prof["tc2d_kernel"][1] == (2 if op == "roundtrip" else 1)
    assert prof["tc16_pass_kernel"][1] == 0 and prof["stats_kernel"][1] == 0
    assert prof2["tc2d_kernel"][1] == 0
    assert kf == kp
    np.testing.assert_array_equal(bits(got), bits(want))


@pytest.mark.parametrize("n0,n1,batch", [(512, 512, 21), (256, 256, 47), (256, 512, 19)])
def test_fused2d_walks_several_slices_per_cluster(n0, n1, batch, cuda_device):
    # more slices than resident clusters: each cluster walks several slices,
    # and the next slice's copies start during the last column tile
    x = phantom.random_complex((batch, n0, n1), seed=91, scale=5.0)
    x[batch // 2] *= np.float32(1e-20)            # a slice of its own, much smaller scale
    got, st, flags, kf, _ = run(x, "e4m3", "forward", True)
    want, _, _, kp, _ = run(x, "e4m3", "forward", False)
    assert st == 0 and kf == kp
    np.testing.assert_array_equal(bits(got), bits(want))


@pytest.mark.parametrize("n0,n1", SHAPES)
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("op", ["forward", "roundtrip"])
def test_fused2d_elementwise_vs_emulation(n0, n1, fmt, op, cuda_device):
    dom = "image" if op == "roundtrip" else "kspace"
    x = phantom.mri_batch(n0, n1, 2, 1, config_id=42, domain=dom)
    got, st, _, _, _ = run(x, fmt, op, True)
    want = tc16_ref.mxfft2d(x, fmt, op)
    assert st == 0
    assert_close_to_emulation(got, want, (n0, n1, fmt, op))


def test_fused2d_edge_slices(cuda_device):
    # zero slice: k = 0 and zeros out; a slice holding NaN: flag set (its
    # output is unspecified); tiny and huge slices: the prescale brings them
    # into range, equal to the passes
    x = phantom.mri_batch(256, 256, 5, 1, config_id=43)
    x[1] = 0
    x[2, 7, 9] = np.nan
    x[3] *= np.float32(1e-30)
    x[4] *= np.float32(1e25)
    got, st, flags, kf, _ = run(x, "e4m3", "forward", True)
    want, st2, flags2, kp, _ = run(x, "e4m3", "forward", False)
    assert flags & 1 and flags2 & 1 and kf == kp
    assert kf[1] == 0 and kf[2] == 0
    assert not got[1].any()
    for s in (0, 1, 3, 4):
        np.testing.assert_array_equal(bits(got[s]), bits(want[s]))


def test_fused2d_in_place(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(512, 512, 2, 1, config_id=44, domain="image")
    want, _, _, _, _ = run(x, "e5m2", "roundtrip", True)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with mxfft.Plan(512, 512, "e5m2", 32, path="tc16", fused2d=True) as p:
        p.roundtrip(xt, out=xt)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(bits(xt.cpu().numpy()), bits(want))


def test_fused2d_engine_step_is_two_launches(cuda_device):
    # forward of one batch + round trip of another through the executor: one
    # fused launch for both forward transforms, one for the inverse; same bits
    # as the plan calls, with and without graphs
    import torch

    from paper_2512_04317_gb300 import mxfft
    xk = torch.from_numpy(phantom.mri_batch(512, 512, 4, 1, config_id=45)).cuda()
    xi = torch.from_numpy(phantom.mri_batch(512, 512, 4, 1, config_id=45, domain="image")).cuda()
    with mxfft.Plan(512, 512, "e4m3", 32, path="tc16") as p:
        wk = p.forward(xk).cpu().numpy()
        wi = p.roundtrip(xi).cpu().numpy()
    for graphs in (False, True):
        with mxfft.Engine(graphs=graphs, tc16=True, fused2d=True) as eng:
            yk, yi = torch.empty_like(xk), torch.empty_like(xi)
            for _ in range(2):
                eng.run([("forward", xk, yk, "e4m3", 32), ("roundtrip", xi, yi, "e4m3", 32)])
                torch.cuda.synchronize()
                assert eng.launches_per_run() == 2
                flags, k = eng.status()
                assert flags == 0
                np.testing.assert_array_equal(bits(yk.cpu().numpy()), bits(wk))
                np.testing.assert_array_equal(bits(yi.cpu().numpy()), bits(wi))


def test_fused2d_bounded_wait_times_out(cuda_device):
    # the products are withheld: every CTA's first wait runs out, the CTAs
    # skip the rest but keep to the cluster barriers, the call reports the
    # time-out, and the same plan then computes the right result
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(512, 512, 2, 1, config_id=46)).cuda()
    with mxfft.Plan(512, 512, "e4m3", 32, path="tc16", fused2d=True) as ref:
        want = ref.forward(x).cpu().numpy()
    with mxfft.Plan(512, 512, "e4m3", 32, path="tc16", fused2d=True) as p:
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
        np.testing.assert_array_equal(bits(got.cpu().numpy()), bits(want))
