"""The FP16 positive control (format code 5) on the GPU: bit for bit equal to
the oracle's control on every op and on sizes from 2x2 to 2048-point axes,
through the plan calls, the batch executor and the server; and, as a
positive control, far more accurate than MXFP8 on the phantom."""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom
from parity_util import assert_bitwise, check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n0,n1,batch", [(2, 2, 3), (4, 8, 2), (64, 64, 3), (256, 256, 2),
                                         (128, 1024, 1), (2048, 32, 1)])
@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip"])
def test_fp16_control_equals_oracle(n0, n1, batch, op, cuda_device):
    x = phantom.random_complex((batch, n0, n1), seed=n0 + 7 * n1, scale=40.0)
    check(x, "fp16", 32, op)


@pytest.mark.parametrize("op", ["forward", "roundtrip"])
def test_fp16_control_on_phantom(op, cuda_device):
    dom = "image" if op == "roundtrip" else "kspace"
    x = phantom.mri_batch(256, 256, 2, 2, config_id=91, domain=dom)
    check(x, "fp16", 32, op)


def test_fp16_overflow_follows_ieee(cuda_device):
    # a large constant makes the late-stage products exceed 65504: infinities
    # and NaNs must appear where the oracle has them
    x = np.full((1, 512, 512), 1.0 + 1.0j, np.complex64)
    x[0, 3, 5] = 1.5
    check(x, "fp16", 32, "forward")


def test_fp16_control_through_engine_and_server(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(128, 128, 1, 4, config_id=92)
    want = oracle.mxfft2d(x, "fp16", 32, op="roundtrip")[0]
    xt = torch.from_numpy(x).cuda()
    with mxfft.Engine(graphs=True) as eng:
        y = torch.empty_like(xt)
        eng.run([("roundtrip", xt, y, "fp16", 32)])
        torch.cuda.synchronize()
    assert_bitwise(y.cpu().numpy(), want, "engine")
    h = torch.from_numpy(x).pin_memory()
    o = torch.empty_like(h).pin_memory()
    with mxfft.Server(slots=2) as srv:
        srv.submit(1, h, o, "fp16", 32, "roundtrip")
        assert srv.wait(60.0)
        assert srv.poll(4)[0].status == 0
    assert_bitwise(o.numpy(), want, "server")


def test_fp16_is_a_positive_control(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(256, 256, 4, 1, config_id=93)
    ref = np.fft.fft2(x.astype(np.complex128))
    xt = torch.from_numpy(x).cuda()
    err = {}
    for fmt in ("fp16", "e4m3"):
        with mxfft.Plan(256, 256, fmt, 32) as p:
            y = p.forward(xt).cpu().numpy().astype(np.complex128)
        err[fmt] = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err["fp16"] < 0.01 and err["fp16"] < err["e4m3"] / 20, err
    with pytest.raises(mxfft.MxfftError):
        mxfft.Plan(256, 256, "fp16", 32, path="tc16")
