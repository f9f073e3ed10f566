"""The FP32 reference ablation (format "fp32") on the GPU: bit for bit equal to
the oracle's on every op, from 2x2 to 2048-point axes, through the plan calls,
the batch executor and the server."""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom
from parity_util import assert_bitwise, check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n0,n1,batch", [(2, 2, 3), (4, 8, 2), (64, 64, 3), (256, 256, 2),
                                         (128, 1024, 1), (2048, 32, 1)])
@pytest.mark.parametrize("op", ["forward", "inverse", "roundtrip", "roundtrip_fused"])
def test_fp32_reference_equals_oracle(n0, n1, batch, op, cuda_device):
    x = phantom.random_complex((batch, n0, n1), seed=n0 + 5 * n1, scale=40.0)
    check(x, "fp32", 32, op)


def test_fp32_reference_on_phantom_and_edge_values(cuda_device):
    x = phantom.mri_batch(256, 256, 2, 2, config_id=95)
    check(x, "fp32", 32, "roundtrip")
    y = phantom.random_complex((2, 64, 64), seed=96)
    y[0, 3, 4] = 1e-40 + 0j           # subnormal input
    y[1] *= np.float32(1e30)
    check(y, "fp32", 32, "forward")


def test_fp32_reference_through_engine_and_server(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.mri_batch(128, 128, 1, 4, config_id=97)
    want = oracle.mxfft2d(x, "fp32", 32, op="roundtrip")[0]
    xt = torch.from_numpy(x).cuda()
    with mxfft.Engine(graphs=True) as eng:
        y = torch.empty_like(xt)
        eng.run([("roundtrip", xt, y, "fp32", 32)])
        torch.cuda.synchronize()
    assert_bitwise(y.cpu().numpy(), want, "engine")
    h = torch.from_numpy(x).pin_memory()
    o = torch.empty_like(h).pin_memory()
    with mxfft.Server(slots=2) as srv:
        srv.submit(1, h, o, "fp32", 32, "roundtrip")
        assert srv.wait(60.0)
        assert srv.poll(4)[0].status == 0
    assert_bitwise(o.numpy(), want, "server")
    with pytest.raises(mxfft.MxfftError):
        mxfft.Plan(256, 256, "fp32", 32, path="tc16")
