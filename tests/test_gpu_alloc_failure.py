"""Allocation failure in the plan allocator (the test hook
mxfft_test_fail_alloc): every device allocation a plan makes -- its twiddle
tables, the tensor-core tables, its statistics records and their growth on a
larger batch -- is made to fail in turn.  Each failure must come back as
MXFFT_ERR_NOMEM from the call that allocated, leave no device memory behind,
and leave the library usable (the next plan computes the same result)."""
import gc

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom

pytestmark = pytest.mark.gpu


def test_every_plan_allocation_failure_is_reported_without_leaks(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(256, 256, 3, 1, config_id=51)).cuda()
    y = torch.empty_like(x)               # allocated by torch before the measurement
    with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as ref:
        want = ref.forward(x, out=y).cpu().numpy()
    torch.cuda.synchronize()
    gc.collect()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    for after in range(40):
        mxfft.mxfft_test_fail_alloc(after)
        try:
            with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as p:
                p.forward(x, out=y)       # grows the statistics records to 3 slices
                torch.cuda.synchronize()
            # no failure left for this position: the hook was not reached
            np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), want.view(np.uint32))
            mxfft.mxfft_test_fail_alloc(-1)
            break
        except mxfft.MxfftError as e:
            assert e.status == mxfft.MXFFT_ERR_NOMEM, (after, e)
            failures += 1
        finally:
            mxfft.mxfft_test_fail_alloc(-1)
        torch.cuda.synchronize()
        gc.collect()                      # a plan whose constructor raised is freed
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (after, free0 - free1)
    assert failures >= 10        # the plan, its tensor-core tables and the statistics growth
    with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as p:
        got = p.forward(x, out=y).cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_hook_rejects_bad_values(cuda_device):
    from paper_2512_04317_gb300 import mxfft
    with pytest.raises(mxfft.MxfftError):
        mxfft.mxfft_test_fail_alloc(-2)
