"""The allocation-free exponent entry point (mxfft_prescale_exponents_noalloc)
against the plan-based transforms.

It exists for callers that cannot allocate device memory at call time (a
fixed memory pool owned by another framework, a real-time loop that must not
reach the allocator); its scratch is a static device array shared by all
calls, so two calls in a row with different shapes also check that each call
clears what it uses.  Collected last on purpose: it must pass both alone in a
fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_2512_04317_gb300 import mxfft, phantom

pytestmark = pytest.mark.gpu


def plan_exponents(x, fmt):
    """k of every slice through the existing entry point (mxfft_forward)."""
    with mxfft.Plan(x.shape[-2], x.shape[-1], fmt, 32) as p:
        p.forward(x)
        st, flags, k = p.status()
    return [int(v) for v in k]


def noalloc_exponents(x, fmt):
    import torch
    batch = x.shape[0]
    k = torch.full((batch,), -9999, dtype=torch.int32, device=x.device)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    st = mxfft.mxfft_prescale_exponents_noalloc(x.data_ptr(), batch, x.shape[-2], x.shape[-1],
                                                fmt, 1e-3, 0.5, k.data_ptr(), stream)
    assert st == mxfft.MXFFT_OK, mxfft.status_string(st)
    torch.cuda.synchronize()
    return k.cpu().tolist()


def test_noalloc_exponents_equal_plan_path_on_two_calls_in_a_row(cuda_device):
    import torch
    big = phantom.mri_batch(256, 256, 12, 1, config_id=11)
    big[3] = 0                                    # an all-zero slice: k = 0
    big[7, 5, 9] = np.nan                         # a non-finite slice: k = 0
    big[9] *= np.float32(1e-30)                   # a tiny slice: large k
    small = phantom.random_complex((5, 64, 32), seed=12, scale=1e4)
    calls = [(big, "e4m3"), (small, "e5m2")]      # the second call reuses the scratch
    for arr, fmt in calls:
        x = torch.from_numpy(arr).to(cuda_device)
        want = plan_exponents(x, fmt)
        got = noalloc_exponents(x, fmt)
        assert got == want, (fmt, got, want)


def test_noalloc_calls_after_the_first_take_no_device_memory(cuda_device):
    """After the set-up call (which may load the library's device code), a
    call leaves both the device's free memory and torch's allocator as they
    were: its scratch is the static array, nothing else."""
    import torch
    x = torch.from_numpy(phantom.mri_batch(128, 128, 6, 1, config_id=13)).to(cuda_device)
    k = torch.zeros(6, dtype=torch.int32, device=cuda_device)
    stream = torch.cuda.current_stream(cuda_device).cuda_stream
    args = (x.data_ptr(), 6, 128, 128, "e4m3", 1e-3, 0.5, k.data_ptr(), stream)
    assert mxfft.mxfft_prescale_exponents_noalloc(*args) == mxfft.MXFFT_OK   # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(cuda_device)
    alloc0 = torch.cuda.memory_allocated(cuda_device)
    for _ in range(3):
        assert mxfft.mxfft_prescale_exponents_noalloc(*args) == mxfft.MXFFT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(cuda_device)
    assert free1 == free0
    assert torch.cuda.memory_allocated(cuda_device) == alloc0
    assert k.cpu().tolist() == plan_exponents(x, "e4m3")


def test_noalloc_rejects_batches_beyond_its_scratch(cuda_device):
    import torch
    x = torch.zeros(2, 4, 4, dtype=torch.complex64, device=cuda_device)
    k = torch.zeros(2, dtype=torch.int32, device=cuda_device)
    st = mxfft.mxfft_prescale_exponents_noalloc(x.data_ptr(), mxfft.NOALLOC_MAX_SLICES + 1, 4, 4,
                                                "e4m3", 1e-3, 0.5, k.data_ptr())
    assert st == mxfft.MXFFT_ERR_INVALID
