"""GPU parity: the CUDA radix-2 MX path through the C ABI equals the oracle bit
for bit (outputs, including signs of zero, and the prescale exponents of
Alg. 1) on seeded inputs: every format, block size and operation, sizes from
2x2 to 2048-long axes, ragged batches, phantom k-space at the benchmark
shapes, and the edge cases of the method."""
import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom
from parity_util import check, run_gpu, run_oracle, assert_bitwise

pytestmark = pytest.mark.gpu

FMTS = ["e4m3", "e5m2", "e2m3", "e3m2", "e2m1"]
KS = [2, 4, 8, 16, 32, 64, 128]
OPS = ["forward", "inverse", "roundtrip"]


@pytest.mark.parametrize("n0,n1", [(2, 2), (2, 4), (4, 2), (4, 4), (8, 8), (2, 64), (64, 2),
                                   (16, 32), (32, 16), (128, 8), (8, 128)])
@pytest.mark.parametrize("op", OPS)
def test_small_sizes_all_formats_all_k(n0, n1, op, cuda_device):
    x = phantom.random_complex((3, n0, n1), seed=n0 * 1000 + n1)
    for fmt in FMTS:
        for k in KS:
            check(x, fmt, k, op)


@pytest.mark.parametrize("n0,n1", [(64, 64), (128, 128), (256, 32), (32, 256), (512, 16),
                                   (16, 512)])
@pytest.mark.parametrize("fmt", FMTS)
def test_medium_sizes(n0, n1, fmt, cuda_device):
    x = phantom.random_complex((2, n0, n1), seed=n0 + 3 * n1)
    for k in KS:
        for op in OPS:
            check(x, fmt, k, op)


@pytest.mark.parametrize("n0,n1", [(2048, 2), (2, 2048), (2048, 16), (16, 2048), (1024, 64)])
def test_long_axes(n0, n1, cuda_device):
    x = phantom.random_complex((1, n0, n1), seed=n0 + n1)
    for fmt, k in (("e4m3", 32), ("e5m2", 128), ("e2m1", 2), ("e3m2", 64)):
        for op in OPS:
            check(x, fmt, k, op)


def test_phantom_single_128_config(cuda_device):
    # single 128x128 phantom k-space, e4m3, k = 32, tau = 1e-3
    ksp = phantom.mri_batch(128, 128, 1, 1, config_id=1)
    img = phantom.mri_batch(128, 128, 1, 1, config_id=1, domain="image")
    check(ksp, "e4m3", 32, "forward")
    check(img, "e4m3", 32, "roundtrip")


def test_phantom_batch_256_config_full(cuda_device):
    # 64 slices of 256x256: every slice compared, e4m3 and e5m2, the k sweep
    ksp = phantom.mri_batch(256, 256, 64, 1, config_id=2)
    img = phantom.mri_batch(256, 256, 64, 1, config_id=2, domain="image")
    for fmt in ("e4m3", "e5m2"):
        check(ksp, fmt, 32, "forward")
        check(img, fmt, 32, "roundtrip")
    for k in (8, 16, 64, 128):
        check(ksp[:8], "e4m3", k, "forward")
        check(img[:8], "e5m2", k, "roundtrip")


def test_phantom_multicoil_512_sampled(cuda_device):
    # 16 coils x 32 slices of 512x512 on the GPU in one call; the oracle checks
    # a seeded sample of slices (each slice is independent)
    ksp = phantom.mri_batch(512, 512, 32, 16, config_id=3)
    got, kg, flags, st = run_gpu(ksp, "e4m3", 32, "forward")
    assert st == 0 and flags == 0
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(ksp.shape[0], 6, replace=False))
    want, kw, _ = run_oracle(ksp[sample], "e4m3", 32, "forward")
    assert_bitwise(got[sample], want, "512x512 sample")
    assert np.array_equal(np.asarray(kg)[sample], kw)


def test_large_2048_sampled(cuda_device):
    ksp = phantom.mri_batch(2048, 2048, 2, 1, config_id=5)
    for fmt, k in (("e4m3", 32), ("e2m1", 16)):
        got, kg, flags, st = run_gpu(ksp, fmt, k, "forward")
        want, kw, _ = run_oracle(ksp[:1], fmt, k, "forward")
        assert_bitwise(got[:1], want, f"2048^2 {fmt}")
        assert int(np.asarray(kg)[0]) == int(kw[0])


@pytest.mark.parametrize("n0,n1", [(64, 64), (256, 128), (128, 512), (2048, 16)])
def test_generic_kernel_matches_oracle(n0, n1, cuda_device):
    # the shared-memory kernel also covers sizes the register-resident one
    # serves; pin it there too
    x = phantom.random_complex((2, n0, n1), seed=n0 + 5 * n1)
    for fmt, k in (("e4m3", 32), ("e5m2", 8), ("e2m1", 2)):
        for op in OPS:
            check(x, fmt, k, op, generic=True)


def test_ragged_batches_and_in_place(cuda_device):
    for batch in (1, 5, 17):
        x = phantom.random_complex((batch, 32, 64), seed=batch)
        check(x, "e4m3", 16, "forward")
        check(x, "e2m3", 32, "roundtrip", inplace=True)
        check(x, "e5m2", 8, "inverse", inplace=True)


def test_edge_zero_and_single_nonzero(cuda_device):
    x = np.zeros((4, 16, 16), np.complex64)
    x[1, 0, 0] = 3 - 2j
    x[2, 7, 9] = 1e-42 + 0j          # a single FP32 subnormal
    x[3, 15, 15] = -2.5e30 + 1e30j
    for op in OPS:
        for fmt in FMTS:
            check(x, fmt, 32, op)


def test_edge_dynamic_range_and_subnormals(cuda_device):
    rng = np.random.default_rng(11)
    shape = (4, 32, 32)
    mant = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    x = (mant * np.exp2(rng.uniform(-150, 120, shape))).astype(np.complex64)
    for fmt in FMTS:
        for op in OPS:
            check(x, fmt, 8, op)


def test_edge_forced_prescale_tiny_and_huge(cuda_device):
    # k pinned to 0: blocks whose scale exponent clamps at -127 (tiny data) and
    # FP32 subnormal decoded products
    tiny = (phantom.random_complex((2, 16, 32), seed=31) * np.float32(1e-38)).astype(np.complex64)
    huge = (phantom.random_complex((2, 16, 32), seed=32) * np.float32(1e30)).astype(np.complex64)
    for fmt in FMTS:
        for x in (tiny, huge):
            check(x, fmt, 16, "forward", kmin=0, kmax=0)
            check(x, fmt, 16, "inverse", kmin=0, kmax=0)


def test_edge_prescale_options(cuda_device):
    x = phantom.mri_batch(64, 64, 3, 1, config_id=7)
    check(x, "e4m3", 32, "forward", tau=0.5, tau_min=2.0 ** -3)
    check(x, "e5m2", 32, "forward", tau=0.999, target=4.0)
    check(x, "e4m3", 32, "roundtrip", kmin=-3, kmax=5)


def test_edge_k1_rounding_boundary(cuda_device):
    # slices whose peak significand sits either side of sqrt(2)
    x = np.zeros((4, 8, 8), np.complex64)
    for i, m in enumerate((11863283, 11863284, 8388608, 16777215)):
        x[i, 3, 3] = np.float32(m * 2.0 ** -23) * np.float32(2.0 ** (i * 7 - 9))
        x[i, 0, 1] = 2.0 ** -20
    check(x, "e4m3", 8, "forward")


def test_nonfinite_inputs_flagged(cuda_device):
    x = phantom.random_complex((3, 16, 16), seed=5)
    x[1, 2, 3] = complex(np.nan, 0)
    x[2, 0, 0] = np.float32(3e38) * (1 + 1j)
    got, kg, flags, st = run_gpu(x, "e4m3", 32, "forward")
    assert st == 5 and flags == 1
    assert list(kg) [1:] == [0, 0]
    want, kw, _ = run_oracle(x[:1], "e4m3", 32, "forward")
    assert_bitwise(got[:1], want, "finite slice next to non-finite ones")


def test_invalid_arguments_on_device(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    p = mxfft.Plan(16, 16, "e4m3", 32)
    x = torch.zeros(2, 16, 16, dtype=torch.complex64, device="cuda")
    buf = torch.zeros(2 * 256 * 2 + 4, dtype=torch.float32, device="cuda")
    lib = mxfft.load()
    # misaligned pointer
    assert lib.mxfft_forward(p.handle, buf.data_ptr() + 4, x.data_ptr(), 1, None) == 1
    # partially overlapping buffers
    assert lib.mxfft_forward(p.handle, x.data_ptr(), x.data_ptr() + 16 * 8, 1, None) == 1
    assert lib.mxfft_forward(p.handle, x.data_ptr(), x.data_ptr(), -1, None) == 1
    assert lib.mxfft_forward(p.handle, x.data_ptr(), x.data_ptr(), 0, None) == 0
    with pytest.raises(mxfft.MxfftError):
        mxfft.mxfft_set_option(p.handle, mxfft.OPT_TAU_MIN, 0.3)
    with pytest.raises(mxfft.MxfftError):
        mxfft.mxfft_set_option(p.handle, mxfft.OPT_K_MAX, 127)
    p.close()


def test_accuracy_equals_stated_tolerance(cuda_device):
    # the radix-2 path reproduces the oracle bit for bit, so its accuracy
    # against FP64 is the stated figure in tests/golden/nrmse_oracle.json
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "nrmse_oracle.json")
    tol = json.load(open(path))
    ksp = phantom.mri_batch(128, 128, 1, 1, config_id=1)
    img = phantom.mri_batch(128, 128, 1, 1, config_id=1, domain="image")
    got_f, _, _, _ = run_gpu(ksp, "e4m3", 32, "forward")
    got_r, _, _, _ = run_gpu(img, "e4m3", 32, "roundtrip")
    ref = np.fft.fft2(ksp.astype(np.complex128))
    nf = np.linalg.norm(got_f - ref) / np.linalg.norm(ref)
    nr = np.linalg.norm(got_r - img.astype(np.complex128)) / np.linalg.norm(img)
    want = tol["single_128x128"]["results"][0]
    assert abs(nf - want["forward"]["nrmse"]) <= 5e-6
    assert abs(nr - want["roundtrip"]["nrmse"]) <= 5e-6
