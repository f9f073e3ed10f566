"""The launch configuration bench.py times -- one batch-executor run per step
replayed as a CUDA graph, with the shipped autotuned geometries loaded, over the
64-slice 256x256 forward and round-trip batches -- checked against the oracle
on every slice, bit for bit."""
import os

import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom
from parity_util import assert_bitwise

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_step_through_tuned_graph_equals_oracle(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    tfile = os.path.join(ROOT, "paper_2512_04317_gb300", "tuning", "gb300_sm103a.json")
    mxfft.mxfft_tune_load(tfile)
    try:
        ksp = phantom.mri_batch(256, 256, 64, 1, config_id=2)
        img = phantom.mri_batch(256, 256, 64, 1, config_id=2, domain="image")
        xk, xi = torch.from_numpy(ksp).cuda(), torch.from_numpy(img).cuda()
        yk, yi = torch.empty_like(xk), torch.empty_like(xi)
        with mxfft.Engine(graphs=True) as eng:
            for _ in range(3):      # capture, then replays
                eng.run([("forward", xk, yk, "e4m3", 32), ("roundtrip", xi, yi, "e4m3", 32)])
            torch.cuda.synchronize()
            flags, ks = eng.status()
        assert flags == 0
        wk, kk, _ = oracle.mxfft2d(ksp, "e4m3", 32, op="forward")
        wi, ki, _ = oracle.mxfft2d(img, "e4m3", 32, op="roundtrip")
        assert_bitwise(yk.cpu().numpy(), wk, "bench forward")
        assert_bitwise(yi.cpu().numpy(), wi, "bench round trip")
        assert [k[0] for k in ks[:64]] == [int(v) for v in kk]
        assert [k for k in ks[64:]] == [[int(a), int(b)] for a, b in ki]
    finally:
        mxfft.mxfft_tune_clear()


@pytest.mark.parametrize("fmt,k,op", [("e2m3", 64, "forward"), ("e3m2", 32, "roundtrip")])
def test_large_2048_fp6_sampled(fmt, k, op, cuda_device):
    from parity_util import run_gpu, run_oracle
    x = phantom.mri_batch(2048, 2048, 2, 1, config_id=5, domain="image" if op == "roundtrip" else "kspace")
    got, kg, flags, st = run_gpu(x, fmt, k, op)
    assert st == 0 and flags == 0
    want, kw, _ = run_oracle(x[:1], fmt, k, op)
    assert_bitwise(got[:1], want, f"2048^2 {fmt} k={k} {op}")


def test_bench_default_step_full_size_sampled(cuda_device):
    # the headline configuration as bench.py times it: 16 coils x 32 slices
    # 512x512 (the same seeded inputs), forward + round trip through one
    # graph-replayed executor run on tensor-core plans, and the radix-2 leg
    # on the same batches; sampled slices against the emulation of the
    # tensor-core variant (element-wise, bounded by each row's peak) and
    # against the oracle (bit for bit)
    import sys

    import bench
    import torch

    from paper_2512_04317_gb300 import mxfft
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import tc16_ref
    w = bench.WORKLOADS["multicoil_16x32_512x512"]
    ksp, img = bench.make_inputs(w, 0)
    assert ksp.shape == (512, 512, 512)
    xk, xi = torch.from_numpy(ksp).cuda(), torch.from_numpy(img).cuda()
    samples = [0, 301, 511]
    for tc in (True, False):
        yk, yi = torch.empty_like(xk), torch.empty_like(xi)
        with mxfft.Engine(graphs=True, tc16=tc) as eng:
            for _ in range(2):
                eng.run([("forward", xk, yk, "e4m3", 32), ("roundtrip", xi, yi, "e4m3", 32)])
            torch.cuda.synchronize()
            flags, _ = eng.status()
            assert flags == 0
            assert eng.launches_per_run() == 6
        for s in samples:
            if tc:
                for got, x, op in ((yk, ksp, "forward"), (yi, img, "roundtrip")):
                    g = got[s].cpu().numpy()
                    want = tc16_ref.mxfft2d(x[s:s + 1], "e4m3", op)[0]
                    err = np.abs(g.astype(np.complex128) - want)
                    peak = np.abs(want.astype(np.complex128)).max(axis=-1, keepdims=True)
                    rel = err / peak
                    assert rel.max() < 0.1 and np.mean(rel > 1e-5) < 1e-3, (s, op, rel.max())
            else:
                wk, _, _ = oracle.mxfft2d(ksp[s:s + 1], "e4m3", 32, op="forward")
                wi, _, _ = oracle.mxfft2d(img[s:s + 1], "e4m3", 32, op="roundtrip")
                assert_bitwise(yk[s:s + 1].cpu().numpy(), wk, f"C3 forward slice {s}")
                assert_bitwise(yi[s:s + 1].cpu().numpy(), wi, f"C3 round trip slice {s}")
