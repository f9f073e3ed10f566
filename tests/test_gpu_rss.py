"""Root-sum-of-squares coil combine of Eq. (1) on the GPU: bit for bit equal to
the oracle's combine, standalone (mxfft_rss), as an output of batch-executor
items (also on graph replays with other buffers) and of server requests."""
import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

pytestmark = pytest.mark.gpu


def same(a, b):
    np.testing.assert_array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


@pytest.mark.parametrize("images,coils,n0,n1", [(1, 1, 2, 2), (3, 16, 64, 64), (2, 5, 128, 32),
                                                 (4, 8, 256, 256), (1, 3, 2048, 8)])
def test_rss_kernel_equals_oracle(images, coils, n0, n1, cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    z = phantom.random_complex((images * coils, n0, n1), seed=images * 100 + coils, scale=1e3)
    got = mxfft.rss(torch.from_numpy(z).cuda(), coils).cpu().numpy()
    same(got, oracle.rss(z, coils))


def test_rss_of_phantom_coils(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    img = phantom.mri_batch(128, 128, 2, 16, config_id=51, domain="image")   # [2 * 16, 128, 128]
    got = mxfft.rss(torch.from_numpy(img).cuda(), 16).cpu().numpy()
    same(got, oracle.rss(img, 16))


@pytest.mark.parametrize("graphs", [False, True])
def test_engine_items_with_rss(graphs, cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    with mxfft.Engine(graphs=graphs) as eng:
        for seed in (1, 2):     # a replay of the same signature on other buffers
            k = torch.from_numpy(phantom.mri_batch(128, 128, 2, 4, config_id=60 + seed)).cuda()
            x = torch.from_numpy(phantom.mri_batch(64, 64, 1, 8, config_id=70 + seed,
                                                   domain="image")).cuda()
            yk, yx = torch.empty_like(k), torch.empty_like(x)
            rk = torch.empty((2, 128, 128), dtype=torch.float32, device="cuda")
            rx = torch.empty((1, 64, 64), dtype=torch.float32, device="cuda")
            eng.run([("forward", k, yk, "e4m3", 32, rk, 4), ("roundtrip", x, yx, "e5m2", 32, rx, 8)])
            torch.cuda.synchronize()
            assert eng.status()[0] == 0
            same(rk.cpu().numpy(), oracle.rss(yk.cpu().numpy(), 4))
            same(rx.cpu().numpy(), oracle.rss(yx.cpu().numpy(), 8))
            # and the transforms themselves equal the oracle's
            same(yk.cpu().numpy(), oracle.mxfft2d(k.cpu().numpy(), "e4m3", 32)[0])


def test_server_returns_rss_images(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(12):
        size = int(rng.choice([64, 128]))
        coils = int(rng.integers(1, 6))
        x = torch.from_numpy(phantom.mri_batch(size, size, 1, coils, config_id=80 + i)).pin_memory()
        reqs.append((i, x, coils, ["forward", "roundtrip"][i % 2], ["e4m3", "e5m2"][(i // 2) % 2]))
    results = {}
    for slots, mbs, one in ((1, 1, True), (4, 64, False)):
        outs = {i: torch.empty((1, x.shape[1], x.shape[2]), dtype=torch.float32).pin_memory()
                for i, x, *_ in reqs}
        with mxfft.Server(slots=slots, max_batch_slices=mbs) as srv:
            for i, x, coils, op, fmt in reqs:
                srv.submit(i, x, None, fmt, 32, op, rss=outs[i], coils=coils)
                if one:
                    assert srv.wait(60.0)
            assert srv.wait(60.0)
            done = srv.poll(100)
        assert len(done) == len(reqs) and all(c.status == 0 for c in done)
        results[one] = {i: o.numpy().copy() for i, o in outs.items()}
    for i, x, coils, op, fmt in reqs:
        same(results[True][i], results[False][i])
        want = oracle.rss(oracle.mxfft2d(x.numpy(), fmt, 32, op=op)[0], coils)
        same(results[False][i], want)
