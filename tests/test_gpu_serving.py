"""Request server with continuous batching: results are bit-identical whether
a request runs alone or admitted into a mix with others, device memory held by
admitted requests never exceeds the budget, and latencies are recorded for
p50 / p99 reporting."""
import time

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom

pytestmark = pytest.mark.gpu


def make_requests(n, seed, sizes=(64, 128, 256), max_coils=4):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        size = int(rng.choice(sizes))
        coils = int(rng.integers(1, max_coils + 1))
        fmt = ["e4m3", "e5m2"][int(rng.integers(0, 2))]
        op = ["forward", "roundtrip"][int(rng.integers(0, 2))]
        x = torch.from_numpy(phantom.random_complex((coils, size, size), seed=seed * 1000 + i,
                                                    scale=float(rng.uniform(0.5, 50.0))))
        reqs.append(dict(tag=i, x=x.pin_memory(), fmt=fmt, op=op))
    return reqs


def serve(reqs, slots, max_batch_slices, mem_budget=0, one_at_a_time=False):
    import torch

    from paper_2512_04317_gb300 import mxfft
    outs = {r["tag"]: torch.empty_like(r["x"]).pin_memory() for r in reqs}
    done = {}
    with mxfft.Server(slots=slots, max_batch_slices=max_batch_slices, mem_budget=mem_budget) as srv:
        for r in reqs:
            srv.submit(r["tag"], r["x"], outs[r["tag"]], r["fmt"], 32, r["op"])
            if one_at_a_time:
                assert srv.wait(60.0)
        assert srv.wait(120.0)
        for c in srv.poll(10 * len(reqs)):
            done[c.tag] = c
        stats = srv.stats()
    assert sorted(done) == [r["tag"] for r in reqs]
    return {t: outs[t].numpy() for t in outs}, done, stats


def test_results_same_alone_and_in_the_mix(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    reqs = make_requests(24, seed=11)
    alone, done_a, stats_a = serve(reqs, slots=1, max_batch_slices=1, one_at_a_time=True)
    mixed, done_m, stats_m = serve(reqs, slots=4, max_batch_slices=64)
    assert stats_a[0] == len(reqs)          # one batch per request
    assert stats_m[0] < len(reqs)           # requests were batched together
    for r in reqs:
        t = r["tag"]
        assert done_a[t].status == 0 and done_m[t].status == 0
        np.testing.assert_array_equal(alone[t].view(np.uint32), mixed[t].view(np.uint32))
    # and equal to the plan API for a few of them
    for r in reqs[:4]:
        x = r["x"].cuda()
        with mxfft.Plan(x.shape[-2], x.shape[-1], r["fmt"], 32) as p:
            want = getattr(p, r["op"])(x).cpu().numpy()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(mixed[r["tag"]].view(np.uint32), want.view(np.uint32))


def test_memory_budget_bounds_admission(cuda_device):
    reqs = make_requests(16, seed=12, sizes=(128,), max_coils=4)    # 128 KiB per coil
    budget = 3 * 4 * 128 * 128 * 8                                  # three largest requests
    _, done, (batches, peak, bud) = serve(reqs, slots=4, max_batch_slices=64, mem_budget=budget)
    assert bud == budget and 0 < peak <= budget
    assert all(c.status == 0 for c in done.values())


def test_request_larger_than_budget_fails_alone(cuda_device):
    from paper_2512_04317_gb300 import mxfft
    reqs = make_requests(3, seed=13, sizes=(64,), max_coils=1)
    big = make_requests(1, seed=14, sizes=(256,), max_coils=1)[0]
    big["tag"] = 99
    _, done, _ = serve(reqs + [big], slots=2, max_batch_slices=8, mem_budget=64 * 64 * 8 * 2)
    assert done[99].status == mxfft.MXFFT_ERR_NOMEM
    assert all(done[r["tag"]].status == 0 for r in reqs)


def test_poisson_arrivals_latency_record(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    reqs = make_requests(120, seed=15, sizes=(64, 128, 256))
    rng = np.random.default_rng(16)
    gaps = rng.exponential(200e-6, len(reqs))
    outs = [torch.empty_like(r["x"]).pin_memory() for r in reqs]
    with mxfft.Server(slots=4, max_batch_slices=64) as srv:
        t = time.perf_counter()
        for r, o, g in zip(reqs, outs, gaps):
            t += g
            while time.perf_counter() < t:
                pass
            srv.submit(r["tag"], r["x"], o, r["fmt"], 32, r["op"])
        assert srv.wait(120.0)
        done = srv.poll(1000)
    assert len(done) == len(reqs)
    lat = np.array([c.t_done_us - c.t_submit_us for c in done])
    assert all(c.status == 0 for c in done)
    assert all(c.t_submit_us <= c.t_admit_us <= c.t_done_us for c in done)
    p50, p99 = np.percentile(lat, [50, 99])
    assert 0 < p50 <= p99
