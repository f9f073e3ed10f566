"""Multi-GPU host logic of bench.py on CPU (gloo, world size 2): every rank
transforms its own slices (weak scaling, no data-path collective), the job time
is the slowest rank's, and the whole-job throughput sums all ranks' points."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = load_bench()
    w = dict(bench.WORKLOADS["single_128x128"])
    w.update(n0=16, n1=16, nslices=2)
    ksp, img = bench.make_inputs(w, rank)
    # rank r pretends its timed region took (r + 1) * 10 ms
    job_ms = bench.job_time_ms((rank + 1) * 10.0, world, dist, None)
    value = bench.job_throughput_mpts(world, ksp.shape[0] * 256, 3, 4, job_ms)
    digest = float(np.abs(ksp).sum() + np.abs(img).sum())
    out_q.put((rank, job_ms, value, digest, bench.rank_config_id(w, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, d0, c0), (r1, t1, v1, d1, c1) = res
    # the job time is the slowest rank's on every rank
    assert t0 == t1 == 20.0
    # whole-job throughput: 2 ranks x 2 slices x 256 points x 3 transforms x 4 steps / 20 ms
    assert v0 == v1 == pytest.approx(2 * 2 * 256 * 3 * 4 / 0.020 / 1e6)
    # ranks work on different slices (distinct seeds), nothing is exchanged
    assert c0 != c1 and d0 != d1


def test_single_rank_needs_no_process_group():
    bench = load_bench()
    assert bench.job_time_ms(12.5, 1) == 12.5
    assert bench.job_throughput_mpts(1, 1000, 3, 10, 1.0) == pytest.approx(30.0)
