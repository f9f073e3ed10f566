"""Ragged batch executor and autotuner on the GPU: an engine run over items
of different shapes, formats, block sizes and ops gives the same bits as the
per-plan calls (each of which matches the oracle bit for bit elsewhere), with
and without CUDA graphs, when a graph is replayed on other buffers, in place,
and under every tuned launch geometry."""
import json

import numpy as np
import pytest

import oracle
from paper_2512_04317_gb300 import phantom

pytestmark = pytest.mark.gpu

# (n0, n1, format, k, op, slices)
MIX = [
    (64, 128, "e4m3", 32, "forward", 3),
    (256, 256, "e5m2", 16, "roundtrip", 2),
    (128, 128, "e4m3", 32, "inverse", 1),
    (256, 256, "e5m2", 16, "forward", 2),     # same plan as item 2, other op
    (2048, 64, "e2m1", 64, "forward", 1),
    (512, 512, "e4m3", 32, "roundtrip", 1),
    (8, 4, "e3m2", 8, "roundtrip", 2),
    (256, 256, "e4m3", 32, "roundtrip_fused", 2),   # fused column kernel
    (128, 64, "e2m3", 64, "roundtrip_fused", 1),    # m = 32: fused columns, generic rows (n = 64)
]


def inputs(seed):
    import torch
    xs = []
    for i, (n0, n1, fmt, k, op, sl) in enumerate(MIX):
        x = phantom.random_complex((sl, n0, n1), seed=seed * 100 + i, scale=2.0 + i)
        xs.append(torch.from_numpy(x).cuda())
    return xs


def per_plan(xs):
    import torch

    from paper_2512_04317_gb300 import mxfft
    outs, ks = [], []
    for (n0, n1, fmt, k, op, sl), x in zip(MIX, xs):
        with mxfft.Plan(n0, n1, fmt, k) as p:
            y = getattr(p, op)(x)
            torch.cuda.synchronize()
            st, flags, kk = p.status()
            assert st == 0 and flags == 0
            outs.append(y.cpu().numpy())
            ks.extend(kk if op == "roundtrip" else [[v, 0] for v in kk])
    return outs, ks


def engine_run(eng, xs, in_place=False):
    import torch
    outs = [x if in_place else torch.empty_like(x) for x in xs]
    eng.run([(op, x, y, fmt, k) for (n0, n1, fmt, k, op, sl), x, y in zip(MIX, xs, outs)])
    torch.cuda.synchronize()
    flags, ks = eng.status()
    assert flags == 0
    return [y.cpu().numpy() for y in outs], ks


def assert_same(a, b):
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u.view(np.uint32), v.view(np.uint32))


@pytest.mark.parametrize("graphs", [False, True])
def test_engine_equals_per_plan_calls(graphs, cuda_device):
    from paper_2512_04317_gb300 import mxfft
    xs = inputs(1)
    want, kwant = per_plan(xs)
    with mxfft.Engine(graphs=graphs) as eng:
        got, k = engine_run(eng, xs)
        assert_same(got, want)
        assert k == kwant
        # same signature, other buffers and data: a graph is replayed with new tables
        xs2 = inputs(2)
        want2, _ = per_plan(xs2)
        got2, _ = engine_run(eng, xs2)
        assert_same(got2, want2)
        # and the first buffers once more
        got3, _ = engine_run(eng, xs)
        assert_same(got3, want)


def test_engine_in_place(cuda_device):
    from paper_2512_04317_gb300 import mxfft
    xs = inputs(3)
    want, _ = per_plan(xs)
    with mxfft.Engine(graphs=True) as eng:
        got, _ = engine_run(eng, [x.clone() for x in xs], in_place=True)
    assert_same(got, want)


def test_engine_tensor_core_plans(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(256, 256, 3, 1, config_id=41)).cuda()
    z = torch.from_numpy(phantom.random_complex((2, 64, 64), seed=5)).cuda()
    with mxfft.Plan(256, 256, "e4m3", 32, path="tc16") as p:
        want = p.roundtrip(x).cpu().numpy()
    with mxfft.Plan(64, 64, "e4m3", 32) as p:         # not covered by the tensor-core pass
        wantz = p.forward(z).cpu().numpy()
    with mxfft.Engine(tc16=True, graphs=True) as eng:
        y, w = torch.empty_like(x), torch.empty_like(z)
        eng.run([("roundtrip", x, y, "e4m3", 32), ("forward", z, w, "e4m3", 32)])
        torch.cuda.synchronize()
        assert eng.status()[0] == 0
    np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), want.view(np.uint32))
    np.testing.assert_array_equal(w.cpu().numpy().view(np.uint32), wantz.view(np.uint32))


def test_engine_rejects_bad_items(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.zeros(4, 64, 64, dtype=torch.complex64, device="cuda")
    with mxfft.Engine() as eng:
        bad = [
            mxfft.Item(64, 64, 0, 32, 0, 1, x.data_ptr() + 8, x.data_ptr() + 8),     # misaligned
            mxfft.Item(64, 64, 0, 32, 0, 2, x.data_ptr(), x.data_ptr() + 64 * 64 * 8),  # overlap
            mxfft.Item(48, 64, 0, 32, 0, 1, x.data_ptr(), x.data_ptr()),             # not 2^j
            mxfft.Item(64, 64, 9, 32, 0, 1, x.data_ptr(), x.data_ptr()),             # format
            mxfft.Item(64, 64, 0, 32, 5, 1, x.data_ptr(), x.data_ptr()),             # op
        ]
        for it in bad:
            with pytest.raises(mxfft.MxfftError) as ei:
                mxfft.mxfft_engine_run(eng.handle, [it], None)
            assert ei.value.status == mxfft.MXFFT_ERR_INVALID
        mxfft.mxfft_engine_run(eng.handle, [], None)   # nothing to do


@pytest.mark.parametrize("k", [32, 64, 128])
def test_tuned_geometries_give_the_same_bits(k, cuda_device, tmp_path):
    # groups of 16, 8 and 4 transforms (k = 32, 64, 128)
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(256, 256, 8, 1, config_id=42)).cuda()
    mxfft.mxfft_tune_clear()
    with mxfft.Plan(256, 256, "e4m3", k) as p:
        want = p.roundtrip(x).cpu().numpy()
        n = mxfft.mxfft_tune(p.handle, 8)
        assert n >= 2
        path = tmp_path / "tune.json"
        mxfft.mxfft_tune_save(str(path))
        entries = json.loads(path.read_text())["entries"]
        assert {e["dim"] for e in entries} == {0, 1}
        np.testing.assert_array_equal(p.roundtrip(x).cpu().numpy().view(np.uint32),
                                      want.view(np.uint32))
        # every candidate geometry, forced through the table
        for ng in (1, 2, 4):
            for e in entries:
                e["ng"] = ng
            path.write_text(json.dumps({"mxfft_tune": 1, "entries": entries}))
            mxfft.mxfft_tune_load(str(path))
            np.testing.assert_array_equal(p.roundtrip(x).cpu().numpy().view(np.uint32),
                                          want.view(np.uint32))
    mxfft.mxfft_tune_clear()


@pytest.mark.parametrize("n0,n1,batch,fmt,k", [(512, 512, 24, "e4m3", 32), (128, 1024, 9, "e5m2", 32),
                                               (1024, 256, 5, "e4m3", 64), (256, 512, 7, "e4m3", 128),
                                               (128, 128, 33, "e5m2", 64), (2048, 512, 2, "e4m3", 32)])
def test_tuned_tensor_core_geometry_gives_the_same_bits(n0, n1, batch, fmt, k, cuda_device, tmp_path):
    # the tensor-core pass on 256-thread CTAs (4096-point tiles) with 1 or 2
    # CTAs per SM and on 128-thread CTAs (2048-point tiles, n <= 1024) with 2
    # to 6: every geometry gives each vector, MX block and product the same
    # arithmetic
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(phantom.mri_batch(n0, n1, batch, 1, config_id=43, domain="image")).cuda()
    mxfft.mxfft_tune_clear()
    with mxfft.Plan(n0, n1, fmt, k, path="tc16") as p:
        want = p.roundtrip(x).cpu().numpy()
        fwd = p.forward(x).cpu().numpy()
        n_small = sum(1 for n in (n0, n1) if n <= 1024)
        assert mxfft.mxfft_tune(p.handle, batch) == 2 * 2 + 5 * n_small
        path = tmp_path / "tune.json"
        mxfft.mxfft_tune_save(str(path))
        entries = json.loads(path.read_text())["entries"]
        assert {(e["kind"], e["dim"]) for e in entries} == {(1, 0), (1, 1)}
        for tile, ctas in ((4096, 1), (4096, 2), (2048, 2), (2048, 3), (2048, 4), (2048, 6)):
            for e in entries:
                e["tile"] = tile if e["n"] <= 1024 else 4096
                e["ctas_per_sm"] = ctas if e["tile"] == tile else 2
            path.write_text(json.dumps({"mxfft_tune": 1, "entries": entries}))
            mxfft.mxfft_tune_load(str(path))
            np.testing.assert_array_equal(p.roundtrip(x).cpu().numpy().view(np.uint32),
                                          want.view(np.uint32))
            np.testing.assert_array_equal(p.forward(x).cpu().numpy().view(np.uint32),
                                          fwd.view(np.uint32))
            assert p.status()[1] == 0
    mxfft.mxfft_tune_clear()


def test_engine_many_groups_beyond_fork_streams(cuda_device):
    # 12 (plan, direction) groups share 8 fork streams; round trips of several
    # plans run as the second stage
    import torch

    from paper_2512_04317_gb300 import mxfft
    shapes = [(32, 64), (64, 32), (16, 16), (128, 64)]
    fmts = [("e4m3", 32), ("e5m2", 16), ("e2m3", 8)]
    work, want = [], []
    for i, (n0, n1) in enumerate(shapes):
        for j, (fmt, k) in enumerate(fmts):
            op = ["forward", "inverse", "roundtrip"][(i + j) % 3]
            x = phantom.random_complex((1 + (i + j) % 3, n0, n1), seed=500 + 10 * i + j, scale=5.0)
            xt = torch.from_numpy(x).cuda()
            work.append((op, xt, torch.empty_like(xt), fmt, k))
            want.append(oracle.mxfft2d(x, fmt, k, op=op)[0])
    with mxfft.Engine(graphs=True) as eng:
        for rep in range(2):
            eng.run(work)
            torch.cuda.synchronize()
            assert eng.status()[0] == 0
            for (op, xt, y, fmt, k), w in zip(work, want):
                assert_same([y.cpu().numpy()], [w])


def test_engine_hundreds_of_small_items(cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.random_complex((300, 8, 16), seed=77, scale=3.0)
    want = oracle.mxfft2d(x, "e4m3", 8, op="roundtrip")[0]
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    work = [("roundtrip", xt[i:i + 1], yt[i:i + 1], "e4m3", 8) for i in range(300)]
    with mxfft.Engine(graphs=False) as eng:
        eng.run(work)
        torch.cuda.synchronize()
    assert_same([yt.cpu().numpy()], [want])


def test_engine_graph_cache_eviction(cuda_device):
    # more signatures than the cache holds: the cache is cleared and rebuilt,
    # results stay exact
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = phantom.random_complex((70, 16, 16), seed=78, scale=2.0)
    want = oracle.mxfft2d(x, "e4m3", 16)[0]
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    with mxfft.Engine(graphs=True) as eng:
        for b in range(1, 71):          # 70 different slice counts = 70 signatures
            eng.run([("forward", xt[:b], yt[:b], "e4m3", 16)])
        torch.cuda.synchronize()
    assert_same([yt.cpu().numpy()], [want])


def _plan_reference(items):
    import torch

    from paper_2512_04317_gb300 import mxfft
    outs = []
    for op, x, fmt, k in items:
        with mxfft.Plan(x.shape[-2], x.shape[-1], fmt, k) as p:
            outs.append(getattr(p, op)(x).cpu().numpy())
    torch.cuda.synchronize()
    return outs


def test_ragged_mix_runs_in_six_launches_and_equals_plan_calls(cuda_device):
    # sizes 128..1024, non-square, three formats, all four ops in one run: the
    # radix-2 passes of every group go into one ragged launch per axis and stage
    import torch

    from paper_2512_04317_gb300 import mxfft
    shapes = [(128, 128), (256, 256), (512, 512), (1024, 1024), (256, 512), (128, 1024), (512, 128)]
    fmts = ["e4m3", "e5m2", "e2m3"]
    ops = ["forward", "inverse", "roundtrip", "roundtrip_fused"]
    items = []
    for i, (n0, n1) in enumerate(shapes):
        for j in range(2):
            op = ops[(i + j) % 4]
            dom = "image" if op.startswith("roundtrip") else "kspace"
            x = torch.from_numpy(phantom.mri_batch(n0, n1, 1 + (i + j) % 3, 1, config_id=70 + 2 * i + j,
                                                   domain=dom)).cuda()
            items.append((op, x, fmts[(i + 2 * j) % 3], 32))
    want = _plan_reference(items)
    for graphs in (False, True):
        for ragged in (True, False):
            with mxfft.Engine(graphs=graphs, ragged=ragged) as eng:
                outs = [torch.empty_like(x) for _, x, _, _ in items]
                for _ in range(2):
                    eng.run([(op, x, y, f, k) for (op, x, f, k), y in zip(items, outs)])
                    torch.cuda.synchronize()
                    if ragged:
                        assert eng.launches_per_run() == 6
                    for y, w in zip(outs, want):
                        np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), w.view(np.uint32))


def test_ragged_groups_beyond_one_launch_fall_back(cuda_device):
    # 60 (plan, direction) groups that fit the ragged launch: the first 48 go
    # into the ragged launches, the rest keep their own; every result is unchanged
    import torch

    from paper_2512_04317_gb300 import mxfft
    items = []
    shapes = [(128, 128), (256, 256), (512, 512), (1024, 1024), (128, 256), (256, 128)]
    for i, (n0, n1) in enumerate(shapes):
        for j, fmt in enumerate(["e4m3", "e5m2", "e2m3", "e3m2", "e2m1"]):
            for op in ("forward", "inverse"):
                x = torch.from_numpy(phantom.random_complex((1, n0, n1), seed=100 + 10 * i + j,
                                                            scale=2.0)).cuda()
                items.append((op, x, fmt, 32))
    want = _plan_reference(items)
    with mxfft.Engine(graphs=True) as eng:
        outs = [torch.empty_like(x) for _, x, _, _ in items]
        eng.run([(op, x, y, f, k) for (op, x, f, k), y in zip(items, outs)])
        torch.cuda.synchronize()
        assert eng.launches_per_run() > 3
    for y, w in zip(outs, want):
        np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), w.view(np.uint32))
