#!/usr/bin/env python
"""Benchmark of the MX-scaled low-precision 2D FFT on GB300.

One step = the whole hot path over one batch: the forward MX-FFT of a batch of
phantom k-space slices plus the round trip (forward then inverse) of the
matching image-domain batch: 3 transforms of every slice.  The value is
points x transforms per second (Mpts/s) of the whole job; inputs are resident
in HBM when the timed region starts and the L2 is flushed (a 256 MiB write)
between timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl mxfft|reference]

Under torchrun each rank runs the full batch on its own GPU (weak scaling, no
collective on the data path; the only collectives are the barrier and the
max-over-ranks of the timings).  --impl reference times the CPU oracle on the
host cores instead.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MXFP8 2D-FFT Mpts/s, % HBM roofline, NRMSE vs FP64, serving p50/p99"

WORKLOADS = {
    "batch64_256x256": dict(n0=256, n1=256, nslices=64, ncoils=1, fmt="e4m3", k=32, config_id=2,
                            desc="64 slices 256x256 complex64 phantom k-space, MXFP8 e4m3, "
                                 "k=32, tau=1e-3; forward + round trip"),
    "single_128x128": dict(n0=128, n1=128, nslices=1, ncoils=1, fmt="e4m3", k=32, config_id=1,
                           desc="single 128x128 phantom, MXFP8 e4m3, k=32; forward + round trip"),
    "multicoil_16x32_512x512": dict(n0=512, n1=512, nslices=32, ncoils=16, fmt="e4m3", k=32,
                                    config_id=3, desc="16 coils x 32 slices 512x512, MXFP8 e4m3, "
                                                      "k=32; forward + round trip"),
    "multicoil_16x4_1024x1024": dict(n0=1024, n1=1024, nslices=4, ncoils=16, fmt="e4m3", k=32,
                                     config_id=7, desc="16 coils x 4 slices 1024x1024, MXFP8 e4m3, "
                                                       "k=32; forward + round trip"),
    "large_8_2048x2048": dict(n0=2048, n1=2048, nslices=8, ncoils=1, fmt="e4m3", k=32,
                              config_id=5, desc="8 x 2048x2048 phantoms, MXFP8 e4m3, k=32; "
                                                "forward + round trip"),
}
DEFAULT_WORKLOAD = "multicoil_16x32_512x512"
TRANSFORMS_PER_STEP = 3          # forward + (forward + inverse) of the round trip
ALG_BYTES_PER_PT = 16            # read complex64 once + write once, per transform
PASS_BYTES_PER_PT = 8            # a row or column pass launch: half a transform's bytes
CPU_SUBSET_SLICES = 4            # fixed oracle sample for slices of 512x512 and more
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["mxfft", "reference"], default="mxfft")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--path", choices=["radix2", "tc16"], default="tc16",
                    help="tc16: radix-16 tcgen05 variant (within the stated NRMSE; the default "
                         "where the workload's shape allows it); radix2: the bit-exact radix-2 "
                         "MX path (always timed beside the headline)")
    ap.add_argument("--fused2d", action="store_true",
                    help="tensor-core path: the fused 2D kernel (MXFFT_OPT_FUSED2D: a whole "
                         "transform per launch on one thread-block cluster per slice) where the "
                         "shape allows it")
    ap.add_argument("--api", choices=["engine", "plan"], default="engine",
                    help="engine: one batch-executor run per step, replayed as a CUDA graph; "
                         "plan: mxfft_forward + mxfft_roundtrip calls")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-tuning", action="store_true",
                    help="ignore the autotuned launch geometries shipped with the package")
    ap.add_argument("--slices", type=int, default=0,
                    help="smaller case of a workload (profiling): about this many slices")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--fmt", choices=["e4m3", "e5m2", "e2m3", "e3m2", "e2m1", "fp16", "fp32"], default=None,
                    help="element format instead of the workload's (format / block-size sweeps)")
    ap.add_argument("--k", type=int, default=0,
                    help="MX block size k instead of the workload's (power of two, 2..128)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_config_id(w, rank):
    """Seed key of a rank's slices: every rank transforms its own full batch
    (weak scaling, independent slices, nothing exchanged on the data path)."""
    return w["config_id"] * 1000 + rank


def make_inputs(w, rank):
    from paper_2512_04317_gb300 import phantom
    cid = rank_config_id(w, rank)
    ksp = phantom.mri_batch(w["n0"], w["n1"], w["nslices"], w["ncoils"], config_id=cid)
    img = phantom.mri_batch(w["n0"], w["n1"], w["nslices"], w["ncoils"], config_id=cid,
                            domain="image")
    return ksp, img


def job_time_ms(local_ms, world, dist=None, device=None):
    """Job time = the slowest rank's time (max over ranks, one all_reduce)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput_mpts(world, pts_per_rank, transforms, steps, job_ms):
    """Whole-job points x transforms per second, in millions."""
    return world * pts_per_rank * transforms * steps / (job_ms * 1e-3) / 1e6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dtype_label(fmt):
    """The arithmetic the path computes in: MX element format + FP32."""
    if fmt == "fp16":
        return "fp16 products, f32 accumulate"
    if fmt == "fp32":
        return "f32 (reference ablation, no quantisation)"
    kind = {"e4m3": "mxfp8", "e5m2": "mxfp8", "e2m3": "mxfp6", "e3m2": "mxfp6",
            "e2m1": "mxfp4"}[fmt]
    return f"{kind}-{fmt} elements, e8m0 block scales, f32 accumulate"


def oracle_sample_slices(w, cores):
    """Slices of the oracle's bounded sample: the fixed 4-slice subset for
    slices of 512x512 and more, else one slice per core."""
    n = w["n0"] * w["n1"]
    total = w["nslices"] * w["ncoils"]
    if n >= 1 << 20:
        return 1
    if n >= 1 << 18:
        return min(total, CPU_SUBSET_SLICES)
    return min(total, max(cores, 1))


# sources each kernel is compiled from (its own file(s) and the shared headers)
KERNEL_SOURCES = {
    "fast_pass_kernel": ("mx_fast", "mx_device.cuh", "mx_internal.h"),
    "pass_kernel": ("mx_pass.cu", "mx_device.cuh", "mx_internal.h"),
    "tc16_pass_kernel": ("mx_tc16.cu", "mx_tcgen05.cuh", "mx_device.cuh", "mx_internal.h"),
    "tc2d_kernel": ("mx_tc2d.cu", "mx_tcgen05.cuh", "mx_device.cuh", "mx_internal.h"),
    "stats_kernel": ("mx_stats.cu", "mx_device.cuh", "mx_internal.h"),
}


def source_digest(kernel, read=None):
    """Digest of the sources of one kernel (see KERNEL_SOURCES)."""
    csrc = os.path.join(ROOT, "paper_2512_04317_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(csrc, name), "rb") as f:
                return f.read()
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")) and name.startswith(KERNEL_SOURCES[kernel]):
            h.update(name.encode() + b"\0" + read(name))
    return h.hexdigest()[:16]


def recorded_lane_instructions(kernel, workload):
    """Executed lane instructions per point of a launch (ncu) of this kernel on
    this workload, when taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    for ent in rec.get("entries", []):
        if (ent.get("kernel") == kernel and ent.get("workload") == workload and
                ent.get("source_digest") == source_digest(kernel) and
                ent.get("lane_instructions_per_point_per_launch") is not None):
            return float(ent["lane_instructions_per_point_per_launch"])
    return None


def recorded_traffic(kernel, workload, pts_per_launch):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload, when it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    for ent in rec.get("entries", []):
        if (ent.get("kernel") == kernel and ent.get("workload") == workload and
                ent.get("source_digest") == source_digest(kernel) and
                ent.get("dram_bytes_per_point_per_launch") is not None):
            return float(ent["dram_bytes_per_point_per_launch"]) * pts_per_launch
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def run_reference(args, w, world, rank):
    """The CPU oracle timed on the host cores on a bounded sample per step."""
    if world > 1 and rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2512_04317_gb300 import phantom
    oracle.build()
    ns = oracle_sample_slices(w, oracle.num_threads())
    cores = min(oracle.num_threads(), ns)       # OpenMP runs over the sample's slices
    n0, n1 = w["n0"], w["n1"]
    ksp = phantom.mri_batch(n0, n1, ns, 1, config_id=w["config_id"])
    img = phantom.mri_batch(n0, n1, ns, 1, config_id=w["config_id"], domain="image")
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.mxfft2d(ksp, w["fmt"], w["k"], op="forward")
        oracle.mxfft2d(img, w["fmt"], w["k"], op="roundtrip")
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    pts = ns * n0 * n1 * TRANSFORMS_PER_STEP
    value = pts * len(times) / total / 1e6
    sample = f"{ns} of {w['nslices'] * w['ncoils']} slices per step, forward + round trip"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(w["fmt"]),
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(w, ksp, img):
    import oracle
    n0, n1 = w["n0"], w["n1"]
    if n0 * n1 >= 1 << 18:
        # the fixed subset of the large configurations
        ns = min(ksp.shape[0], CPU_SUBSET_SLICES)
    else:
        # bounded sample: about 10-30 s of CPU work
        per_slice_core_s = 0.3 * (n0 * n1) / 65536 * max(1.0, (n0 * n1) ** 0.5 / 256) ** 0.1
        ns = int(max(1, min(ksp.shape[0], 25.0 / per_slice_core_s)))
    cores = min(oracle.num_threads(), ns)       # OpenMP runs over the sample's slices
    # whole passes over the sample until at least 10 s (at most ~30 s) of wall time
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.mxfft2d(ksp[:ns], w["fmt"], w["k"], op="forward")
        oracle.mxfft2d(img[:ns], w["fmt"], w["k"], op="roundtrip")
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= 10.0 or dt * (reps + 1) / reps > 30.0:
            break
    return {"value": reps * ns * n0 * n1 * TRANSFORMS_PER_STEP / dt / 1e6, "unit": "Mpts/s",
            "cores": cores, "kind": "oracle",
            "sample": f"{ns} of {ksp.shape[0]} slices, forward + round trip, {reps} passes, "
                      f"{dt:.2f} s wall"}


SERVING_SIZES = (128, 256, 512, 1024)
SERVING_FRACTIONS = (0.3, 0.5, 0.7, 0.9)


def serving_requests(n, seed=20251204):
    """The serving mix: sizes uniform in {128, 256, 512, 1024}^2, 1-16 coils,
    e4m3 / e5m2, k = 32, forward or round trip, Poisson arrivals (unit rate)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = rng.choice(SERVING_SIZES, n)
    coils = rng.integers(1, 17, n)
    fmts = rng.choice(["e4m3", "e5m2"], n)
    ops = rng.choice(["forward", "roundtrip"], n)
    gaps = rng.exponential(1.0, n)
    return [dict(size=int(sizes[i]), coils=int(coils[i]), fmt=str(fmts[i]), op=str(ops[i]),
                 gap=float(gaps[i])) for i in range(n)]


def _pct(lat_ms):
    import numpy as np
    p50, p99 = np.percentile(lat_ms, [50, 99])
    return float(p50), float(p99)


def serving_leg(n_req, torch, slots=8, batch_slices=64, batch_mb=64, fp32=True,
                fractions=SERVING_FRACTIONS, rates=None, rss=True, tc16=False, ragged=True):
    """Continuous-batching server under the serving mix: saturated rate, then
    Poisson arrivals at fractions of it, p50 / p99 latency (submit to result in
    host memory); the plain FP32 per-slice GPU path (torch.fft, one call per
    coil slice, FIFO on one stream) under the same arrivals as comparator."""
    from paper_2512_04317_gb300 import mxfft, phantom
    reqs = serving_requests(n_req)
    pool = 4
    h_in, h_out = {}, {}
    for sz in SERVING_SIZES:
        x = phantom.mri_batch(sz, sz, 1, 16, config_id=4000 + sz)
        h_in[sz] = torch.from_numpy(x).pin_memory()
        if rss:   # one RSS image per request
            h_out[sz] = [torch.empty((1, sz, sz), dtype=torch.float32).pin_memory()
                         for _ in range(pool)]
        else:
            h_out[sz] = [torch.empty_like(h_in[sz]).pin_memory() for _ in range(pool)]
    work = [r["coils"] * r["size"] ** 2 * (3 if r["op"] == "roundtrip" else 1) for r in reqs]
    pts_total = sum(r["coils"] * r["size"] ** 2 * (2 if r["op"] == "roundtrip" else 1)
                    for r in reqs)

    def run_mx(rate):
        with mxfft.Server(slots=slots, max_batch_slices=batch_slices,
                          max_batch_bytes=batch_mb << 20, tc16=tc16, ragged=ragged) as srv:
            # plans of every (size, format) resident before the clock starts
            def submit(tag, sz, c, fmt, op, slot):
                if rss:
                    srv.submit(tag, h_in[sz][:c], None, fmt, 32, op, rss=h_out[sz][slot], coils=c)
                else:
                    srv.submit(tag, h_in[sz][:c], h_out[sz][slot][:c], fmt, 32, op)
            for i, sz in enumerate(SERVING_SIZES):
                for f in ("e4m3", "e5m2"):
                    submit(10 ** 6 + 2 * i + (f == "e5m2"), sz, 1, f, "roundtrip", 0)
            srv.wait(60.0)
            srv.poll(100)
            t = time.perf_counter()
            t0 = t
            for i, r in enumerate(reqs):
                if rate:
                    t += r["gap"] / rate
                    while time.perf_counter() < t:
                        pass
                submit(i, r["size"], r["coils"], r["fmt"], r["op"], i % pool)
            assert srv.wait(600.0)
            wall = time.perf_counter() - t0
            done = srv.poll(len(reqs) + 16)
            batches, peak, budget = srv.stats()
        lat = [(c.t_done_us - c.t_submit_us) / 1e3 for c in done if c.tag < 10 ** 6]
        assert len(lat) == len(reqs) and all(c.status == 0 for c in done)
        return wall, lat, batches

    def run_fp32(rate):
        dev = torch.device("cuda")
        d = {sz: torch.empty_like(h_in[sz], device=dev) for sz in SERVING_SIZES}
        arrivals = []
        t = time.perf_counter()
        for r in reqs:
            if rate:
                t += r["gap"] / rate
            arrivals.append(t)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        base = arrivals[0] if rate else t0
        arrivals = [t0 + (a - base) if rate else t0 for a in arrivals]
        lat = []
        for i, r in enumerate(reqs):
            while time.perf_counter() < arrivals[i]:
                pass
            sz, c = r["size"], r["coils"]
            x = d[sz][:c]
            x.copy_(h_in[sz][:c], non_blocking=True)
            for j in range(c):
                y = torch.fft.fft2(x[j])
                if r["op"] == "roundtrip":
                    y = torch.fft.ifft2(y)
                x[j].copy_(y)
            if rss:
                h_out[sz][i % pool].copy_(torch.sqrt((x.abs() ** 2).sum(0, keepdim=True)),
                                          non_blocking=True)
            else:
                h_out[sz][i % pool][:c].copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - arrivals[i]) * 1e3)
        return time.perf_counter() - t0, lat

    out = {"requests": n_req, "mix": "sizes {128,256,512,1024}^2, 1-16 coils, e4m3/e5m2, "
                                     "k=32, forward/roundtrip, Poisson arrivals",
           "latency": "submit to result in pinned host memory",
           "result": "one root-sum-of-squares image per request (Eq. (1))" if rss
                     else "the complex coil images",
           "server": f"{slots} slots, batches of at most {batch_slices} slices and "
                     f"{batch_mb} MiB, memory budget 80% of free",
           "path": "tensor-core plans where a request's shape allows them (128-1024), radix-2 "
                   "otherwise" if tc16 else "radix-2"}
    # no garbage-collector pauses in the submitting loop while it keeps time
    gc.collect()
    gc_was_enabled = gc.isenabled()
    gc.disable()
    run_mx(0.0)                      # warm-up phase (first use of kernels and plans), not reported
    wall, lat, batches = run_mx(0.0)
    sat = n_req / wall
    out["saturated"] = {"req_per_s": sat, "mpts_per_s": pts_total / wall / 1e6,
                        "batches": batches, "p50_ms": _pct(lat)[0], "p99_ms": _pct(lat)[1]}
    fsat = None
    if fp32:
        fw, flat = run_fp32(0.0)
        fsat = n_req / fw
        out["fp32_per_slice_saturated"] = {"req_per_s": fsat,
                                           "mpts_per_s": pts_total / fw / 1e6,
                                           "p50_ms": _pct(flat)[0], "p99_ms": _pct(flat)[1]}
    # Poisson arrivals at fractions of the MX server's saturated rate, every
    # phase run twice (repeat spread of p99); the FP32 path under the same
    # arrivals is far past its own capacity there (queue growth)
    out["poisson"] = []
    for frac in (rates if rates else fractions):
        rate = frac if rates else frac * sat
        reps = []
        for _ in range(2):
            wall, lat, batches = run_mx(rate)
            reps.append((_pct(lat), batches, pts_total / wall / 1e6))
        p99s = [r[0][1] for r in reps]
        ent = {"load": frac, "req_per_s": rate,
               "mx": {"p50_ms": reps[-1][0][0], "p99_ms": reps[-1][0][1],
                      "p50_ms_repeats": [r[0][0] for r in reps], "p99_ms_repeats": p99s,
                      "p99_spread": max(p99s) / max(min(p99s), 1e-9),
                      "batches": reps[-1][1], "mpts_per_s": reps[-1][2]}}
        if fp32:
            fw, flat = run_fp32(rate)
            f50, f99 = _pct(flat)
            ent["fp32_per_slice"] = {"p50_ms": f50, "p99_ms": f99,
                                     "mpts_per_s": pts_total / fw / 1e6,
                                     "note": "same arrivals: above the FP32 path's capacity"}
        out["poisson"].append(ent)
    # like for like: arrivals at fractions of the FP32 path's own saturated
    # rate, each path at the same arrival times
    if fp32 and not rates:
        out["poisson_at_fp32_load"] = []
        for frac in fractions:
            rate = frac * fsat
            fw, flat = run_fp32(rate)
            wall, lat, batches = run_mx(rate)
            out["poisson_at_fp32_load"].append({
                "load_of_fp32_capacity": frac, "req_per_s": rate,
                "fp32_per_slice": {"p50_ms": _pct(flat)[0], "p99_ms": _pct(flat)[1]},
                "mx": {"p50_ms": _pct(lat)[0], "p99_ms": _pct(lat)[1], "batches": batches}})
    if gc_was_enabled:
        gc.enable()
    del work
    return out


def ssim(a, b, data_range):
    """SSIM (Wang et al. 2004): Gaussian window sigma 1.5 (11 x 11), K1 0.01,
    K2 0.03, mean over the image; a is the reference."""
    from scipy.ndimage import gaussian_filter
    g = lambda z: gaussian_filter(z, 1.5, truncate=3.5)
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    ma, mb = g(a), g(b)
    va, vb, cab = g(a * a) - ma * ma, g(b * b) - mb * mb, g(a * b) - ma * mb
    s = ((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))
    return float(s.mean())


def rss_image_metrics(torch, n=256, slices=2, coils=8):
    """Eq. (1) evaluation as in Sec. 2.3: PSNR / SSIM / NMSE of root-sum-of-
    squares images of the per-coil transforms against FP64, for MXFP8 e4m3 and
    e5m2 (k = 32) and the FP16 positive control; forward from k-space and round
    trip from the coil images."""
    import numpy as np

    from paper_2512_04317_gb300 import mxfft, phantom
    ksp = phantom.mri_batch(n, n, slices, coils, config_id=6)
    img = phantom.mri_batch(n, n, slices, coils, config_id=6, domain="image")
    def rss64(z):
        return np.sqrt((np.abs(z.reshape(slices, coils, n, n)) ** 2).sum(axis=1))
    refs = {"forward": rss64(np.fft.fft2(ksp.astype(np.complex128))),
            "roundtrip": rss64(img.astype(np.complex128))}
    out = {}
    for fmt in ("e4m3", "e5m2", "fp16", "fp32"):
        for op, x in (("forward", ksp), ("roundtrip", img)):
            with mxfft.Plan(n, n, fmt, 32) as p:
                y = getattr(p, op)(torch.from_numpy(x).cuda())
                r = mxfft.rss(y, coils).cpu().numpy().astype(np.float64)
            ref = refs[op]
            nm, ps, ss = [], [], []
            for s_ in range(slices):
                err = r[s_] - ref[s_]
                nm.append(float((err ** 2).sum() / (ref[s_] ** 2).sum()))
                ps.append(float(20 * np.log10(ref[s_].max() / np.sqrt((err ** 2).mean()))))
                ss.append(ssim(ref[s_], r[s_], float(ref[s_].max())))
            out[f"{fmt}_{op}"] = {"psnr_db": float(np.mean(ps)), "ssim": float(np.mean(ss)),
                                  "nmse": float(np.mean(nm))}
    return {"images": f"{slices} slices x {coils} coils {n}x{n} phantom, RSS of the per-coil "
                      "transforms (Eq. (1)), mean over slices", "metrics": out}


def accuracy(plan, xk, xi, torch):
    """NRMSE / PSNR of the forward and round trip against FP64 (cuFFT double)."""
    y = plan.forward(xk)
    z = plan.roundtrip(xi)
    ref = torch.fft.fft2(xk.to(torch.complex128))
    def nrmse(a, r):
        return float(torch.linalg.vector_norm((a.to(torch.complex128) - r).flatten()) /
                     torch.linalg.vector_norm(r.flatten()))
    def psnr(a, r):
        err = (a.to(torch.complex128) - r).abs()
        rms = float(torch.sqrt(torch.mean(err ** 2)))
        return 20.0 * float(torch.log10(r.abs().max() / rms))
    xi64 = xi.to(torch.complex128)
    out = {"forward_nrmse": nrmse(y, ref), "forward_psnr_db": psnr(y, ref),
           "roundtrip_nrmse": nrmse(z, xi64), "roundtrip_psnr_db": psnr(z, xi64)}
    if plan.fmt != "fp16":
        f = plan.roundtrip_fused(xi)
        out.update({"roundtrip_fused_nrmse": nrmse(f, xi64),
                    "roundtrip_fused_psnr_db": psnr(f, xi64)})
    return out


def timed_steps(torch, run, steps, flush, stream, world, dist, dev, barrier):
    """Device time of `steps` calls of run(): CUDA events on the launch stream
    around each step, L2 flushed between steps (outside the events), barrier
    and synchronize on both sides, max over ranks.  Returns the job ms."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    barrier()
    for i in range(steps):
        flush.fill_(i & 0xff)
        evs[i][0].record(stream)
        run()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    return job_time_ms(sum(a.elapsed_time(b) for a, b in evs), world, dist, dev)


def main():
    args = parse()
    w = dict(WORKLOADS[args.workload])
    if args.slices > 0:
        w["nslices"] = max(1, -(-args.slices // w["ncoils"]))
        w["desc"] += f" (reduced to {w['nslices'] * w['ncoils']} slices)"
    if args.fmt or args.k:
        w["fmt"] = args.fmt or w["fmt"]
        w["k"] = args.k or w["k"]
        w["desc"] += f" (run with format {w['fmt']}, k={w['k']})"
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, w, world, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2512_04317_gb300 import build as _b
    from paper_2512_04317_gb300 import mxfft
    _b.build()
    mxfft.load()

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tuning = None
    tfile = os.path.join(ROOT, "paper_2512_04317_gb300", "tuning", "gb300_sm103a.json")
    if not args.no_tuning and os.path.exists(tfile):
        mxfft.mxfft_tune_load(tfile)     # launch geometries measured by mxfft_tune
        tuning = os.path.relpath(tfile, ROOT)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    n0, n1 = w["n0"], w["n1"]
    # the tensor-core variant where the shape, format and k allow it, else radix-2
    path = args.path
    if path == "tc16" and not mxfft.tc16_supported(n0, n1, w["fmt"], w["k"]):
        path = "radix2"
    ksp_np, img_np = make_inputs(w, rank)
    batch = ksp_np.shape[0]
    pts = batch * n0 * n1
    xk = torch.from_numpy(ksp_np).to(dev)
    xi = torch.from_numpy(img_np).to(dev)
    yk = torch.empty_like(xk)
    yi = torch.empty_like(xi)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    fused2d = args.fused2d and path == "tc16"
    plan = mxfft.Plan(n0, n1, w["fmt"], w["k"], path=path, fused2d=fused2d)
    stream = torch.cuda.current_stream(dev)
    engine = None
    if args.api == "engine":
        # one run per step: a statistics launch over both batches, the forward
        # passes of both as one launch per axis, then the round trip's
        # statistics and inverse passes; captured once, replayed as a graph
        engine = mxfft.Engine(graphs=True, tc16=path == "tc16", fused2d=fused2d)
        work = [("forward", xk, yk, w["fmt"], w["k"]), ("roundtrip", xi, yi, w["fmt"], w["k"])]

        def step():
            engine.run(work)
        launches_per_step = 6
    else:
        def step():
            plan.forward(xk, out=yk)
            plan.roundtrip(xi, out=yi)
        launches_per_step = 3 + 6   # forward: stats, rows, cols; round trip: twice that

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if engine is not None:
        launches_per_step = engine.launches_per_run()   # kernels of the replayed graph

    # ---- device-timed region: K steps, L2 flushed between them ----------------
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    wall0 = time.perf_counter()
    t_ms = timed_steps(torch, step, args.steps, flush, stream, world, dist, dev, barrier)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ms_per_step = t_ms / args.steps
    value = job_throughput_mpts(world, pts, TRANSFORMS_PER_STEP, args.steps, t_ms)

    # ---- the same step with the fused round trip (Sec. 4.3 variant: one
    # prescale, both column transforms of a tile in one launch, no second
    # statistics pass), timed the same way -----------------------------------
    fused = None
    if engine is not None and w["fmt"] != "fp16":
        yf = torch.empty_like(xi)
        work_f = [("forward", xk, yk, w["fmt"], w["k"]),
                  ("roundtrip_fused", xi, yf, w["fmt"], w["k"])]
        for _ in range(args.warmup):
            engine.run(work_f)
        tf_ms = timed_steps(torch, lambda: engine.run(work_f), args.steps, flush, stream, world,
                            dist, dev, barrier)
        fused = {"value": job_throughput_mpts(world, pts, TRANSFORMS_PER_STEP, args.steps, tf_ms),
                 "unit": "Mpts/s", "ms_per_step": tf_ms / args.steps,
                 "speedup_vs_separate_round_trip": ms_per_step / (tf_ms / args.steps),
                 "launches_per_step": engine.launches_per_run(),
                 "step": "forward of the k-space batch + fused round trip of the image batch"}

    # ---- the other path on the same workload and step, timed the same way:
    # beside the tensor-core headline the bit-exact radix-2 path of Alg. 2,
    # beside a radix-2 headline the tensor-core variant --------------------------
    other_leg = None
    other = "radix2" if path == "tc16" else "tc16"
    if engine is not None and (other == "radix2" or
                               mxfft.tc16_supported(n0, n1, w["fmt"], w["k"])):
        eng_o = mxfft.Engine(graphs=True, tc16=other == "tc16")
        yok, yoi = torch.empty_like(xk), torch.empty_like(xi)
        work_o = [("forward", xk, yok, w["fmt"], w["k"]), ("roundtrip", xi, yoi, w["fmt"], w["k"])]
        for _ in range(args.warmup):
            eng_o.run(work_o)
        to_ms = timed_steps(torch, lambda: eng_o.run(work_o), args.steps, flush, stream, world,
                            dist, dev, barrier)
        to_step = to_ms / args.steps
        with mxfft.Plan(n0, n1, w["fmt"], w["k"], path=other) as po:
            o_acc = accuracy(po, xk, xi, torch)
        other_leg = {"path": other,
                     "value": job_throughput_mpts(world, pts, TRANSFORMS_PER_STEP, args.steps, to_ms),
                     "unit": "Mpts/s", "ms_per_step": to_step,
                     "hbm_roofline_frac_per_transform":
                         pts * TRANSFORMS_PER_STEP * ALG_BYTES_PER_PT / (to_step * 1e-3) / 1e9
                         / load_peaks()[0],
                     "accuracy_vs_fp64": o_acc,
                     "launches_per_step": eng_o.launches_per_run(),
                     "bit_exact_with_oracle": other == "radix2",
                     "step": "the same engine run (forward + round trip) on this path's plans"}
        eng_o.close()

    # ---- per-kernel device time (event pairs around each launch on the launch
    # stream; the same kernels through the plan calls, since launches inside a
    # graph cannot be bracketed one by one) ------------------------------------
    mxfft.mxfft_profile(plan.handle, True)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        plan.forward(xk, out=yk)
        plan.roundtrip(xi, out=yi)
    torch.cuda.synchronize()
    mxfft.mxfft_profile(plan.handle, False)
    prof = mxfft.mxfft_profile_read(plan.handle)
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    avg_ms = dom_ms / max(dom_n, 1)
    peak, peak_src = load_peaks()
    # the headline fraction counts 16 B per point per transform (read the
    # complex64 input once, write the output once) over the step's device time
    whole_gbs = pts * TRANSFORMS_PER_STEP * ALG_BYTES_PER_PT / (ms_per_step * 1e-3) / 1e9
    # the dominant kernel per launch, at its own algorithmic bytes: 8 B per
    # point for a statistics launch (read) and for a row or column pass
    # (half a transform), 16 B per point for a whole-transform launch
    dom_bpp = mxfft.KERNEL_ALG_BYTES_PER_PT.get(dom, PASS_BYTES_PER_PT)
    dom_gbs = dom_bpp * pts / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": whole_gbs, "peak": peak, "unit": "GB/s",
                "frac": whole_gbs / peak,
                "traffic": recorded_traffic(dom, args.workload, pts),
                "basis": f"{ALG_BYTES_PER_PT} B per point per transform x {pts} points x "
                         f"{TRANSFORMS_PER_STEP} transforms / ms_per_step",
                "kernel": dom, "avg_launch_ms": avg_ms, "peak_source": peak_src,
                "dominant_kernel": {"kernel": dom, "avg_launch_ms": avg_ms, "launches": dom_n,
                                    "alg_bytes_per_point_per_launch": dom_bpp,
                                    "achieved": dom_gbs, "frac": dom_gbs / peak},
                "kernel_share": {k: v[0] / max(sum(x[0] for x in prof.values()), 1e-12)
                                 for k, v in prof.items()}}
    # instruction-issue roofline of the same kernel: one warp instruction per
    # scheduler and cycle, 4 schedulers of 32 lanes per SM, at the sampled clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    alu_peak = sms * 4 * 32 * mhz * 1e6 / 1e12
    ipp = recorded_lane_instructions(dom, args.workload)
    roofline_alu = None
    if ipp is not None:
        ach = ipp * pts / (avg_ms * 1e-3) / 1e12
        roofline_alu = {"bound": "alu", "achieved": ach, "peak": alu_peak,
                        "unit": "T lane-instructions/s", "frac": ach / alu_peak, "kernel": dom,
                        "lane_instructions_per_point": ipp,
                        "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz"}

    # ---- end to end through the public API with host buffers ------------------
    hk = torch.from_numpy(ksp_np).pin_memory()
    hi = torch.from_numpy(img_np).pin_memory()
    ok = torch.empty_like(hk).pin_memory()
    oi = torch.empty_like(hi).pin_memory()
    e2e_steps = max(6, min(args.steps, 60))
    e2e_mode = "one stream, steps in sequence"
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if engine is not None:
        # the way a caller streams batches through the executor: one stream
        # copies inputs in, one copies results out, and steps rotate over 3
        # device buffer sets, each with its own compute stream and engine, so
        # the two copy directions run back to back and at the same time while
        # the transforms overlap them; every step still copies its inputs in
        # and its results out.  Events order a buffer set's reuse.
        e2e_mode = "copy-in stream, copy-out stream, 3 buffer sets with a compute stream each"
        h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        lanes = []
        for j in range(3):
            b = {"xk": torch.empty_like(xk), "xi": torch.empty_like(xi), "yk": torch.empty_like(yk),
                 "yi": torch.empty_like(yi), "ok": torch.empty_like(hk).pin_memory(),
                 "oi": torch.empty_like(hi).pin_memory(),
                 "in_done": torch.cuda.Event(), "run_done": torch.cuda.Event(),
                 "out_done": torch.cuda.Event()}
            lanes.append((torch.cuda.Stream(dev), mxfft.Engine(graphs=True, tc16=path == "tc16",
                                                               fused2d=fused2d), b))

        def e2e_step(i):
            st_, eng_j, b = lanes[i % len(lanes)]
            if i >= len(lanes):
                h2d_s.wait_event(b["run_done"])      # the set's inputs were consumed
            with torch.cuda.stream(h2d_s):
                b["xk"].copy_(hk, non_blocking=True)
                b["xi"].copy_(hi, non_blocking=True)
            b["in_done"].record(h2d_s)
            st_.wait_event(b["in_done"])
            if i >= len(lanes):
                st_.wait_event(b["out_done"])        # the set's outputs were copied out
            with torch.cuda.stream(st_):
                eng_j.run([("forward", b["xk"], b["yk"], w["fmt"], w["k"]),
                           ("roundtrip", b["xi"], b["yi"], w["fmt"], w["k"])])
            b["run_done"].record(st_)
            d2h_s.wait_event(b["run_done"])
            with torch.cuda.stream(d2h_s):
                b["ok"].copy_(b["yk"], non_blocking=True)
                b["oi"].copy_(b["yi"], non_blocking=True)
            b["out_done"].record(d2h_s)
        for i in range(2 * len(lanes)):
            e2e_step(i)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for st_ in [h2d_s, d2h_s] + [ln[0] for ln in lanes]:
            st_.wait_event(e0)
        for i in range(e2e_steps):
            e2e_step(i + 2 * len(lanes))
        for st_ in [h2d_s, d2h_s] + [ln[0] for ln in lanes]:
            ev = torch.cuda.Event()
            ev.record(st_)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        for _, eng_j, _ in lanes:
            eng_j.close()
    else:
        for i in range(2):
            xk.copy_(hk, non_blocking=True); xi.copy_(hi, non_blocking=True)
            step()
            ok.copy_(yk, non_blocking=True); oi.copy_(yi, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for i in range(e2e_steps):
            xk.copy_(hk, non_blocking=True)
            xi.copy_(hi, non_blocking=True)
            step()
            ok.copy_(yk, non_blocking=True)
            oi.copy_(yi, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
    te_ms = job_time_ms(e0.elapsed_time(e1), world, dist, dev)
    e2e_value = job_throughput_mpts(world, pts, TRANSFORMS_PER_STEP, e2e_steps, te_ms)
    bytes_io = 2 * pts * 8

    # ---- the step's results equal the plan calls bit for bit -------------------
    same = None
    if engine is not None:
        xk.copy_(torch.from_numpy(ksp_np).to(dev))
        xi.copy_(torch.from_numpy(img_np).to(dev))
        step()
        a = torch.cat([yk.view(torch.int32).flatten(), yi.view(torch.int32).flatten()])
        plan.forward(xk, out=yk)
        plan.roundtrip(xi, out=yi)
        b = torch.cat([yk.view(torch.int32).flatten(), yi.view(torch.int32).flatten()])
        same = bool(torch.equal(a, b))

    # ---- accuracy and the FP32 comparator (context) ----------------------------
    acc = accuracy(plan, xk, xi, torch)
    st, flags, _ = plan.status()
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    c0.record(stream)
    for _ in range(reps):
        for s in range(batch):
            torch.fft.fft2(xk[s])
            torch.fft.ifft2(torch.fft.fft2(xi[s]))
    c1.record(stream)
    torch.cuda.synchronize()
    per_slice_fp32 = pts * TRANSFORMS_PER_STEP * reps / (c0.elapsed_time(c1) * 1e-3) / 1e6
    c0.record(stream)
    for _ in range(reps):
        torch.fft.fft2(xk)
        torch.fft.ifft2(torch.fft.fft2(xi))
    c1.record(stream)
    torch.cuda.synchronize()
    batched_fp32 = pts * TRANSFORMS_PER_STEP * reps / (c0.elapsed_time(c1) * 1e-3) / 1e6

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, ksp_np, img_np)
    serving = None
    if world == 1 and not args.no_serving:
        serving = serving_leg(args.serving_requests, torch, tc16=path == "tc16")
    rss_acc = rss_image_metrics(torch) if rank == 0 else None

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(w["fmt"]), "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"],
                       "path": path + ("+fused2d" if fused2d else ""),
                       "api": args.api, "tuning": tuning,
                       "n0": n0, "n1": n1,
                       "batch_per_gpu": batch, "format": w["fmt"], "k": w["k"],
                       "transforms_per_step": TRANSFORMS_PER_STEP,
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "other_path": other_leg,
            "roofline_alu": roofline_alu,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Mpts/s", "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io, "steps": e2e_steps, "mode": e2e_mode},
            "gpu_launches": launches_per_step * args.steps,
            "launches_per_step": launches_per_step,
            "accuracy_vs_fp64": acc,
            "device_status": st,
            "fp32_cufft_comparator": {"per_slice_mpts_s": per_slice_fp32,
                                      "batched_mpts_s": batched_fp32},
            "clocks": clk,
            "wall_s_timed_region": wall,
            "engine_equals_plan_calls": same,
            "fused_roundtrip_variant": fused,
            "rss_image_accuracy_vs_fp64": rss_acc,
            "serving": serving,
        }
        print(json.dumps(out), flush=True)
    if engine is not None:
        engine.close()
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
