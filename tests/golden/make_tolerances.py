"""Writes tests/golden/nrmse_oracle.json: the oracle's accuracy against an FP64
FFT on the seeded phantom workloads.  These are the stated tolerances of the
radix-2 path (which must reproduce the oracle bit for bit) and the reference
figure for any approximate variant.  Calls only oracle/ and the input
generator.

    python tests/golden/make_tolerances.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_04317_gb300 import phantom  # noqa: E402


def metrics(y, ref):
    err = y.astype(np.complex128) - ref
    nrmse = float(np.linalg.norm(err) / np.linalg.norm(ref))
    rms = float(np.sqrt(np.mean(np.abs(err) ** 2)))
    psnr = float(20 * np.log10(np.abs(ref).max() / rms))
    return {"nrmse": round(nrmse, 6), "psnr_db": round(psnr, 3)}


def run(name, n0, n1, nslices, ncoils, config_id, fmts, ks, sample=None):
    ksp = phantom.mri_batch(n0, n1, nslices, ncoils, config_id=config_id)
    img = phantom.mri_batch(n0, n1, nslices, ncoils, config_id=config_id, domain="image")
    if sample is not None:
        ksp, img = ksp[:sample], img[:sample]
    ref_f = np.fft.fft2(ksp.astype(np.complex128))
    ref_r = img.astype(np.complex128)
    out = []
    for fmt in fmts:
        for k in ks:
            yf, _, _ = oracle.mxfft2d(ksp, fmt, k, op="forward")
            yr, _, _ = oracle.mxfft2d(img, fmt, k, op="roundtrip")
            out.append({"format": fmt, "k": k, "forward": metrics(yf, ref_f),
                        "roundtrip": metrics(yr, ref_r)})
            print(name, fmt, k, out[-1], flush=True)
    return {"n0": n0, "n1": n1, "slices": int(ksp.shape[0]), "config_id": config_id,
            "results": out}


def main():
    res = {
        "note": "oracle NRMSE / PSNR vs numpy FP64 FFT (forward) or the input (round trip); "
                "tau = 1e-3, target 0.5, default tau_min",
        "single_128x128": run("single_128x128", 128, 128, 1, 1, 1, ["e4m3"], [32]),
        "batch64_256x256": run("batch64_256x256", 256, 256, 64, 1, 2, ["e4m3", "e5m2"],
                               [8, 16, 32, 64, 128]),
        "multicoil_512x512_sample4": run("multicoil_512x512", 512, 512, 1, 16, 3, ["e4m3"], [32],
                                         sample=4),
        "large_2048x2048_sample1": run("large_2048x2048", 2048, 2048, 1, 1, 5,
                                       ["e4m3", "e5m2", "e2m3", "e3m2", "e2m1"], [16, 32, 64]),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nrmse_oracle.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
