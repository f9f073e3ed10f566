"""Small transforms that reach every kernel family the bounds-check build
instruments (register-resident passes with k = 32 / 64 / 128 and n up to
2048, the generic pass and the FP16 control, the fused round trip, the
tensor-core passes and the fused 2D tensor-core kernel).  Run as a script with
a library path, it writes every result and the violation count to an .npz
file; imported, it offers the same cases to the test."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (n0, n1, batch, format, k, op, plan options)
CASES = [
    (64, 256, 2, "e4m3", 32, "forward", {}),
    (256, 128, 2, "e5m2", 64, "roundtrip", {}),
    (128, 256, 1, "e4m3", 128, "inverse", {}),
    (2048, 64, 1, "e4m3", 32, "forward", {}),
    (8, 16, 3, "e2m3", 4, "roundtrip", {}),
    (32, 32, 2, "fp16", 32, "forward", {}),
    (128, 128, 2, "e4m3", 32, "roundtrip_fused", {}),
    (16, 64, 2, "e2m1", 8, "forward", {"generic": True}),
    (256, 512, 2, "e4m3", 32, "roundtrip", {"path": "tc16"}),
    (1024, 256, 1, "e5m2", 64, "forward", {"path": "tc16"}),
    (2048, 256, 1, "e4m3", 32, "roundtrip", {"path": "tc16"}),
    (128, 128, 9, "e4m3", 32, "roundtrip", {"path": "tc16"}),
    (128, 512, 2, "e5m2", 64, "forward", {"path": "tc16", "fold_stats": True}),
    (512, 128, 2, "e4m3", 32, "roundtrip", {"path": "tc16", "fold_stats": True}),
    (256, 256, 5, "e4m3", 32, "forward", {"path": "tc16", "fused2d": True}),
    (512, 512, 2, "e5m2", 32, "roundtrip", {"path": "tc16", "fused2d": True}),
]


def run_all(lib_path=None):
    import torch

    from paper_2512_04317_gb300 import mxfft, phantom
    mxfft.load(lib_path)
    mxfft.mxfft_debug_bounds()                    # clears the counters
    outs = {}
    for i, (n0, n1, b, fmt, k, op, opts) in enumerate(CASES):
        dom = "image" if op.startswith("roundtrip") else "kspace"
        x = torch.from_numpy(phantom.mri_batch(n0, n1, b, 1, config_id=60 + i, domain=dom)).cuda()
        with mxfft.Plan(n0, n1, fmt, k, **opts) as p:
            outs[f"case{i}"] = getattr(p, op)(x).cpu().numpy()
    torch.cuda.synchronize()
    enabled, bad = mxfft.mxfft_debug_bounds()
    return outs, enabled, bad


if __name__ == "__main__":
    outs, enabled, bad = run_all(sys.argv[1])
    np.savez(sys.argv[2], enabled=enabled, violations=bad, **outs)
