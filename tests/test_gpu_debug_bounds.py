"""The bounds-check build (MXFFT_DEBUG_BOUNDS; a memory checker is not
available on this pool): the library compiled with the checks runs small
transforms that reach every instrumented kernel family (debug_bounds_cases),
in a separate process; no index may leave its buffer and every result must
equal the normal build's bit for bit (the checks only observe)."""
import os
import subprocess
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import debug_bounds_cases  # noqa: E402

pytestmark = pytest.mark.gpu


def test_debug_bounds_build_reports_no_violation(cuda_device, tmp_path):
    from paper_2512_04317_gb300 import build
    lib = build.build(debug_bounds=True)
    out = tmp_path / "debug.npz"
    script = os.path.join(os.path.dirname(os.path.abspath(__file__)), "debug_bounds_cases.py")
    subprocess.run([sys.executable, script, lib, str(out)], check=True, timeout=600)
    dbg = np.load(out)
    assert int(dbg["enabled"]) == 1
    assert int(dbg["violations"]) == 0
    ref, enabled, bad = debug_bounds_cases.run_all()       # the normal build, this process
    assert not enabled and bad == 0
    for name, want in ref.items():
        np.testing.assert_array_equal(dbg[name].view(np.uint32), want.view(np.uint32), name)
