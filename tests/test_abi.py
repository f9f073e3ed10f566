"""The C ABI library loads, exports every function include/mxfft.h declares and
rejects bad arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2512_04317_gb300 import build, mxfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mxfft.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "mxfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mxfft_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(mxfft.EXPORTS)


def test_plan_argument_validation_without_device(lib):
    h = ctypes.c_void_p()
    bad = [
        (3, 4, 0, 32, 1e-3, 0.5),      # n0 not a power of two
        (1, 4, 0, 32, 1e-3, 0.5),      # n0 < 2
        (4096, 4, 0, 32, 1e-3, 0.5),   # n0 > 2048
        (4, 4, 7, 32, 1e-3, 0.5),      # unknown format
        (4, 4, 0, 3, 1e-3, 0.5),       # k not a power of two
        (4, 4, 0, 256, 1e-3, 0.5),     # k > 128
        (4, 4, 0, 1, 1e-3, 0.5),       # k < 2
        (4, 4, 0, 32, 0.0, 0.5),       # tau not in (0, 1)
        (4, 4, 0, 32, 1.0, 0.5),
        (4, 4, 0, 32, 1e-3, -0.5),     # target <= 0
    ]
    for args in bad:
        assert lib.mxfft_plan(*args, ctypes.byref(h)) == mxfft.MXFFT_ERR_INVALID, args
        assert h.value is None
    assert lib.mxfft_plan(4, 4, 0, 32, 1e-3, 0.3, ctypes.byref(h)) == mxfft.MXFFT_ERR_UNSUPPORTED
    assert lib.mxfft_plan(4, 4, 0, 32, 1e-3, 0.5, None) == mxfft.MXFFT_ERR_INVALID


def test_null_plan_calls_are_rejected(lib):
    assert lib.mxfft_forward(None, None, None, 1, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_inverse(None, None, None, 1, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_roundtrip(None, None, None, 1, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_roundtrip_fused(None, None, None, 1, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_set_option(None, 0, 2.0 ** -10) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_get_status(None, None, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_profile(None, 1) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_profile_read(None, None, None, 2) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_destroy(None) == mxfft.MXFFT_OK


def test_status_strings(lib):
    for code in range(7):
        s = lib.mxfft_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.mxfft_status_string(99).decode() == "unknown status"


def test_library_is_built_for_sm103a():
    flags = " ".join(build.ARCH + build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    for f in ("-fmad=false", "-ftz=false", "-prec-sqrt=true"):
        assert f in flags
    assert "--use_fast_math" not in flags
