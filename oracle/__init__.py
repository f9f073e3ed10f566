"""CPU oracle for the MX-scaled low-precision 2D FFT (arXiv 2512.04317).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``mxfft_oracle.c`` (plain C, FP32 with a fixed
operation order, ``-ffp-contract=off``); this module compiles it with gcc and
wraps it with ctypes over numpy arrays.

Functions and the passages they follow:
  * ``mxfft2d``         Alg. 1 + Alg. 2 inside a radix-2 DIT 2D FFT; Eq. (1);
                        op "roundtrip_fused": the fused encode -> F -> F^-1 ->
                        decode round trip of Sec. 4.3 (reading C17)
  * ``prescale_k``      Alg. 1 (Sec. 2.1)
  * ``magnitude``       |x| as used by Alg. 1 (reading C3)
  * ``quantize``        the OCP element rounding used by EncodeBlockMX (Sec. 2.2)
  * ``butterfly_block`` Alg. 2 on one block
  * ``fft2d_exact``     FP64 dataflow without quantisation (structural pin only)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mxfft_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_mxfft.so")

FORMATS = {"e4m3": 0, "e5m2": 1, "e2m3": 2, "e3m2": 3, "e2m1": 4, "fp16": 5, "fp32": 6}
# tau_min defaults: 2^-10 for e4m3 and 2^-12 for e5m2 (Alg. 1 notes); 2^-10 for
# the FP6/FP4 formats, where the paper gives none; the smallest binary16
# magnitude for the FP16 control and binary32's smallest normal for the FP32
# reference ablation.
TAU_MIN_DEFAULT = {"e4m3": 2.0**-10, "e5m2": 2.0**-12, "e2m3": 2.0**-10,
                   "e3m2": 2.0**-10, "e2m1": 2.0**-10, "fp16": 2.0**-24, "fp32": 2.0**-126}
OP = {"forward": 0, "inverse": 1, "roundtrip": 2, "roundtrip_fused": 3}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc; returns its path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, f32, f64, i64 = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_long
        lib.oracle_mxfft2d.argtypes = [P, P, i32, i32, i32, i32, i32, f32, f64, f64,
                                       i32, i32, i32, i32, i32, P, P]
        lib.oracle_mxfft2d.restype = i32
        lib.oracle_prescale_k.argtypes = [P, i64, f32, f64, f64, i32, i32, P]
        lib.oracle_prescale_k.restype = i32
        lib.oracle_magnitude.argtypes = [P, P, i64]
        lib.oracle_magnitude.restype = None
        lib.oracle_quantize.argtypes = [P, P, i64, i32]
        lib.oracle_quantize.restype = i32
        lib.oracle_quantize_f64.argtypes = [P, P, i64, i32]
        lib.oracle_quantize_f64.restype = i32
        lib.oracle_butterfly_block.argtypes = [i32, P, P, P, P, P, P, i32, i32, i32]
        lib.oracle_butterfly_block.restype = i32
        lib.oracle_format_info.argtypes = [i32, P, P, P, P]
        lib.oracle_format_info.restype = i32
        lib.oracle_fft2d_exact.argtypes = [P, P, i32, i32, i32, i32]
        lib.oracle_fft2d_exact.restype = i32
        lib.oracle_rss.argtypes = [P, P, i64, i32, i64]
        lib.oracle_rss.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fmt(fmt) -> int:
    return FORMATS[fmt] if isinstance(fmt, str) else int(fmt)


def _fmt_name(fmt) -> str:
    if isinstance(fmt, str):
        return fmt
    return {v: k for k, v in FORMATS.items()}[int(fmt)]


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def format_info(fmt):
    """(emax, emin, mbits, maxnorm) of an element format."""
    lib = _load()
    a, b, c = (np.zeros(1, np.int32) for _ in range(3))
    d = np.zeros(1, np.float64)
    if lib.oracle_format_info(_fmt(fmt), _ptr(a), _ptr(b), _ptr(c), _ptr(d)):
        raise ValueError(f"unknown format {fmt!r}")
    return int(a[0]), int(b[0]), int(c[0]), float(d[0])


def mxfft2d(x: np.ndarray, fmt="e4m3", k: int = 32, tau: float = 1e-3,
            target: float = 0.5, tau_min: float | None = None,
            kmin: int = -126, kmax: int = 126, op: str = "forward",
            renorm: bool = True, direct_enc: bool = False):
    """MX-FFT of a batch of complex64 slices ``x[..., n0, n1]``.

    Returns ``(out, kexp, flags)``: ``out`` complex64 with the shape of ``x``;
    ``kexp`` the prescale exponents, shape ``[batch]`` (``[batch, 2]`` for the
    round trip: forward k, inverse k; the fused round trip has one k per
    slice); ``flags`` nonzero where a prescale saw a non-finite magnitude.
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex64)
    if x.ndim < 2:
        raise ValueError("need at least 2 dims")
    n0, n1 = x.shape[-2:]
    batch = int(np.prod(x.shape[:-2], dtype=np.int64)) if x.ndim > 2 else 1
    out = np.empty_like(x)
    nk = 2 * batch if op == "roundtrip" else batch
    kexp = np.zeros(max(nk, 1), np.int32)
    flags = np.zeros(max(batch, 1), np.int32)
    if tau_min is None:
        tau_min = TAU_MIN_DEFAULT[_fmt_name(fmt)]
    rc = lib.oracle_mxfft2d(_ptr(x), _ptr(out), batch, n0, n1, _fmt(fmt), int(k),
                            float(tau), float(target), float(tau_min), int(kmin),
                            int(kmax), OP[op], int(renorm), int(direct_enc),
                            _ptr(kexp), _ptr(flags))
    if rc:
        raise ValueError("oracle_mxfft2d rejected its arguments")
    kexp = kexp[:nk]
    if op == "roundtrip":
        kexp = kexp.reshape(batch, 2)
    return out, kexp, flags[:batch]


def prescale_k(x: np.ndarray, fmt="e4m3", tau: float = 1e-3, target: float = 0.5,
               tau_min: float | None = None, kmin: int = -126, kmax: int = 126):
    """Alg. 1 on one slice: returns (k, nonfinite)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex64).ravel()
    nf = np.zeros(1, np.int32)
    if tau_min is None:
        tau_min = TAU_MIN_DEFAULT[_fmt_name(fmt)]
    k = lib.oracle_prescale_k(_ptr(x), x.size, float(tau), float(target),
                              float(tau_min), int(kmin), int(kmax), _ptr(nf))
    return int(k), bool(nf[0])


def magnitude(x: np.ndarray) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex64)
    m = np.empty(x.shape, np.float32)
    lib.oracle_magnitude(_ptr(x), _ptr(m), x.size)
    return m


def quantize(x: np.ndarray, fmt) -> np.ndarray:
    """Element rounding (no block scale) of FP32 or FP64 values."""
    lib = _load()
    if np.asarray(x).dtype == np.float64:
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(x)
        lib.oracle_quantize_f64(_ptr(x), _ptr(out), x.size, _fmt(fmt))
        return out
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib.oracle_quantize(_ptr(x), _ptr(out), x.size, _fmt(fmt))
    return out


def butterfly_block(u, v, w, fmt="e4m3", renorm=True, direct_enc=False):
    """Alg. 2 on one block: u, v complex64 [nb], w complex128 [nb]."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.complex64)
    v = np.ascontiguousarray(v, dtype=np.complex64)
    w = np.asarray(w, dtype=np.complex128)
    wr = np.ascontiguousarray(w.real)
    wi = np.ascontiguousarray(w.imag)
    y0 = np.empty_like(u)
    y1 = np.empty_like(u)
    rc = lib.oracle_butterfly_block(u.size, _ptr(u), _ptr(v), _ptr(wr), _ptr(wi),
                                    _ptr(y0), _ptr(y1), _fmt(fmt), int(renorm),
                                    int(direct_enc))
    if rc:
        raise ValueError("bad butterfly arguments")
    return y0, y1


def rss(z: np.ndarray, coils: int) -> np.ndarray:
    """Eq. (1) coil combine: z complex64 [images * coils, n0, n1] (coil fastest)
    -> float32 [images, n0, n1]."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.complex64)
    if z.ndim < 2 or coils < 1 or z.shape[0] % coils:
        raise ValueError("z must be [images * coils, n0, n1]")
    images = z.shape[0] // coils
    npts = int(np.prod(z.shape[1:]))
    out = np.empty((images,) + z.shape[1:], np.float32)
    lib.oracle_rss(_ptr(z), _ptr(out), images, int(coils), npts)
    return out


def fft2d_exact(x: np.ndarray, op: str = "forward") -> np.ndarray:
    """FP64 same-dataflow FFT of complex128 slices ``x[..., n0, n1]``."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex128)
    n0, n1 = x.shape[-2:]
    batch = int(np.prod(x.shape[:-2], dtype=np.int64)) if x.ndim > 2 else 1
    out = np.empty_like(x)
    if lib.oracle_fft2d_exact(_ptr(x), _ptr(out), batch, n0, n1, OP[op]):
        raise ValueError("bad arguments")
    return out
