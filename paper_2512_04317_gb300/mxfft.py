"""Python binding of libmxfft (include/mxfft.h): argument marshalling only.

Every step of the transform runs in the CUDA library; this module passes
pointers, sizes and the current torch stream through ctypes.  PyTorch is used
for device memory and streams only.  If the library has not been built the
first call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MXFFT_OK = 0
MXFFT_ERR_INVALID = 1
MXFFT_ERR_UNSUPPORTED = 2
MXFFT_ERR_NOMEM = 3
MXFFT_ERR_CUDA = 4
MXFFT_ERR_NONFINITE = 5
MXFFT_ERR_TIMEOUT = 6

FORMATS = {"e4m3": 0, "e5m2": 1, "e2m3": 2, "e3m2": 3, "e2m1": 4, "fp16": 5, "fp32": 6}
OPT_TAU_MIN, OPT_K_MIN, OPT_K_MAX, OPT_GENERIC, OPT_PATH, OPT_TEST_STALL, OPT_FUSED2D, OPT_FOLD_STATS = range(8)

OPS = {"forward": 0, "inverse": 1, "roundtrip": 2, "roundtrip_fused": 3}
ENGINE_GRAPHS, ENGINE_TC16, ENGINE_FUSED2D, ENGINE_NO_RAGGED, ENGINE_FOLD_STATS = 1, 2, 4, 8, 16

# every symbol include/mxfft.h declares
EXPORTS = ("mxfft_plan", "mxfft_set_option", "mxfft_forward", "mxfft_inverse",
           "mxfft_roundtrip", "mxfft_roundtrip_fused", "mxfft_get_status", "mxfft_destroy", "mxfft_profile",
           "mxfft_profile_read", "mxfft_prescale_exponents_noalloc",
           "mxfft_engine_create", "mxfft_engine_run", "mxfft_engine_get_status",
           "mxfft_engine_launches", "mxfft_engine_destroy", "mxfft_tune", "mxfft_tune_save", "mxfft_tune_load",
           "mxfft_tune_clear", "mxfft_server_create", "mxfft_server_submit",
           "mxfft_server_poll", "mxfft_server_wait", "mxfft_server_stats",
           "mxfft_server_destroy", "mxfft_rss", "mxfft_quantize", "mxfft_test_fail_alloc",
           "mxfft_debug_bounds", "mxfft_status_string")


class Item(ctypes.Structure):
    """mxfft_item"""
    _fields_ = [("n0", ctypes.c_int), ("n1", ctypes.c_int), ("format", ctypes.c_int),
                ("k", ctypes.c_int), ("op", ctypes.c_int), ("slices", ctypes.c_int),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("coils", ctypes.c_int), ("reserved", ctypes.c_int), ("rss", ctypes.c_void_p)]


class Request(ctypes.Structure):
    """mxfft_request"""
    _fields_ = [("n0", ctypes.c_int), ("n1", ctypes.c_int), ("format", ctypes.c_int),
                ("k", ctypes.c_int), ("op", ctypes.c_int), ("slices", ctypes.c_int),
                ("host_in", ctypes.c_void_p), ("host_out", ctypes.c_void_p),
                ("tag", ctypes.c_uint64), ("coils", ctypes.c_int), ("reserved", ctypes.c_int),
                ("host_rss", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    """mxfft_completion"""
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("device_flags", ctypes.c_int), ("t_submit_us", ctypes.c_double),
                ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    """mxfft_server_config"""
    _fields_ = [("slots", ctypes.c_int), ("max_batch_slices", ctypes.c_int),
                ("mem_budget", ctypes.c_uint64), ("tau", ctypes.c_float),
                ("target", ctypes.c_float), ("engine_flags", ctypes.c_int),
                ("max_batch_bytes", ctypes.c_uint64)]

_lock = threading.Lock()
_lib = None


# algorithmic bytes per point of one launch of a kernel (profiling kinds of
# mxfft_profile_read): a statistics launch reads the slice once; a row or
# column pass moves half of a transform's 16 B per point
KERNEL_ALG_BYTES_PER_PT = {"stats_kernel": 8, "pass_kernel": 8, "fast_pass_kernel": 8,
                           "tc16_pass_kernel": 8, "tc2d_kernel": 16}


def tc16_supported(n0: int, n1: int, fmt, k: int) -> bool:
    """Whether a plan of this shape, format and k can take the tensor-core
    variant (MXFFT_OPT_PATH = 1)."""
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    sizes = (128, 256, 512, 1024, 2048)
    return n0 in sizes and n1 in sizes and f in (0, 1) and k in (32, 64, 128)


class MxfftError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load libmxfft.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"libmxfft.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, I, F, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
        lib.mxfft_plan.argtypes = [I, I, I, I, F, F, ctypes.POINTER(P)]
        lib.mxfft_set_option.argtypes = [P, I, D]
        for name in ("mxfft_forward", "mxfft_inverse", "mxfft_roundtrip", "mxfft_roundtrip_fused"):
            getattr(lib, name).argtypes = [P, P, P, I, P]
        lib.mxfft_get_status.argtypes = [P, P, P]
        lib.mxfft_destroy.argtypes = [P]
        lib.mxfft_profile.argtypes = [P, I]
        lib.mxfft_profile_read.argtypes = [P, P, P, I]
        lib.mxfft_prescale_exponents_noalloc.argtypes = [P, I, I, I, I, F, F, P, P]
        PP, U64 = ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64
        lib.mxfft_engine_create.argtypes = [F, F, I, PP]
        lib.mxfft_engine_run.argtypes = [P, ctypes.POINTER(Item), I, P]
        lib.mxfft_engine_get_status.argtypes = [P, P, P, I]
        lib.mxfft_engine_launches.argtypes = [P, P]
        lib.mxfft_quantize.argtypes = [P, P, ctypes.c_longlong, I, I, P]
        lib.mxfft_test_fail_alloc.argtypes = [I]
        lib.mxfft_debug_bounds.argtypes = [P, P]
        lib.mxfft_engine_destroy.argtypes = [P]
        lib.mxfft_tune.argtypes = [P, I, P, P]
        lib.mxfft_tune_save.argtypes = [ctypes.c_char_p]
        lib.mxfft_tune_load.argtypes = [ctypes.c_char_p]
        lib.mxfft_tune_clear.argtypes = []
        lib.mxfft_server_create.argtypes = [ctypes.POINTER(ServerConfig), PP]
        lib.mxfft_server_submit.argtypes = [P, ctypes.POINTER(Request)]
        lib.mxfft_server_poll.argtypes = [P, ctypes.POINTER(Completion), I, P]
        lib.mxfft_server_wait.argtypes = [P, D]
        lib.mxfft_server_stats.argtypes = [P, P, P, P]
        lib.mxfft_server_destroy.argtypes = [P]
        lib.mxfft_rss.argtypes = [P, P, I, I, I, I, P]
        lib.mxfft_status_string.argtypes = [I]
        lib.mxfft_status_string.restype = ctypes.c_char_p
        for name in EXPORTS[:-1]:
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load().mxfft_status_string(int(status)).decode()
    except Exception:
        return f"status {status}"


# ---- thin C-ABI wrappers with the header's names -------------------------------

def mxfft_plan(n0: int, n1: int, fmt, k: int, tau: float, target: float) -> int:
    h = ctypes.c_void_p()
    st = load().mxfft_plan(int(n0), int(n1), _fmt(fmt), int(k), float(tau), float(target),
                           ctypes.byref(h))
    if st:
        raise MxfftError(st, "mxfft_plan")
    return h.value


def mxfft_set_option(plan: int, key: int, value: float) -> None:
    st = load().mxfft_set_option(plan, int(key), float(value))
    if st:
        raise MxfftError(st, "mxfft_set_option")


def _call(name, plan, x_ptr, y_ptr, batch, stream_ptr):
    st = getattr(load(), name)(plan, x_ptr, y_ptr, int(batch), stream_ptr)
    if st:
        raise MxfftError(st, name)


def mxfft_forward(plan, in_ptr, out_ptr, batch, stream=None):
    _call("mxfft_forward", plan, in_ptr, out_ptr, batch, stream)


def mxfft_inverse(plan, in_ptr, out_ptr, batch, stream=None):
    _call("mxfft_inverse", plan, in_ptr, out_ptr, batch, stream)


def mxfft_roundtrip(plan, in_ptr, out_ptr, batch, stream=None):
    _call("mxfft_roundtrip", plan, in_ptr, out_ptr, batch, stream)


def mxfft_roundtrip_fused(plan, in_ptr, out_ptr, batch, stream=None):
    _call("mxfft_roundtrip_fused", plan, in_ptr, out_ptr, batch, stream)


def mxfft_get_status(plan, k_count: int = 0):
    """Returns (status, device_flags, k list of length k_count)."""
    flags = ctypes.c_int(0)
    karr = (ctypes.c_int32 * max(k_count, 1))()
    st = load().mxfft_get_status(plan, ctypes.byref(flags), karr if k_count else None)
    return st, flags.value, list(karr)[:k_count]


def mxfft_destroy(plan) -> None:
    if plan:
        load().mxfft_destroy(plan)


def mxfft_profile(plan, enable: bool) -> None:
    st = load().mxfft_profile(plan, int(bool(enable)))
    if st:
        raise MxfftError(st, "mxfft_profile")


PROFILE_KINDS = ("stats_kernel", "pass_kernel", "fast_pass_kernel", "tc16_pass_kernel",
                 "tc2d_kernel")


def mxfft_profile_read(plan):
    """{kernel name: (total_ms, launches)} recorded since the last read."""
    n = len(PROFILE_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    st = load().mxfft_profile_read(plan, ms, cnt, n)
    if st:
        raise MxfftError(st, "mxfft_profile_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_KINDS)}


NOALLOC_MAX_SLICES = 1024


def mxfft_prescale_exponents_noalloc(in_ptr, batch, n0, n1, fmt, tau, target, k_out_ptr,
                                     stream=None) -> int:
    """Alg. 1 exponents of `batch` slices without any device allocation
    (for callers that cannot allocate at call time); returns the status."""
    return load().mxfft_prescale_exponents_noalloc(in_ptr, int(batch), int(n0), int(n1),
                                                   _fmt(fmt), float(tau), float(target),
                                                   k_out_ptr, stream)


def _fmt(fmt) -> int:
    return FORMATS[fmt] if isinstance(fmt, str) else int(fmt)


def _op(op) -> int:
    return OPS[op] if isinstance(op, str) else int(op)


def _check(st, what):
    if st:
        raise MxfftError(st, what)


# ---- ragged batch executor ------------------------------------------------------

def mxfft_engine_create(tau: float = 1e-3, target: float = 0.5, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().mxfft_engine_create(float(tau), float(target), int(flags), ctypes.byref(h)),
           "mxfft_engine_create")
    return h.value


def mxfft_engine_run(engine, items, stream=None) -> None:
    arr = (Item * max(len(items), 1))(*items)
    _check(load().mxfft_engine_run(engine, arr, len(items), stream), "mxfft_engine_run")


def mxfft_engine_get_status(engine, k_count: int = 0):
    """(device_flags, k list of length k_count) of the engine's last run."""
    flags = ctypes.c_int(0)
    karr = (ctypes.c_int32 * max(k_count, 1))()
    _check(load().mxfft_engine_get_status(engine, ctypes.byref(flags), karr if k_count else None,
                                          int(k_count)), "mxfft_engine_get_status")
    return flags.value, list(karr)[:k_count]


def mxfft_engine_launches(engine) -> int:
    """Kernels the engine's last run enqueued (a graph replay: its kernels)."""
    n = ctypes.c_int(0)
    _check(load().mxfft_engine_launches(engine, ctypes.byref(n)), "mxfft_engine_launches")
    return n.value


def mxfft_engine_destroy(engine) -> None:
    if engine:
        load().mxfft_engine_destroy(engine)


def mxfft_debug_bounds():
    """(enabled, violations since the last call) of the bounds-check build."""
    en, v = ctypes.c_int(0), ctypes.c_ulonglong(0)
    _check(load().mxfft_debug_bounds(ctypes.byref(en), ctypes.byref(v)), "mxfft_debug_bounds")
    return bool(en.value), int(v.value)


def mxfft_test_fail_alloc(after: int) -> None:
    """Test hook: the plan allocation after `after` more successful ones fails
    (MXFFT_ERR_NOMEM); -1 disarms it."""
    _check(load().mxfft_test_fail_alloc(int(after)), "mxfft_test_fail_alloc")


# ---- element quantiser (Alg. 2's rounding Q) --------------------------------------------

def mxfft_quantize(in_ptr, out_ptr, n, fmt, path, stream=None) -> None:
    _check(load().mxfft_quantize(in_ptr, out_ptr, int(n), _fmt(fmt), int(path), stream),
           "mxfft_quantize")


# ---- root-sum-of-squares coil combine (Eq. (1)) -------------------------------------

def mxfft_rss(z_ptr, out_ptr, images, coils, n0, n1, stream=None) -> None:
    _check(load().mxfft_rss(z_ptr, out_ptr, int(images), int(coils), int(n0), int(n1), stream),
           "mxfft_rss")


def rss(z, coils: int, out=None):
    """RSS images float32 [images, n0, n1] of z complex64 CUDA [images * coils, n0, n1]."""
    import torch
    _check_tensor(z, "z")
    if not z.is_cuda or z.shape[0] % coils:
        raise ValueError("z must be a CUDA tensor [images * coils, n0, n1]")
    images = z.shape[0] // coils
    n0, n1 = z.shape[-2], z.shape[-1]
    if out is None:
        out = torch.empty((images, n0, n1), dtype=torch.float32, device=z.device)
    mxfft_rss(z.data_ptr(), out.data_ptr(), images, coils, n0, n1,
              torch.cuda.current_stream(z.device).cuda_stream)
    return out


# ---- autotuner -------------------------------------------------------------------

def mxfft_tune(plan, batch: int, stream=None) -> int:
    """Measure the launch geometries of `plan`'s passes at `batch` (radix-2:
    groups per CTA; tensor-core path: resident CTAs per SM); returns the
    number of candidates timed."""
    n = ctypes.c_int(0)
    _check(load().mxfft_tune(plan, int(batch), stream, ctypes.byref(n)), "mxfft_tune")
    return n.value


def mxfft_tune_save(path: str) -> None:
    _check(load().mxfft_tune_save(os.fsencode(path)), "mxfft_tune_save")


def mxfft_tune_load(path: str) -> None:
    _check(load().mxfft_tune_load(os.fsencode(path)), "mxfft_tune_load")


def mxfft_tune_clear() -> None:
    _check(load().mxfft_tune_clear(), "mxfft_tune_clear")


# ---- request server --------------------------------------------------------------

def mxfft_server_create(slots=4, max_batch_slices=256, mem_budget=0, tau=1e-3, target=0.5,
                        engine_flags=0, max_batch_bytes=0) -> int:
    cfg = ServerConfig(int(slots), int(max_batch_slices), int(mem_budget), float(tau),
                       float(target), int(engine_flags), int(max_batch_bytes))
    h = ctypes.c_void_p()
    _check(load().mxfft_server_create(ctypes.byref(cfg), ctypes.byref(h)), "mxfft_server_create")
    return h.value


def mxfft_server_submit(server, req: Request) -> None:
    _check(load().mxfft_server_submit(server, ctypes.byref(req)), "mxfft_server_submit")


def mxfft_server_poll(server, max_n: int = 256):
    arr = (Completion * max(max_n, 1))()
    n = ctypes.c_int(0)
    _check(load().mxfft_server_poll(server, arr, int(max_n), ctypes.byref(n)), "mxfft_server_poll")
    return [arr[i] for i in range(n.value)]


def mxfft_server_wait(server, timeout_s: float) -> int:
    return load().mxfft_server_wait(server, float(timeout_s))


def mxfft_server_stats(server):
    """(batches, peak device bytes of admitted requests, budget)."""
    b, pk, bud = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(load().mxfft_server_stats(server, ctypes.byref(b), ctypes.byref(pk), ctypes.byref(bud)),
           "mxfft_server_stats")
    return b.value, pk.value, bud.value


def mxfft_server_destroy(server) -> None:
    if server:
        load().mxfft_server_destroy(server)


# ---- torch convenience ---------------------------------------------------------

class Plan:
    """A plan for n0 x n1 complex64 slices; transforms torch CUDA tensors of
    shape [..., n0, n1] (contiguous complex64) on the current torch stream."""

    def __init__(self, n0: int, n1: int, fmt="e4m3", k: int = 32, tau: float = 1e-3,
                 target: float = 0.5, tau_min: float | None = None,
                 kmin: int | None = None, kmax: int | None = None, generic: bool = False,
                 path: str = "radix2", fused2d: bool = False, fold_stats: bool = False):
        self.n0, self.n1, self.fmt, self.k = int(n0), int(n1), fmt, int(k)
        self.handle = mxfft_plan(n0, n1, fmt, k, tau, target)
        self._last = (0, 0)   # (batch, op)
        if tau_min is not None:
            mxfft_set_option(self.handle, OPT_TAU_MIN, tau_min)
        if kmin is not None:
            mxfft_set_option(self.handle, OPT_K_MIN, kmin)
        if kmax is not None:
            mxfft_set_option(self.handle, OPT_K_MAX, kmax)
        if generic:
            mxfft_set_option(self.handle, OPT_GENERIC, 1)
        if path not in ("radix2", "tc16"):
            raise ValueError(path)
        if path == "tc16":
            mxfft_set_option(self.handle, OPT_PATH, 1)
            if fused2d:
                mxfft_set_option(self.handle, OPT_FUSED2D, 1)
            if fold_stats:
                mxfft_set_option(self.handle, OPT_FOLD_STATS, 1)
        self.path = path

    def _run(self, name, x, out):
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous complex64 CUDA tensor")
        if tuple(x.shape[-2:]) != (self.n0, self.n1):
            raise ValueError(f"expected [..., {self.n0}, {self.n1}], got {tuple(x.shape)}")
        if out is None:
            out = torch.empty_like(x)
        elif out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError("out must match x")
        batch = x.numel() // (self.n0 * self.n1)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        _call(name, self.handle, x.data_ptr(), out.data_ptr(), batch, stream)
        self._last = (batch, 2 if name == "mxfft_roundtrip" else 1)
        return out

    def forward(self, x, out=None):
        return self._run("mxfft_forward", x, out)

    def inverse(self, x, out=None):
        return self._run("mxfft_inverse", x, out)

    def roundtrip(self, x, out=None):
        return self._run("mxfft_roundtrip", x, out)

    def roundtrip_fused(self, x, out=None):
        """The fused encode -> F -> F^-1 -> decode round trip (one prescale)."""
        return self._run("mxfft_roundtrip_fused", x, out)

    def status(self):
        """(status, device_flags, k) of the last call; k is [batch] or [batch][2]."""
        batch, per = self._last
        st, flags, k = mxfft_get_status(self.handle, batch * per)
        if per == 2:
            k = [k[2 * i:2 * i + 2] for i in range(batch)]
        return st, flags, k

    def close(self):
        if getattr(self, "handle", None):
            mxfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_tensor(x, name):
    import torch
    if x.dtype != torch.complex64 or not x.is_contiguous() or x.dim() < 2:
        raise ValueError(f"{name}: expected a contiguous complex64 tensor [..., n0, n1]")


class Engine:
    """Ragged batch executor: run([(op, x, out, fmt, k), ...]) transforms each
    CUDA tensor x [..., n0, n1] into out (may be x) in one set of launches on the
    current torch stream, with the same bits as the per-plan calls."""

    def __init__(self, tau: float = 1e-3, target: float = 0.5, graphs: bool = False,
                 tc16: bool = False, fused2d: bool = False, ragged: bool = True,
                 fold_stats: bool = False):
        flags = ((ENGINE_GRAPHS if graphs else 0) | (ENGINE_TC16 if tc16 else 0) |
                 (ENGINE_FUSED2D if fused2d else 0) | (0 if ragged else ENGINE_NO_RAGGED) |
                 (ENGINE_FOLD_STATS if fold_stats else 0))
        self.handle = mxfft_engine_create(tau, target, flags)
        self._slices = 0

    def run(self, work, stream=None):
        """work: (op, x, out, fmt, k) or (op, x, out, fmt, k, rss, coils) tuples; rss is a
        float32 CUDA tensor [slices / coils, n0, n1] receiving the RSS images of out."""
        import torch
        items = []
        dev = None
        for w in work:
            op, x, out, fmt, k = w[:5]
            rss_t, coils = (w[5], int(w[6])) if len(w) > 5 else (None, 0)
            _check_tensor(x, "x")
            _check_tensor(out, "out")
            if not x.is_cuda or out.shape != x.shape:
                raise ValueError("x must be a CUDA tensor and out must match it")
            dev = x.device
            n0, n1 = x.shape[-2], x.shape[-1]
            items.append(Item(n0, n1, _fmt(fmt), int(k), _op(op), x.numel() // (n0 * n1),
                              x.data_ptr(), out.data_ptr(), coils, 0,
                              rss_t.data_ptr() if rss_t is not None else None))
        if stream is None and dev is not None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        mxfft_engine_run(self.handle, items, stream)
        self._slices = sum(it.slices for it in items)

    def launches_per_run(self) -> int:
        """Kernels the last run enqueued."""
        return mxfft_engine_launches(self.handle)

    def status(self):
        """(device_flags, [[k, k_inverse] per slice]) of the last run."""
        flags, k = mxfft_engine_get_status(self.handle, 2 * self._slices)
        return flags, [k[2 * i:2 * i + 2] for i in range(self._slices)]

    def close(self):
        if getattr(self, "handle", None):
            mxfft_engine_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Request server with continuous batching.  submit() takes host tensors
    (pinned CPU complex64 [slices, n0, n1] for overlapped copies) that must
    stay alive until their completion is returned by poll()."""

    def __init__(self, slots=4, max_batch_slices=256, mem_budget=0, tau=1e-3, target=0.5,
                 graphs=False, tc16=False, max_batch_bytes=0, ragged=True):
        flags = ((ENGINE_GRAPHS if graphs else 0) | (ENGINE_TC16 if tc16 else 0) |
                 (0 if ragged else ENGINE_NO_RAGGED))
        self.handle = mxfft_server_create(slots, max_batch_slices, mem_budget, tau, target, flags,
                                          max_batch_bytes)
        self._keep = {}

    def submit(self, tag: int, x, out, fmt="e4m3", k: int = 32, op="forward", rss=None,
               coils: int = 1) -> None:
        """out: host tensor like x, or None when rss (float32 host [slices / coils, n0, n1])
        receives the RSS images of the result."""
        _check_tensor(x, "x")
        if out is not None:
            _check_tensor(out, "out")
            if out.is_cuda or out.shape != x.shape:
                raise ValueError("out: a host tensor like x")
        if x.is_cuda or (out is None and rss is None):
            raise ValueError("host tensors expected, and out or rss")
        n0, n1 = x.shape[-2], x.shape[-1]
        req = Request(n0, n1, _fmt(fmt), int(k), _op(op), x.numel() // (n0 * n1), x.data_ptr(),
                      out.data_ptr() if out is not None else None, int(tag),
                      int(coils) if rss is not None else 0, 0,
                      rss.data_ptr() if rss is not None else None)
        self._keep[int(tag)] = (x, out, rss)
        mxfft_server_submit(self.handle, req)

    def poll(self, max_n: int = 1024):
        done = mxfft_server_poll(self.handle, max_n)
        for c in done:
            self._keep.pop(int(c.tag), None)
        return done

    def wait(self, timeout_s: float = 60.0) -> bool:
        return mxfft_server_wait(self.handle, timeout_s) == MXFFT_OK

    def stats(self):
        return mxfft_server_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mxfft_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
