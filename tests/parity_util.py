"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs and compare bit for bit."""
import numpy as np

import oracle


def run_gpu(x: np.ndarray, fmt="e4m3", k=32, op="forward", tau=1e-3, target=0.5,
            tau_min=None, kmin=None, kmax=None, inplace=False, generic=False):
    import torch

    from paper_2512_04317_gb300 import mxfft
    n0, n1 = x.shape[-2:]
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).to(dev)
    with mxfft.Plan(n0, n1, fmt, k, tau, target, tau_min=tau_min, kmin=kmin, kmax=kmax,
                    generic=generic) as p:
        out = xt if inplace else None
        y = getattr(p, op)(xt, out=out)
        torch.cuda.synchronize()
        st, flags, kk = p.status()
    return y.cpu().numpy(), np.array(kk), flags, st


def run_oracle(x, fmt="e4m3", k=32, op="forward", tau=1e-3, target=0.5, tau_min=None,
               kmin=None, kmax=None):
    kw = {}
    if tau_min is not None:
        kw["tau_min"] = tau_min
    if kmin is not None:
        kw["kmin"] = kmin
    if kmax is not None:
        kw["kmax"] = kmax
    return oracle.mxfft2d(x, fmt, k, tau=tau, target=target, op=op, **kw)


def assert_bitwise(got: np.ndarray, want: np.ndarray, what=""):
    """Bit-for-bit equality, except that a NaN matches any NaN (payloads and
    the sign of a NaN are not specified by IEEE arithmetic)."""
    g = np.ascontiguousarray(got).view(np.uint32).copy()
    w = np.ascontiguousarray(want).view(np.uint32).copy()
    gn = np.isnan(np.ascontiguousarray(got).view(np.float32))
    wn = np.isnan(np.ascontiguousarray(want).view(np.float32))
    g[gn] = 0x7fc00000
    w[wn] = 0x7fc00000
    if not np.array_equal(g, w):
        bad = np.argwhere(g.reshape(got.shape + (2,)) != w.reshape(want.shape + (2,)))
        first = tuple(bad[0][:-1])
        raise AssertionError(
            f"{what}: {len(bad)} of {g.size} words differ; first at {first}: "
            f"got {got[first]!r} want {want[first]!r}")


def check(x, fmt="e4m3", k=32, op="forward", **kw):
    """Bitwise output parity and exact prescale exponents."""
    inplace = kw.pop("inplace", False)
    generic = kw.pop("generic", False)
    got, kg, flags, st = run_gpu(x, fmt, k, op, inplace=inplace, generic=generic, **kw)
    want, kw_, wflags = run_oracle(x, fmt, k, op, **kw)
    assert st == (5 if wflags.any() else 0), (st, wflags)
    assert bool(flags) == bool(wflags.any())
    ok = ~wflags.astype(bool)
    shape = x.shape
    got = got.reshape((-1,) + shape[-2:])
    want = want.reshape((-1,) + shape[-2:])
    assert_bitwise(got[ok], want[ok], f"{fmt} k={k} {op} {shape}")
    assert np.array_equal(np.asarray(kg).reshape(np.asarray(kw_).shape), kw_), (kg, kw_)
    return got, want


def assert_close_to_emulation(got, want, what=""):
    """Element-wise comparison of the tensor-core variant with its emulation.
    The hardware accumulates the 32 exact products of a DFT row in FP32 and
    the emulation in FP64, so a rare element can differ by one FP32 rounding,
    which may move a later 8-bit rounding by one grid step of its block.  Such
    a flip in the columns pass changes the outputs of that one column
    transform (a flip in the rows pass: of one row, before the columns pass
    spreads it thinly); it never changes many lines of both orientations.
    Each element's error is measured against the peak of its row and,
    separately, of its column: (1) none exceeds 10 % of its line's peak, (2)
    the elements off by more than 1e-5 of a peak lie in at most max(2, 1 %)
    of the rows or in at most that many columns.  An index error (a swapped
    operand, a wrong twiddle or slot) gives errors of order one across many
    rows and columns and fails both."""
    g = np.asarray(got).astype(np.complex128)
    w = np.asarray(want).astype(np.complex128)
    assert np.isfinite(g).all(), what
    g = g.reshape((-1,) + g.shape[-2:])
    w = w.reshape(g.shape)
    err = np.abs(g - w)
    off = np.zeros(g.shape, bool)
    for axis in (-1, -2):
        peak = np.abs(w).max(axis=axis, keepdims=True)
        rel = err / np.maximum(peak, 1e-300)
        assert rel.max() < 0.1, (what, axis, rel.max())
        off |= rel > 1e-5
    rows = int(off.any(axis=-1).sum())      # (slice, row) lines holding an off element
    cols = int(off.any(axis=-2).sum())
    limit = max(2, (g.shape[0] * min(g.shape[-2], g.shape[-1])) // 100)
    assert min(rows, cols) <= limit, (what, "rows", rows, "cols", cols, "limit", limit)
