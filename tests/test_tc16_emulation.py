"""CPU checks of the tensor-core variant's emulation (tests/tc16_ref.py) and of
the n = 128 geometry of its kernel (mx_tc16.cu).

(1) The emulation is pinned to the exact DFT: its NRMSE against numpy's FFT
    is of the order of the element format's rounding (8-bit elements), while
    an index error (a wrong twiddle, a transposed round, a swapped pair)
    gives errors of order one.
(2) The matrix of the n = 128 second round holds two 8-point DFTs on its
    diagonal and nothing else, with one row scale 2^-emax per row, as the
    kernel assumes.
(3) The n = 128 index maps of the kernel, re-derived here: every shared-
    memory access stays inside the tile buffer, round A writes and the
    8-point round reads cover every element of a tile once, and each warp
    access takes the minimum number of shared-memory wavefronts (no bank
    conflicts)."""
import os
import sys

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import tc16_ref  # noqa: E402

BOUND = {"e4m3": 0.08, "e5m2": 0.16}


@pytest.mark.parametrize("n", [128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
@pytest.mark.parametrize("sgn", [-1, 1])
def test_emulation_close_to_exact_dft(n, fmt, sgn):
    x = phantom.random_complex((4, n), seed=n + (sgn > 0))
    y = tc16_ref.fft1d(x, fmt, sgn).astype(np.complex128)
    xd = x.astype(np.complex128)
    ref = np.fft.fft(xd, axis=-1) if sgn < 0 else np.fft.ifft(xd, axis=-1) * n
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < BOUND[fmt], (n, fmt, sgn, err)
    # a planted index error in the input order is far outside that bound
    bad = np.linalg.norm(y - np.roll(ref, 1, axis=-1)) / np.linalg.norm(ref)
    assert bad > 0.5


@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
def test_eight_point_pair_matrix(fmt):
    Fq, sF = tc16_ref.dft8pair_matrix(-1, fmt)
    emax = tc16_ref.EMAX[fmt]
    assert np.all(sF == -emax)
    assert np.all(Fq[:16, 16:] == 0) and np.all(Fq[16:, :16] == 0)
    np.testing.assert_array_equal(Fq[:16, :16], Fq[16:, 16:])
    # the exact entries (0, +-1) stay exact; k2 = 0 sums its inputs
    F = Fq * 2.0 ** sF[:, None]
    assert np.all(F[0, 0:16:2] == 1) and np.all(F[0, 1:16:2] == 0)
    # within one element grid step of the exact 8-point DFT
    W = np.exp(-2j * np.pi * np.outer(np.arange(8), np.arange(8)) / 8)
    R = np.zeros((16, 16))
    R[0::2, 0::2], R[0::2, 1::2] = W.real, -W.imag
    R[1::2, 0::2], R[1::2, 1::2] = W.imag, W.real
    step = 2.0 ** -(3 if fmt == "e4m3" else 2)
    assert np.abs(F[:16, :16] - R).max() <= step / 2 + 1e-12


# ---- n = 128 geometry of the kernel (both CTA shapes) ----------------------
N, M = 128, 8
TS, PADR, LGP = N + 2 * (N >> 4) + 8, 2, 4        # rows: pads after every 16 elements


def geo(nt):
    T = 16 * nt // N
    return dict(NT=nt, T=T, LGT=T.bit_length() - 1, BUF=max(T * TS, N * T))


def slot_row(g, t, e):
    return t * TS + e + PADR * (e >> LGP)


def slot_col(g, t, e):
    return e * g["T"] + t


def wavefronts(byte_addrs, width):
    """Shared-memory wavefronts of one warp access: the largest number of
    distinct 4-byte words any of the 32 banks holds."""
    words = set()
    for a in byte_addrs:
        for w in range(width // 4):
            words.add(a // 4 + w)
    per_bank = {}
    for w in words:
        per_bank.setdefault(w % 32, set()).add(w)
    return max(len(v) for v in per_bank.values())


def check_access(g, addrs_per_lane, width):
    """addrs_per_lane: slot index (8-byte units) per thread for one access."""
    for w0 in range(0, g["NT"], 32):
        lanes = [addrs_per_lane[w0 + i] * 8 for i in range(32)]
        assert all(0 <= a and a + width <= g["BUF"] * 8 for a in lanes)
        assert all(a % width == 0 for a in lanes), "aligned vector access"
        need = 32 * width // 128
        assert wavefronts(lanes, width) == need, (w0, wavefronts(lanes, width), need)


@pytest.mark.parametrize("nt", [256, 128])
def test_geometry_and_shared_memory(nt):
    g = geo(nt)
    assert g["T"] * M == nt
    off_buf = (nt * 32 + 1024 + M * 18 * 8 + 8 * 18 * 8 + 127) // 128 * 128
    smem = off_buf + 2 * g["BUF"] * 8
    per_sm = 2 if nt == 256 else 4
    # per_sm CTAs on an SM: per_sm x (dynamic + static + 1024 reserved) <= 228 KB
    assert per_sm * (smem + 1152 + 1024) <= 228 * 1024
    # the 8-point pair matrix (1 KB) fits the unused C2 twiddle rows
    assert 8 * 18 * 8 >= 1024


@pytest.mark.parametrize("nt", [256, 128])
@pytest.mark.parametrize("dim", [1, 0])
def test_tile_copies(dim, nt):
    g = geo(nt)
    T, NT = g["T"], nt
    seen = np.zeros(g["BUF"], int)
    for i in range(8):
        addrs = []
        for tid in range(NT):
            q = tid + i * NT
            if dim == 1:
                t, e = q >> 6, 2 * (q & 63)
                s = slot_row(g, t, e)
            else:
                e, t = q >> (g["LGT"] - 1), 2 * (q & (T // 2 - 1))
                s = slot_col(g, t, e)
            addrs.append(s)
            seen[s] += 1
            seen[s + 1] += 1
        check_access(g, addrs, 16)
    # every element of the tile lands once
    slots = [slot_row(g, t, e) if dim == 1 else slot_col(g, t, e) for t in range(T) for e in range(N)]
    assert sorted(slots) == sorted(np.nonzero(seen)[0].tolist())
    assert seen.max() == 1


@pytest.mark.parametrize("nt", [256, 128])
@pytest.mark.parametrize("dim", [1, 0])
def test_round_a_and_eight_point_round(dim, nt):
    g = geo(nt)
    T, NT = g["T"], nt
    slot = (lambda t, e: slot_row(g, t, e)) if dim == 1 else (lambda t, e: slot_col(g, t, e))
    written = np.zeros(g["BUF"], int)
    for j in range(16):                      # round A: read x[M j + j2], write Y[M k1 + j2]
        addrs = []
        for v in range(NT):
            t, j2 = (v >> 3, v & 7) if dim == 1 else (v & (T - 1), v >> g["LGT"])
            addrs.append(slot(t, M * j + j2))
            written[slot(t, M * j + j2)] += 1
        check_access(g, addrs, 8)
    assert written.sum() == T * N and written.max() == 1
    read = np.zeros(g["BUF"], int)
    if dim == 1:                             # 8-point round: 8 16-byte pairs per thread
        for c in range(8):
            addrs = []
            for v in range(NT):
                t, p = v >> 3, v & 7
                addrs.append(slot(t, 16 * p) + 2 * c)
                for h in range(2):
                    read[slot(t, 16 * p) + 2 * c + h] += 1
                # the pair is elements 16 p + 2 c, + 1: contiguous in the layout
                assert slot(t, 16 * p) + 2 * c == slot(t, 16 * p + 2 * c)
                assert slot(t, 16 * p + 2 * c) + 1 == slot(t, 16 * p + 2 * c + 1)
            check_access(g, addrs, 16)
    else:
        for j in range(16):
            addrs = []
            for v in range(NT):
                t, p = v & (T - 1), v >> g["LGT"]
                addrs.append(slot(t, 16 * p + j))
                read[slot(t, 16 * p + j)] += 1
            check_access(g, addrs, 8)
    np.testing.assert_array_equal(read, written)
