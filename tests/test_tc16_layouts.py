"""Design check of the tensor-core pass's shared-memory layouts (no GPU),
re-derived from its index maps for n = 256 r, r in {1, 2, 4, 8}, on both CTA
shapes (256 threads with 4096-point tiles; 128 threads with 2048-point tiles
for n <= 1024): every element of a tile has its own slot inside the buffer, the
cp.async copies write 16-byte aligned pairs that cover the tile once, rounds
A, C1 and C2 each visit every element once, and their shared-memory accesses
take the minimum number of wavefronts (no bank conflicts): 8-byte accesses in
groups of 16 lanes, 16-byte accesses in groups of 8."""
from collections import Counter

import pytest


def geo(logn, nt=256):
    n = 1 << logn
    r = n // 256
    M = 16 * r
    T = 16 * nt // n
    padr = {1: 2, 2: 2, 4: 4, 8: 8}[r]
    ts = n + padr * (n // M)
    rows = T * ts
    cols = n * T + (T * (n // 16) if T < 16 else 0)
    return dict(n=n, r=r, M=M, LGM=M.bit_length() - 1, LGR=r.bit_length() - 1, T=T,
                LGT=T.bit_length() - 1, TS=ts, PADR=padr, BUF=max(rows, cols), NT=nt)


def slot(g, dim, t, e):
    if dim == 1:
        return t * g["TS"] + e + g["PADR"] * (e >> g["LGM"])
    return e * g["T"] + (g["T"] * (e >> 4) if g["T"] < 16 else 0) + t


def extra_wavefronts(addrs, width):
    """Wavefronts beyond the minimum for one warp's accesses of `width` bytes."""
    per = 128 // width
    x = 0
    for q in range(0, 32, per):
        c = Counter((a // width) % per for a in addrs[q:q + per])
        x += max(c.values()) - 1
    return x


def c2_item(g, dim, u):
    """(t, k1, k21) of the C2 work item u (T x 16 x 16 items)."""
    T, r = g["T"], g["r"]
    if dim == 1:
        return u >> 8, u & 15, (u >> 4) & 15
    if T == 8:
        return u & 7, (u >> 4) & 15, 8 * ((u >> 3) & 1) + (u >> 8)
    if T == 4 and r == 2:                                           # 128 threads, n = 512
        return u & 3, (u >> 4) & 15, (((u >> 2) & 1) << 3) | ((u >> 3) & 1) | (((u >> 8) & 3) << 1)
    if T == 4:
        return u & 3, (u >> 4) & 15, 4 * ((u >> 2) & 3) + (u >> 8)
    if r == 4:                                                      # 128 threads, n = 1024
        return u & 1, (u >> 4) & 15, (((u >> 1) & 3) << 2) | ((u >> 3) & 1) | (((u >> 8) & 1) << 1)
    return u & 1, (u >> 4) & 15, 2 * ((u >> 1) & 7) + (u >> 8)      # T == 2, n = 2048


@pytest.mark.parametrize("logn,nt", [(8, 256), (9, 256), (10, 256), (11, 256),
                                     (8, 128), (9, 128), (10, 128)])
@pytest.mark.parametrize("dim", [0, 1])
def test_tile_layout(logn, nt, dim):
    g = geo(logn, nt)
    n, r, M, T = g["n"], g["r"], g["M"], g["T"]
    nw = nt // 32
    slots = {slot(g, dim, t, e) for t in range(T) for e in range(n)}
    assert len(slots) == T * n and min(slots) >= 0 and max(slots) < g["BUF"]
    # cp.async: 8 copies of 16 bytes per thread, 256 threads
    cov = Counter()
    for q in range(8 * nt):
        if dim == 1:
            t, e = q >> (logn - 1), 2 * (q & ((n >> 1) - 1))
            pair = [(t, e), (t, e + 1)]
        else:
            e, t = q >> (g["LGT"] - 1), 2 * (q & ((T >> 1) - 1))
            pair = [(t, e), (t + 1, e)]
        s0 = slot(g, dim, *pair[0])
        assert s0 % 2 == 0 and slot(g, dim, *pair[1]) == s0 + 1
        cov.update(pair)
    assert len(cov) == T * n and set(cov.values()) == {1}
    # round A: vector v = (t, j2), elements M j + j2
    seen, x = Counter(), 0
    for j in range(16):
        ad = []
        for v in range(nt):
            t, j2 = (v >> g["LGM"], v & (M - 1)) if dim == 1 else (v & (T - 1), v >> g["LGT"])
            seen[(t, M * j + j2)] += 1
            ad.append(8 * slot(g, dim, t, M * j + j2))
        x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 8) for w in range(nw))
    assert len(seen) == T * n and set(seen.values()) == {1} and x == 0
    # round C1: vector (t, k1, j22), elements M k1 + r j + j22 (r = 1: 16-byte pairs)
    seen, x = Counter(), 0
    for j in range(16):
        ad = []
        for v in range(nt):
            t, rem = (v >> g["LGM"], v & (M - 1)) if dim == 1 else (v & (T - 1), v >> g["LGT"])
            k1, j22 = rem >> g["LGR"], rem & (r - 1)
            e = M * k1 + r * j + j22
            seen[(t, e)] += 1
            ad.append(8 * slot(g, dim, t, e))
        if dim == 1 and r == 1:
            if j % 2 == 0:
                x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 16) for w in range(nw))
        else:
            x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 8) for w in range(nw))
    assert len(seen) == T * n and set(seen.values()) == {1} and x == 0
    # round C2 (r > 1): item (t, k1, k21) reads elements M k1 + r k21 + j22
    if r == 1:
        return
    seen, x = Counter(), 0
    for i in range(T * 256 // nt):
        items = [c2_item(g, dim, tid + i * nt) for tid in range(nt)]
        for t, k1, k21 in items:
            assert t < T and k1 < 16 and k21 < 16
            for j22 in range(r):
                seen[(t, M * k1 + r * k21 + j22)] += 1
        if dim == 1 and r in (4, 8):
            # 16-byte chunks read in a per-lane order (r = 4: swap when bit 2
            # of k1 is set; r = 8: chunk c ^ ((k1 >> 1) & 3))
            for step in range(r // 2):
                ad = []
                for t, k1, k21 in items:
                    c = (step ^ ((k1 >> 2) & 1)) if r == 4 else (step ^ ((k1 >> 1) & 3))
                    ad.append(8 * slot(g, dim, t, M * k1 + r * k21) + 16 * c)
                x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 16) for w in range(nw))
        elif dim == 1:   # r = 2: one 16-byte pair per item
            ad = [8 * slot(g, dim, t, M * k1 + r * k21) for t, k1, k21 in items]
            x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 16) for w in range(nw))
        else:
            for j22 in range(r):
                ad = [8 * slot(g, dim, t, M * k1 + r * k21 + j22) for t, k1, k21 in items]
                x += sum(extra_wavefronts(ad[32 * w:32 * w + 32], 8) for w in range(nw))
    assert len(seen) == T * n and set(seen.values()) == {1}
    assert x == 0, x
