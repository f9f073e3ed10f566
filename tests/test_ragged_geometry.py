"""Design check of the ragged register-resident launch (mx_fast_ragged.cu,
the executor's ragged phases), re-derived on the CPU: every group gets 256
threads per CTA (TG transforms of n / 32 slots, NG groups), its shared rows
fit, its CTA table entries (slice, first transform) cover every transform of
every slice exactly once, and the lanes that hold one MX block of 16
butterflies (slots sigma and sigma ^ 1, TG lanes apart) share a warp."""
import pytest

THREADS = 256


def geometry(n, other, m=16):
    """(TG, S, NG) of the ragged pass or None (mirror of fast_ragged_geometry)."""
    if m != 16 or n < 64 or n > 1024:
        return None
    tg = 8 if n == 1024 else 16
    s = 16 if tg == 16 else tg + 1
    per_group = tg * (n // 32)
    if per_group > THREADS or THREADS % per_group:
        return None
    ng = THREADS // per_group
    if other % (tg * ng):
        return None
    return tg, s, ng


@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024])
@pytest.mark.parametrize("other", [64, 128, 256, 512, 1024, 2048])
def test_ragged_geometry_covers_every_transform_once(n, other):
    g = geometry(n, other)
    if g is None:            # the group keeps its per-plan launch
        assert other % (THREADS * 32 // n if n < 1024 else 8) != 0
        return
    tg, s, ng = g
    assert tg * (n // 32) * ng == THREADS
    assert ng * n * s * 8 <= 227 * 1024
    tpc = tg * ng
    for slices in (1, 3):
        seen = {}
        entries = [(sl, t0) for sl in range(slices) for t0 in range(0, other, tpc)]
        for sl, t0 in entries:
            for tid in range(THREADS):
                lg_pg = (tg.bit_length() - 1) + (n.bit_length() - 1) - 5
                grp, w = tid >> lg_pg, tid & ((1 << lg_pg) - 1)
                tau = w & (tg - 1)
                tr = t0 + grp * tg + tau
                assert 0 <= tr < other
                seen[(sl, tr)] = seen.get((sl, tr), 0) + 1
        # every transform: n / 32 slot threads, each once per transform
        assert set(seen) == {(sl, t) for sl in range(slices) for t in range(other)}
        assert set(seen.values()) == {n // 32}


@pytest.mark.parametrize("n", [128, 256, 512, 1024])
def test_block_partner_lanes_share_a_warp(n):
    tg, s, ng = geometry(n, 2048)
    lg_tg = tg.bit_length() - 1
    for tid in range(THREADS):
        lane = tid & 31
        w = tid & ((1 << (lg_tg + (n.bit_length() - 1) - 5)) - 1)
        sigma = w >> lg_tg
        partner = tid ^ tg                     # slot sigma ^ 1, same transform
        assert (partner >> 5) == (tid >> 5), (n, tid)
        assert ((partner & ((1 << (lg_tg + (n.bit_length() - 1) - 5)) - 1)) >> lg_tg) == sigma ^ 1
        assert lane ^ tg == partner & 31
