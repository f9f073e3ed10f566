"""Design check of the fused 2D tensor-core kernel's index maps (mx_tc2d.cu),
re-derived on the CPU for every slice shape it serves: the shared-memory
budget, the slab's bulk copies, the statistics read, the row rounds, the
gather of column tiles through distributed shared memory, the column rounds
and the global stores.  Every access must stay inside its buffer and every
element must be covered exactly once where the kernel relies on it."""
import numpy as np
import pytest

THREADS, TILE, SLAB = 256, 4096, 16384
TWROW = 17
SMEM_MAX = 232448 - 1024          # opt-in limit minus the static shared memory


class Ax:
    def __init__(self, n):
        self.n = n
        self.r = n // 256
        self.LGR = 0 if self.r == 1 else 1
        self.M = 16 * self.r
        self.LGM = 4 + self.LGR
        self.T = TILE // n
        self.LGT = 4 if self.T == 16 else 3
        self.PADR = 2
        self.TS = n + self.PADR * (n // self.M)


class Geo:
    def __init__(self, n0, n1):
        self.A0, self.A1 = Ax(n0), Ax(n1)
        self.n0, self.n1 = n0, n1
        self.C = n0 * n1 // SLAB
        self.R = SLAB // n1
        self.Cc = n1 // self.C
        self.ROW_TILES = self.R // self.A1.T
        self.COL_TILES = self.Cc // self.A0.T
        self.SLAB_SLOTS = self.R * self.A1.TS
        A0 = self.A0
        self.STG_SLOTS = n0 * A0.T + (A0.T * (n0 // 16) if A0.T < 16 else 0)
        off = 8192 + 2048
        off += self.A1.M * TWROW * 16 + self.A1.r * TWROW * 16
        off += A0.M * TWROW * 16 + A0.r * TWROW * 16
        off += (4 + 280) * 4
        self.OFF_SLAB = (off + 127) // 128 * 128
        self.SMEM = self.OFF_SLAB + self.SLAB_SLOTS * 8 + self.STG_SLOTS * 8


def slot_row(A, t, e):
    return t * A.TS + e + A.PADR * (e >> A.LGM)


def slot_col(A, t, e):
    return e * A.T + (A.T * (e >> 4) if A.T < 16 else 0) + t


SHAPES = [(256, 256), (256, 512), (512, 256), (512, 512)]


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_geometry_and_shared_memory(n0, n1):
    g = Geo(n0, n1)
    assert g.C in (4, 8, 16) and g.C * g.R == n0 and g.C * g.Cc == n1
    assert g.ROW_TILES == 4 and g.COL_TILES == 4
    assert g.SMEM <= SMEM_MAX
    assert g.STG_SLOTS * 8 >= (4 + 280) * 4        # the cluster totals fit the staging tile
    assert g.OFF_SLAB % 16 == 0 and (g.OFF_SLAB + g.SLAB_SLOTS * 8) % 16 == 0


def data_slots(g):
    """Slab slots that hold data (natural element e of slab row t)."""
    A1 = g.A1
    s = np.array([slot_row(A1, t, e) for t in range(g.R) for e in range(g.n1)])
    return s


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_slab_copies_cover_the_slab_once(n0, n1):
    g, A1 = Geo(n0, n1), Geo(n0, n1).A1
    runs = g.R * (A1.n // A1.M)
    cover = np.zeros(g.SLAB_SLOTS, np.int32)
    for rank in range(g.C):
        src_seen = set()
        for q in range(runs):
            row, run = q // (A1.n // A1.M), q % (A1.n // A1.M)
            dst = slot_row(A1, row, run * A1.M)
            assert (dst * 8) % 16 == 0 and (A1.M * 8) % 16 == 0
            src = (rank * g.R + row) * A1.n + run * A1.M          # element offset in the slice
            assert src % 2 == 0 and 0 <= src and src + A1.M <= n0 * n1
            src_seen.add(src)
            if rank == 0:
                cover[dst:dst + A1.M] += 1
        assert len(src_seen) == runs
    assert cover.max() == 1 and cover.sum() == g.R * g.n1
    assert set(np.nonzero(cover)[0]) == set(data_slots(g).tolist())
    assert cover.shape[0] == g.SLAB_SLOTS


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_statistics_read_every_point_once(n0, n1):
    g = Geo(n0, n1)
    seen = np.zeros(g.SLAB_SLOTS, np.int32)
    for tid in range(THREADS):
        for i in range(SLAB // 2 // THREADS):
            c = tid + i * THREADS
            row, col = c // (g.n1 // 2), 2 * (c % (g.n1 // 2))
            s = slot_row(g.A1, row, col)
            assert s % 2 == 0
            seen[s] += 1
            seen[s + 1] += 1
    assert seen.max() == 1 and seen.sum() == SLAB
    assert set(np.nonzero(seen)[0]) == set(data_slots(g).tolist())


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_row_rounds_stay_in_their_tile_and_end_in_natural_order(n0, n1):
    g = Geo(n0, n1)
    A1 = g.A1
    tile_slots = A1.T * A1.TS
    for rt in range(g.ROW_TILES):
        base = rt * tile_slots
        assert base + tile_slots <= g.SLAB_SLOTS
        # round A: vector (t, j2) reads and writes x[M j1 + j2]; all vectors
        # together touch each data slot of the tile once
        cov = np.zeros(tile_slots, np.int32)
        for tid in range(THREADS):
            t, j2 = tid >> A1.LGM, tid & (A1.M - 1)
            for j in range(16):
                cov[slot_row(A1, t, A1.M * j + j2)] += 1
        assert cov.max() == 1 and cov.sum() == TILE
        # round C1
        cov[:] = 0
        outs = np.zeros(tile_slots, np.int32)
        for tid in range(THREADS):
            t, rem = tid >> A1.LGM, tid & (A1.M - 1)
            k1, j22 = rem >> A1.LGR, rem & (A1.r - 1)
            for j in range(16):
                cov[slot_row(A1, t, A1.M * k1 + A1.r * j + j22)] += 1
            if A1.r == 1:
                for k in range(16):
                    outs[slot_row(A1, t, k1 + 16 * k)] += 1
        assert cov.max() == 1 and cov.sum() == TILE
        if A1.r == 1:
            assert outs.max() == 1 and outs.sum() == TILE
        else:
            # C2: reads each pair once, writes each natural position once
            rd = np.zeros(tile_slots, np.int32)
            wr = np.zeros(tile_slots, np.int32)
            for tid in range(THREADS):
                for i in range(8):
                    u = tid + i * THREADS
                    c1, k21, tt = u & 15, (u >> 4) & 15, u >> 8
                    s = slot_row(A1, tt, A1.M * c1 + 2 * k21)
                    assert s % 2 == 0
                    rd[s] += 1
                    rd[s + 1] += 1
                    wr[slot_row(A1, tt, c1 + 16 * k21)] += 1
                    wr[slot_row(A1, tt, c1 + 16 * k21 + 256)] += 1
            assert rd.max() == 1 and rd.sum() == TILE
            assert wr.max() == 1 and wr.sum() == TILE
        # natural-order results and round inputs use the same data slots
        nat = {slot_row(A1, t, e) for t in range(A1.T) for e in range(A1.n)}
        assert nat == set(np.nonzero(cov)[0].tolist())


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_gather_fills_each_staging_slot_from_the_right_element(n0, n1):
    g = Geo(n0, n1)
    A0, A1 = g.A0, g.A1
    CPR = A0.T // 2
    for rank in (0, g.C - 1):
        for q in range(g.COL_TILES):
            col0 = g.Cc * rank + A0.T * q
            stg = np.full(g.STG_SLOTS, -1, np.int64)
            for tid in range(THREADS):
                for i in range(8):
                    gi = tid + i * THREADS
                    j, rem = gi // (g.R * CPR), gi % (g.R * CPR)
                    rho, c2 = rem // CPR, rem % CPR
                    assert 0 <= j < g.C
                    src = slot_row(A1, rho, col0 + 2 * c2)
                    assert src % 2 == 0 and src + 2 <= g.SLAB_SLOTS
                    dst = slot_col(A0, 2 * c2, g.R * j + rho)
                    assert dst % 2 == 0 and dst + 2 <= g.STG_SLOTS
                    for h in range(2):
                        assert stg[dst + h] == -1
                        # global (row, column) of the element the slab slot holds
                        stg[dst + h] = (g.R * j + rho) * n1 + col0 + 2 * c2 + h
            want = {slot_col(A0, t, e): e * n1 + col0 + t for t in range(A0.T) for e in range(n0)}
            got = {s: int(v) for s, v in enumerate(stg) if v >= 0}
            assert got == want


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_column_rounds_and_stores_cover_the_slice_once(n0, n1):
    g = Geo(n0, n1)
    A0 = g.A0
    stored = np.zeros(n0 * n1, np.int32)
    for rank in range(g.C):
        for q in range(g.COL_TILES):
            col0 = g.Cc * rank + A0.T * q
            cov = np.zeros(g.STG_SLOTS, np.int32)
            for tid in range(THREADS):                   # round A
                t, j2 = tid & (A0.T - 1), tid >> A0.LGT
                for j in range(16):
                    cov[slot_col(A0, t, A0.M * j + j2)] += 1
            assert cov.max() == 1 and cov.sum() == TILE
            cov[:] = 0
            for tid in range(THREADS):                   # round C1
                t, rem = tid & (A0.T - 1), tid >> A0.LGT
                k1, j22 = rem >> A0.LGR, rem & (A0.r - 1)
                for j in range(16):
                    cov[slot_col(A0, t, A0.M * k1 + A0.r * j + j22)] += 1
                if A0.r == 1:
                    for k in range(16):
                        stored[(k1 + 16 * k) * n1 + col0 + t] += 1
            assert cov.max() == 1 and cov.sum() == TILE
            if A0.r == 2:                                # C2
                rd = np.zeros(g.STG_SLOTS, np.int32)
                for tid in range(THREADS):
                    for i in range(8):
                        u = tid + i * THREADS
                        tt, k21, c1 = u & 7, 8 * ((u >> 3) & 1) + (u >> 8), (u >> 4) & 15
                        e = A0.M * c1 + 2 * k21
                        rd[slot_col(A0, tt, e)] += 1
                        rd[slot_col(A0, tt, e + 1)] += 1
                        e0 = c1 + 16 * k21
                        stored[e0 * n1 + col0 + tt] += 1
                        stored[(e0 + 256) * n1 + col0 + tt] += 1
                assert rd.max() == 1 and rd.sum() == TILE
    assert stored.min() == 1 and stored.max() == 1


@pytest.mark.parametrize("n0,n1", SHAPES)
def test_twiddle_reads_stay_in_their_tables(n0, n1):
    g = Geo(n0, n1)
    for A in (g.A0, g.A1):
        # round A: row j2 < M of 16 entries; round C1: row j22 < r
        assert max(j2 * TWROW + 15 for j2 in range(A.M)) < A.M * TWROW
        assert max(j22 * TWROW + 15 for j22 in range(A.r)) < A.r * TWROW
