"""Work lists of the grouped launch, checked on the host (no GPU): every
(segment, row tile, column tile) of the lower triangle is covered by its
items exactly once over its k-range; chunks carry slots; the segment-by-
segment order the dynamic schedule takes keeps each segment's items together
(most work first), longest first inside a segment, with the column tiles of a
row tile (or chunk) next to each other."""
import ctypes

import numpy as np
import pytest

OP_ROWS, OP_KB, TC_COLS = 256, 32, 128


@pytest.fixture(scope="module")
def libtd():
    from paper_2603_06010_b300 import build
    build.build()
    from paper_2603_06010_b300 import td
    return td.lib()


def _plan(td, nk, K, bn, S, by_segment):
    lib = td.lib()
    n = len(nk)
    nk_a = (ctypes.c_int64 * n)(*nk)
    K_a = (ctypes.c_int64 * n)(*K)
    cnt = lib.td_debug_plan(nk_a, K_a, n, bn, S, by_segment, None, 0)
    assert cnt <= 0
    cap = -cnt
    out = (ctypes.c_int * max(1, 6 * cap))()
    got = lib.td_debug_plan(nk_a, K_a, n, bn, S, by_segment, out, cap)
    assert got == cap
    return np.frombuffer(out, dtype=np.int32)[:6 * cap].reshape(-1, 6)


def _check_cover(items, nk, K, bn, S):
    per = bn // OP_KB
    for i, (n, k) in enumerate(zip(nk, K)):
        nkp = -(-n // OP_ROWS) * OP_ROWS
        nm, nc, nkb_max = nkp // bn, -(-k // TC_COLS), -(-n // OP_KB)
        mine = items[items[:, 0] == i]
        assert len(mine) == sum(-(-min(per * (m + 1), nkb_max) // S) * nc for m in range(nm)) if k else len(mine) == 0
        for m in range(nm):
            row = min(per * (m + 1), nkb_max)
            for c in range(nc):
                it = mine[(mine[:, 1] == m) & (mine[:, 2] == c)]
                cover = np.zeros(row, np.int32)
                for _, _, _, kb0, nkb, slot in it:
                    assert 0 <= kb0 and nkb >= 1 and kb0 + nkb <= row
                    cover[kb0:kb0 + nkb] += 1
                    assert (slot >= 0) == (row > S)   # split rows write accumulator slots
                assert np.all(cover == 1), (i, m, c)


@pytest.mark.parametrize("case", range(12))
def test_plan_covers_each_tile_once(libtd, case):
    from paper_2603_06010_b300 import td
    rng = np.random.default_rng(31000 + case)
    nseg = int(rng.integers(1, 9))
    nk = [int(x) for x in rng.integers(1, 9000, nseg)]
    K = [int(rng.choice([0, 1, 100, 128, 129, 300, 512])) for _ in range(nseg)]
    bn = int(rng.choice([256, 128, 64]))
    S = int(rng.choice([4, 17, 64, 1000]))
    for by_segment in (0, 1):
        items = _plan(td, nk, K, bn, S, by_segment)
        _check_cover(items, nk, K, bn, S)


def test_plan_order_segment_by_segment(libtd):
    from paper_2603_06010_b300 import td
    nk = [3000, 8000, 700, 8000, 5000]
    K = [300, 129, 512, 16, 0]
    items = _plan(td, nk, K, 256, 40, 1)
    _check_cover(items, nk, K, 256, 40)
    seg = items[:, 0]
    blocks = [seg[0]] + [s for a, s in zip(seg[:-1], seg[1:]) if s != a]
    assert len(blocks) == len(set(blocks)) == 4   # one block per segment with work
    work = [int(items[seg == s][:, 4].sum()) for s in blocks]
    assert work == sorted(work, reverse=True)
    for s in blocks:
        mine = items[seg == s]
        assert np.all(np.diff(mine[:, 4]) <= 0)                  # longest first
        for j in range(1, len(mine)):                            # column tiles together
            if mine[j, 2] > 0:
                assert tuple(mine[j - 1, [1, 3]]) == tuple(mine[j, [1, 3]]) and mine[j - 1, 2] == mine[j, 2] - 1


def test_plan_order_longest_first(libtd):
    from paper_2603_06010_b300 import td
    items = _plan(td, [3000, 8000, 700], [300, 129, 512], 128, 40, 0)
    assert np.all(np.diff(items[:, 4]) <= 0)


def test_plan_bad_arguments(libtd):
    from paper_2603_06010_b300 import td
    lib = td.lib()
    one = (ctypes.c_int64 * 1)(100)
    assert lib.td_debug_plan(one, one, 1, 96, 8, 0, None, 0) == -1      # tile height
    assert lib.td_debug_plan(one, one, 1, 256, 0, 0, None, 0) == -1     # chunk
    assert lib.td_debug_plan(one, one, 0, 256, 8, 0, None, 0) == -1     # no segments
