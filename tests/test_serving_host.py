"""Host logic of the serving runtime, without a GPU: the admission arena
(first fit, alignment, coalescing, budget) and the tick planner (tiles, pixel
budget, frame order, ragged tails).  CPU only."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def gl():
    from paper_2507_02674_gb300 import build as B
    B.build()
    from paper_2507_02674_gb300 import glint
    return glint


def test_arena_first_fit_alignment_and_coalescing(gl):
    a = gl.Arena(1 << 20, 256)
    offs = [a.alloc(1000) for _ in range(4)]
    assert offs == [0, 1024, 2048, 3072] and a.used == 4096
    assert a.free(1024) == 0 and a.free(1024) == -1  # double free is refused
    assert a.alloc(1024) == 1024                     # first fit reuses the hole
    assert a.free(1024) == 0 and a.free(2048) == 0   # neighbours coalesce
    assert a.alloc(2048) == 1024
    for o in (0, 1024, 3072):
        assert a.free(o) == 0
    assert a.used == 0 and a.largest_free == 1 << 20
    assert a.alloc((1 << 20) + 1) == -1 and a.alloc(0) == -1


def test_arena_random_workload_never_overlaps(gl):
    rng = np.random.default_rng(0)
    size = 64 << 20
    a = gl.Arena(size, 256)
    live = {}
    for _ in range(3000):
        if live and rng.uniform() < 0.45:
            o = list(live)[rng.integers(len(live))]
            assert a.free(o) == 0
            del live[o]
        else:
            n = int(rng.integers(1, 4 << 20))
            o = a.alloc(n)
            if o < 0:
                assert a.largest_free < -(-n // 256) * 256
                continue
            assert o % 256 == 0 and o + n <= size
            for lo, ln in live.items():
                assert o + n <= lo or lo + ln <= o
            live[o] = n
        assert a.used == sum(-(-n // 256) * 256 for n in live.values())
    for o in list(live):
        a.free(o)
    assert a.used == 0 and a.largest_free == size


def test_planner_tiles_budget_and_order(gl):
    npix = np.array([640 * 360, 3840 * 2160, 100, 1920 * 1080])
    items, nxt = gl.plan_tick(np.zeros(4), npix, tick_pixels=4 << 20, tile_pixels=16384)
    # every unfinished frame gets a tile first, then the budget goes to the
    # frames with the fewest pixels left: 640x360, then 1080p, then the 4K frame
    assert items[:4, 0].tolist() == [0, 1, 2, 3]
    rest = items[4:, 0].tolist()
    assert rest == sorted(rest, key=[0, 2, 3, 1].index)
    for f in range(4):
        it = items[items[:, 0] == f]
        assert it[0, 1] == 0 and np.all(it[1:, 1] == it[:-1, 1] + it[:-1, 2])
        assert np.all(it[:, 1] % 16384 == 0) and np.all(it[:, 2] <= 16384)
    assert nxt[0] == npix[0] and 0 < nxt[1] < npix[1] and nxt[2] == npix[2] and nxt[3] == npix[3]
    planned = items[:, 2].sum()
    assert 4 << 20 <= planned < (4 << 20) + 16384
    # later ticks cover every pixel of every frame exactly once
    nxt = np.zeros(4)
    covered = [np.zeros(n, bool) for n in npix]
    while np.any(nxt < npix):
        items, nxt = gl.plan_tick(nxt, npix, tick_pixels=int(3e6), tile_pixels=16384)
        for f, first, c in items:
            assert not covered[f][first:first + c].any()
            covered[f][first:first + c] = True
    assert all(c.all() for c in covered)


def test_planner_ragged_and_limits(gl):
    items, nxt = gl.plan_tick(np.array([100]), np.array([1000]), tick_pixels=10 ** 9, tile_pixels=256)
    assert items.tolist() == [[0, 100, 156], [0, 256, 256], [0, 512, 256], [0, 768, 232]]
    items, nxt = gl.plan_tick(np.zeros(3), np.array([1000, 1000, 1000]), 10 ** 9, 128, max_items=5)
    assert len(items) == 5 and nxt.tolist() == [384, 128, 128]
    # a small budget still moves every frame by one tile
    items, nxt = gl.plan_tick(np.zeros(3), np.array([1000, 1000, 1000]), 1, 128)
    assert items[:, 0].tolist() == [0, 1, 2] and nxt.tolist() == [128, 128, 128]
