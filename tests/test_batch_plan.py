"""CPU tests of the batch's work-unit plan (host logic; no GPU needed): the
plan starmap_batch_create uses, on the shapes of the 256-instance workload
and on small corner cases.  Every tile of every instance is covered exactly
once, short tiles go in strips of consecutive tiles in y and long tiles in
strided runs (one item per CTA and instance), and the CTAs get about the
same number of pipeline stages."""
import math

import numpy as np
import pytest

from paper_1211_2205_gb300 import inputs

SMS = 152


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1211_2205_gb300 import capi as c
    return c


def _tiles(items, tiles_x, tiles_y):
    """Per instance, how often each tile is covered."""
    cover = [np.zeros(tx * ty, dtype=np.int64) for tx, ty in zip(tiles_x, tiles_y)]
    for inst, first, count, stride in items:
        assert count >= 1 and stride >= 1
        t = first + stride * np.arange(count)
        assert t.max() < cover[inst].size
        np.add.at(cover[inst], t, 1)
    return cover


def _check(capi, tiles_x, tiles_y, cost, slots):
    items, off = capi.batch_plan(tiles_x, tiles_y, cost, slots)
    grid = off.size - 1
    assert 1 <= grid <= slots
    assert off[0] == 0 and off[-1] == len(items) and np.all(np.diff(off) >= 0)
    for c in _tiles(items, tiles_x, tiles_y):
        assert np.all(c == 1)
    load = np.array([sum(int(items[e, 2]) * cost[items[e, 0]] for e in range(off[c], off[c + 1]))
                     for c in range(grid)])
    return items, off, grid, load


@pytest.mark.parametrize("rows", [10, 5])
def test_workload_plan_covers_every_tile_once_and_balances(capi, rows):
    """The 256 instances of the batched workload (grids 64^2..512^2, N in
    {3..15}) with 64 x `rows` tiles; cost per tile = stages of the longer
    pass, from the kernel's own schedule."""
    tiles_x, tiles_y, cost = [], [], []
    stages = {}
    for k in range(256):
        p = inputs.batched_instance(k)
        extra = 1 if p.bc[0] == "extrapolation" else 0        # node grids hold n + 1 points
        nmax = p.n[0] + extra
        tiles_x.append(math.ceil(nmax / 64))
        tiles_y.append(math.ceil(nmax / rows))
        if p.N not in stages:
            stages[p.N] = max(len(capi.tiled_schedule(p.N, P)[0]) for P in (0, 1))
        cost.append(stages[p.N])
    slots = SMS * (1 if rows == 10 else 2)
    items, off, grid, load = _check(capi, tiles_x, tiles_y, cost, slots)
    assert grid == slots
    # short tiles in strips of consecutive rows, long tiles in runs with stride grid
    for inst, first, count, stride in items:
        if cost[inst] <= 48:
            assert stride == tiles_x[inst]
        else:
            assert stride == grid
    runs = {}
    for e, (inst, first, count, stride) in enumerate(items):
        if cost[inst] > 48:
            cta = int(np.searchsorted(off, e, side="right") - 1)
            assert (inst, cta) not in runs
            runs[(inst, cta)] = count
    # dealt by load, the CTAs stay within 2 % of the mean (plain round
    # robin over the same list left 7 % with 5-row and 12 % with 10-row tiles)
    assert load.max() <= 1.03 * load.mean()
    assert load.min() >= 0.97 * load.mean()


def test_few_small_instances_still_spread_over_the_grid(capi):
    """Four short instances: strips are shortened until there are at least
    four units per CTA or single tiles remain, so no CTA idles needlessly."""
    tiles_x, tiles_y, cost = [2, 1, 3, 2], [40, 13, 52, 7], [6, 6, 10, 6]
    items, off, grid, load = _check(capi, tiles_x, tiles_y, cost, 304)
    tiles = sum(x * y for x, y in zip(tiles_x, tiles_y))
    assert grid == min(304, tiles)
    assert np.count_nonzero(load) == grid


def test_single_tile_and_bad_shapes(capi):
    items, off = capi.batch_plan([1], [1], [5], 152)
    assert off.tolist() == [0, 1] and items.tolist() == [[0, 0, 1, 1]]
    with pytest.raises(capi.StarmapError):
        capi.batch_plan([1, 0], [1, 1], [5, 5], 152)
    with pytest.raises(capi.StarmapError):
        capi.batch_plan([1], [1], [5], 0)
