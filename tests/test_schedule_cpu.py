"""The planner's ticket schedule (host logic, no GPU): the invariants that
make the persistent kernels deadlock-free and keep each grid's
intermediate in L2.

A grid's slab items (z) wait for its plane items (x, y); a ticket holder may
wait only on smaller tickets, so every slab block must come after its grid's
plane block.  Slab blocks trail their plane blocks by the number of items
resident at once (so they rarely wait), unless the intermediates of grids
with planes done and slabs pending would overflow the L2 budget."""
import ctypes

import numpy as np
import pytest

from paper_2006_08435_gb300 import _lib as L


def preview(lib, dims, concurrency, budget, phase_items=0):
    c = len(dims)
    d = (ctypes.c_int * c)(*dims)
    g, ph, st = (ctypes.c_int * (2 * c))(), (ctypes.c_int * (2 * c))(), (ctypes.c_int * (2 * c))()
    nb, tot = ctypes.c_int(), ctypes.c_int()
    rc = lib.fft3d_schedule_preview(c, d, concurrency, float(budget), phase_items, 2 * c,
                                    g, ph, st, ctypes.byref(nb), ctypes.byref(tot))
    assert rc == 0
    return [(g[i], ph[i], st[i]) for i in range(nb.value)], tot.value


def check(blocks, total, dims, concurrency, budget, phase_items=0):
    """Independent statement of the schedule's contract; raises on a breach."""
    items = lambda g: phase_items if phase_items else dims[g]  # noqa: E731
    # tickets contiguous from 0, blocks in ticket order
    t = 0
    for g, ph, st in blocks:
        assert st == t, "tickets not contiguous"
        t += items(g)
    assert t == total
    # one plane and one slab block per grid, plane first
    seen = {}
    for i, (g, ph, _) in enumerate(blocks):
        assert (g, ph) not in seen, "duplicate block"
        seen[(g, ph)] = i
    for g in range(len(dims)):
        assert (g, 0) in seen and (g, 1) in seen, "grid missing a phase"
        assert seen[(g, 0)] < seen[(g, 1)], "slab before its planes"
    # planes largest edge first, ties in grid order
    planes = [g for g, ph, _ in blocks if ph == 0]
    assert planes == sorted(range(len(dims)), key=lambda g: (-dims[g], g))
    # pending intermediates within budget whenever a plane block is emitted
    # (a single grid larger than the budget is allowed alone)
    pending = set()
    for g, ph, _ in blocks:
        if ph == 0:
            pending.add(g)
            b = sum(8.0 * dims[p] ** 3 for p in pending)
            assert b <= budget or len(pending) == 1, "L2 budget exceeded"
        else:
            pending.discard(g)
    # a slab block emitted before the last plane block either trails its
    # plane block by `concurrency` tickets or was forced out by the budget
    last_plane = max(i for i, (_, ph, _) in enumerate(blocks) if ph == 0)
    plane_end = {g: st + items(g) for g, ph, st in blocks if ph == 0}
    for i, (g, ph, st) in enumerate(blocks):
        if ph == 1 and i < last_plane and st - plane_end[g] < concurrency:
            later_plane = next(b for b in blocks[i:] if b[1] == 0)
            pend = {p for p, q, _ in blocks[:i] if q == 0} - {p for p, q, _ in blocks[:i] if q == 1}
            b = sum(8.0 * dims[p] ** 3 for p in pend) + 8.0 * dims[later_plane[0]] ** 3
            assert b > budget, "slab block emitted early without budget pressure"


def test_single_edge_batches_like_the_plans(fft3d_lib):
    """128^3 x 32 and 64^3 x 256 with the plans' parameters: 152 blocks, the
    items each keeps in flight, 40% of a 126.5 MB L2."""
    l2 = 0.4 * 132_644_864
    for dims, conc, pitems in (([128] * 32, 152 * 7, 256), ([64] * 256, 152 * 7, 32)):
        blocks, total = preview(fft3d_lib, dims, conc, l2, pitems)
        check(blocks, total, dims, conc, l2, pitems)
        assert total == 2 * pitems * len(dims)


@pytest.mark.parametrize("seed", range(6))
def test_mixed_edges_random(fft3d_lib, seed):
    rng = np.random.default_rng(seed)
    dims = [int(x) for x in rng.choice([16, 32, 48, 64, 80, 96, 128], size=int(rng.integers(1, 80)))]
    conc = int(rng.integers(0, 3000))
    budget = float(rng.choice([0.0, 5e6, 5e7, 1e12]))
    blocks, total = preview(fft3d_lib, dims, conc, budget)
    check(blocks, total, dims, conc, budget)


def test_degenerate_schedules(fft3d_lib):
    dims = [32, 64, 16]
    # no concurrency: each slab right after its planes
    blocks, _ = preview(fft3d_lib, dims, 0, 1e12)
    assert [(g, ph) for g, ph, _ in blocks] == [(1, 0), (1, 1), (0, 0), (0, 1), (2, 0), (2, 1)]
    # no L2 budget: the same, forced
    blocks, _ = preview(fft3d_lib, dims, 10 ** 6, 0.0)
    assert [(g, ph) for g, ph, _ in blocks] == [(1, 0), (1, 1), (0, 0), (0, 1), (2, 0), (2, 1)]
    # unlimited budget and concurrency: all planes, then all slabs in order
    blocks, _ = preview(fft3d_lib, dims, 10 ** 6, 1e12)
    assert [(g, ph) for g, ph, _ in blocks] == [(1, 0), (0, 0), (2, 0), (1, 1), (0, 1), (2, 1)]
    # one grid
    blocks, total = preview(fft3d_lib, [48], 5, 1e12)
    assert blocks == [(0, 0, 0), (0, 1, 48)] and total == 96


def test_checker_rejects_planted_mistakes(fft3d_lib):
    """The contract check bites: a slab moved before its planes, or two
    blocks swapped out of ticket order, fails it."""
    dims = [64, 64, 32]
    blocks, total = preview(fft3d_lib, dims, 100, 1e12)
    check(blocks, total, dims, 100, 1e12)
    bad = list(blocks)
    i_plane = bad.index(next(b for b in bad if b[:2] == (0, 0)))
    i_slab = bad.index(next(b for b in bad if b[:2] == (0, 1)))
    bad[i_plane], bad[i_slab] = (0, 1, bad[i_plane][2]), (0, 0, bad[i_slab][2])
    with pytest.raises(AssertionError):
        check(bad, total, dims, 100, 1e12)
    swapped = [blocks[1], blocks[0]] + blocks[2:]
    with pytest.raises(AssertionError):
        check(swapped, total, dims, 100, 1e12)


def test_preview_validation(fft3d_lib):
    d = (ctypes.c_int * 2)(64, 64)
    g = (ctypes.c_int * 4)()
    nb, tot = ctypes.c_int(), ctypes.c_int()
    f = fft3d_lib.fft3d_schedule_preview
    assert f(2, None, 1, 1.0, 0, 4, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_NULL_PTR
    assert f(0, d, 1, 1.0, 0, 4, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_INVALID_ARG
    assert f(2, d, 1, 1.0, 0, 3, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_INVALID_ARG
    assert f(2, d, -1, 1.0, 0, 4, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_INVALID_ARG
    assert f(2, d, 1, -1.0, 0, 4, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_INVALID_ARG
    bad = (ctypes.c_int * 2)(64, 0)
    assert f(2, bad, 1, 1.0, 0, 4, g, g, g, ctypes.byref(nb), ctypes.byref(tot)) == L.FFT3D_ERR_INVALID_ARG
