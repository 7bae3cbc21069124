"""Mixed-edge batches (64 grids, edges from {32, 48, 64, 80, 96, 128}):
forward then inverse inside one captured CUDA graph, the launch schedules
of a mixed plan (one launch, one per edge, one per edge as concurrent
branches), and the autotuner on the device."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2006_08435_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6


def _packed(sizes, seed):
    grids = synth.mixed_grids(sizes, seed=seed)
    return grids, torch.from_numpy(np.concatenate([g.ravel() for g in grids])).cuda()


@pytest.fixture
def mixed_env():
    old = os.environ.get("FFT3D_MIXED_VARIANT")
    yield
    if old is None:
        os.environ.pop("FFT3D_MIXED_VARIANT", None)
    else:
        os.environ["FFT3D_MIXED_VARIANT"] = old


def test_config2_forward_inverse_in_one_graph(cuda):
    """Both transforms of all 64 grids are captured once and replayed on new
    data; every grid round-trips and one grid of each edge matches the
    oracle."""
    from paper_2006_08435_gb300 import MixedPlan
    sizes = synth.mixed_sizes(64, seed=0)
    fwd = MixedPlan(sizes)
    inv = MixedPlan(sizes, inverse=True)
    x = torch.zeros(fwd.total_points, dtype=torch.complex64, device="cuda")
    y, back = torch.empty_like(x), torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fwd.execute(x, y)
        inv.execute(y, back)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fwd.execute(x, y)
        inv.execute(y, back)
    grids, packed = _packed(sizes, seed=1)
    x.copy_(packed)
    g.replay()
    torch.cuda.synchronize()
    assert fwd.device_status() == 0 and inv.device_status() == 0
    off = fwd.offsets
    yc, bc = y.cpu().numpy(), back.cpu().numpy()
    seen = set()
    for i, n in enumerate(sizes):
        seg = bc[off[i]:off[i + 1]] / float(n) ** 3
        assert oracle.rel_l2(seg, grids[i].ravel()) <= 2 * FP32_TOL
        if n not in seen:
            seen.add(n)
            ref = oracle.dft3d(grids[i].astype(np.complex128), -1)
            assert oracle.rel_l2(yc[off[i]:off[i + 1]].reshape(n, n, n), ref) <= FP32_TOL


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_mixed_schedules_agree(cuda, mixed_env, variant):
    """One mixed-edge launch (0), one launch per edge (1) and the same as
    concurrent branches (2), packed and pointer-array addressing, give the
    same spectra."""
    from paper_2006_08435_gb300 import MixedPlan
    sizes = [128, 32, 48, 128, 64, 96, 80, 32, 64]
    grids, packed = _packed(sizes, seed=2)
    os.environ["FFT3D_MIXED_VARIANT"] = str(variant)
    p = MixedPlan(sizes)
    assert p.variant == variant
    y = torch.empty_like(packed)
    p.execute(packed, y)
    outs = [torch.empty(n ** 3, dtype=torch.complex64, device="cuda") for n in sizes]
    ins = [packed[p.offsets[i]:p.offsets[i + 1]].clone() for i in range(len(sizes))]
    ip = torch.tensor([t.data_ptr() for t in ins], dtype=torch.int64, device="cuda")
    op = torch.tensor([t.data_ptr() for t in outs], dtype=torch.int64, device="cuda")
    p.execute_ptrs(ip, op)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    yc = y.cpu().numpy()
    for i, n in enumerate(sizes):
        ref = oracle.dft3d(grids[i].astype(np.complex128), -1)
        assert oracle.rel_l2(yc[p.offsets[i]:p.offsets[i + 1]].reshape(n, n, n), ref) <= FP32_TOL
        assert oracle.rel_l2(outs[i].cpu().numpy().reshape(n, n, n), ref) <= FP32_TOL


def test_per_edge_schedule_with_many_grids_per_edge(cuda, mixed_env):
    """One launch per edge (variant 1) when an edge has enough grids that its
    default kernel would be a tensor-map kernel (which needs one packed
    batch): the 64 grids of the mixed workload agree with the one-launch
    schedule, and sampled grids with the oracle; calls with pointer arrays
    (other kernels for those edges) agree with the packed ones."""
    from paper_2006_08435_gb300 import MixedPlan
    sizes = synth.mixed_sizes(64, seed=0) + [64] * 16
    grids, packed = _packed(sizes, seed=8)
    outs = []
    for variant in (0, 1, 2):
        os.environ["FFT3D_MIXED_VARIANT"] = str(variant)
        p = MixedPlan(sizes)
        assert p.variant == variant
        y = torch.empty_like(packed)
        p.execute(packed, y)
        torch.cuda.synchronize()
        assert p.device_status() == 0
        outs.append(y)
    assert oracle.rel_l2(outs[1].cpu().numpy(), outs[0].cpu().numpy()) <= FP32_TOL
    # the same kernels on the same grids, concurrently: the same bits
    assert torch.equal(outs[2], outs[1])
    # pointer arrays: the edges whose packed units use per-grid tensor maps
    # (128^3 split-y, 96^3 / 80^3 thread pairs) run kernels that address
    # grids through pointers instead; every grid agrees with the packed call
    ins = [packed[p.offsets[i]:p.offsets[i + 1]].clone() for i in range(len(sizes))]
    res = [torch.empty_like(t) for t in ins]
    ip = torch.tensor([t.data_ptr() for t in ins], dtype=torch.int64, device="cuda")
    op = torch.tensor([t.data_ptr() for t in res], dtype=torch.int64, device="cuda")
    p.execute_ptrs(ip, op)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    for i in range(len(sizes)):
        seg = outs[2][p.offsets[i]:p.offsets[i + 1]]
        assert oracle.rel_l2(res[i].cpu().numpy(), seg.cpu().numpy()) <= FP32_TOL, i
    yc = outs[1].cpu().numpy()
    for i in (sizes.index(128), len(sizes) - 1):
        n = sizes[i]
        ref = oracle.dft3d(grids[i].astype(np.complex128), -1)
        assert oracle.rel_l2(yc[p.offsets[i]:p.offsets[i + 1]].reshape(n, n, n), ref) <= FP32_TOL


def test_autotune_records_and_plans_use_the_choice(cuda, tmp_path, monkeypatch):
    from paper_2006_08435_gb300 import Plan, MixedPlan, autotune, autotune_mixed
    cache = str(tmp_path / "tune.json")
    best = autotune(64, 16, cache_path=cache)
    assert best in (0, 1, 5, 7, 8, 10)  # the 64^3 candidates
    sizes = synth.mixed_sizes(16, seed=3)
    best_m = autotune_mixed(sizes, cache_path=cache)
    assert best_m in (0, 1, 2)
    entries = json.load(open(cache))
    assert len(entries) == 2 and best in entries.values()
    monkeypatch.delenv("FFT3D_VARIANT", raising=False)
    monkeypatch.delenv("FFT3D_MIXED_VARIANT", raising=False)
    monkeypatch.setenv("FFT3D_TUNE_CACHE", cache)
    assert Plan(64, 64, 64, 16).variant == best
    assert MixedPlan(sizes).variant == best_m
    # a tuned plan still computes Eq. 1
    x = torch.from_numpy(synth.uniform_grids(64, 16, seed=4)).cuda()
    y = torch.empty_like(x)
    Plan(64, 64, 64, 16).execute(x, y)
    ref = oracle.dft3d(x[5].cpu().numpy().astype(np.complex128), -1)
    assert oracle.rel_l2(y[5].cpu().numpy(), ref) <= FP32_TOL


def test_per_grid_tensor_maps_in_place_and_beyond_the_table(cuda, mixed_env):
    """One launch per edge on packed buffers: the 128^3 grids run the split-y
    kernel with one pair of tensor maps per grid, also in place (in == out)
    with distinct grids; with more 128^3 grids than one launch takes maps for
    (33 > 32) the unit falls back to the warp-owned kernel; 96^3 and 80^3
    grids (4 and 9 of them) run the thread-pair kernel with per-grid maps.
    Sampled grids against the oracle, every grid back through the inverse."""
    from paper_2006_08435_gb300 import MixedPlan
    for variant, sizes in (("1", [128, 32, 128, 64, 128, 96, 128]), ("2", [128, 32, 128, 64, 128, 96, 128]),
                           ("1", [32] + [128] * 33), ("2", [96, 48, 96, 96, 80, 96] + [80] * 8)):
        os.environ["FFT3D_MIXED_VARIANT"] = variant
        grids, packed = _packed(sizes, seed=len(sizes))
        fwd, inv = MixedPlan(sizes), MixedPlan(sizes, inverse=True)
        x = packed.clone()
        fwd.execute(x, x)  # in place
        torch.cuda.synchronize()
        assert fwd.device_status() == 0
        xc = x.cpu().numpy()
        big = 128 if 128 in sizes else 96
        idx = [i for i, n in enumerate(sizes) if n == big]
        for i in (idx[0], idx[-1], 0, len(sizes) - 1):
            n = sizes[i]
            ref = oracle.dft3d(grids[i].astype(np.complex128), -1)
            assert oracle.rel_l2(xc[fwd.offsets[i]:fwd.offsets[i + 1]].reshape(n, n, n), ref) <= FP32_TOL
        back = torch.empty_like(x)
        inv.execute(x, back)
        torch.cuda.synchronize()
        assert inv.device_status() == 0
        bc, pc = back.cpu().numpy(), packed.cpu().numpy()
        for i, n in enumerate(sizes):
            seg = slice(fwd.offsets[i], fwd.offsets[i + 1])
            assert oracle.rel_l2(bc[seg] / float(n) ** 3, pc[seg]) <= 2 * FP32_TOL


def test_concurrent_branches_in_a_captured_graph(cuda, mixed_env):
    """Mixed variant 2 (the per-edge launches as concurrent branches on the
    plan's side streams) captured in a CUDA graph with its inverse: replays
    give the bits of the eager calls, and the round trip is n^3 times the
    input."""
    from paper_2006_08435_gb300 import MixedPlan
    os.environ["FFT3D_MIXED_VARIANT"] = "2"
    sizes = [128, 32, 48, 128, 64, 96, 80, 32, 64]
    grids, packed = _packed(sizes, seed=21)
    fwd, inv = MixedPlan(sizes), MixedPlan(sizes, inverse=True)
    assert fwd.variant == 2 and inv.variant == 2
    y, back = torch.empty_like(packed), torch.empty_like(packed)
    fwd.execute(packed, y)
    inv.execute(y, back)
    torch.cuda.synchronize()
    y_eager, back_eager = y.clone(), back.clone()
    y.zero_()
    back.zero_()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fwd.execute(packed, y)
        inv.execute(y, back)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fwd.execute(packed, y)
        inv.execute(y, back)
    y.zero_()
    back.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert fwd.device_status() == 0 and inv.device_status() == 0
    assert torch.equal(y, y_eager) and torch.equal(back, back_eager)
    bc, pc = back.cpu().numpy(), packed.cpu().numpy()
    for i, n in enumerate(sizes):
        seg = slice(fwd.offsets[i], fwd.offsets[i + 1])
        assert oracle.rel_l2(bc[seg] / float(n) ** 3, pc[seg]) <= 2 * FP32_TOL
    i = sizes.index(96)
    ref = oracle.dft3d(grids[i].astype(np.complex128), -1)
    yc = y.cpu().numpy()
    assert oracle.rel_l2(yc[fwd.offsets[i]:fwd.offsets[i + 1]].reshape(96, 96, 96), ref) <= FP32_TOL
