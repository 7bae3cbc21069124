"""Benchmark: batched 3D C2C FFT throughput (transforms/s) and fraction of
the HBM roofline on one GB300, plus end-to-end throughput with host buffers
and the FP64 oracle timed on the host cores.

Step = one forward 3D FFT (Eq. 1, FP32) of a batch of complex64 grids
already resident in HBM (default 128^3 x 32 = 537 MB in, 537 MB out, larger
than L2, so no flush is needed between steps).  Roofline bytes per
transform = 16 * N^3 (one read and one write of the grid).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 128x32|64x256|128x16|64x64|64x128|256x2|96x16]
                  [--no-cpu-baseline]
                  [--no-e2e] [--no-split] [--no-real] [--no-64] [--no-mixed] [--no-batch1]
                  [--no-general] [--no-hartree]

The small workloads exist for profiler captures of the same kernels.  Beside
the headline the line carries sub-objects: split_fp16 (the same batch in
split FP16), tensor_core_kinds (split BF16, FP16, block floating point
FP16, split FP8, FP8 on the same batch), real_r2c_fp32 / real_c2r_fp32 (real grids),
real_16cubed_fp32 (16^3 x 16384 real grids), w64x256 (64^3 x 256 in FP32 and
split FP16), mixed_c2 (64 mixed-edge grids, forward + inverse in one CUDA
graph), general_path (256^3 and a non-cubic batch on the per-axis passes), hartree
(energy + gradient of real densities, the differentiation workload; one
density also replayed from a captured CUDA graph)
and batch1 (one grid per launch, L2 flushed, the paper's setting).

Under torchrun each rank transforms its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "128x32": (128, 32),
    "64x256": (64, 256),
    # smaller cases of the same kernels for ncu captures (inputs still > L2)
    "128x16": (128, 16),
    "64x64": (64, 64),
    "64x128": (64, 128),
    # the general path (edges without a fused kernel), for profiler captures
    "256x2": (256, 2),
    # the thread-pair kernel (96^3), for profiler captures
    "96x16": (96, 16),
}
METRIC = "batched 3D FFT transforms/s and % of HBM roofline at 64^3/128^3 (FP32 vs split-FP16)"
# The sources each default FP32 kernel is built from (its own file and the
# headers it includes); their hash keys the recorded DRAM traffic.
_COMMON_SOURCES = ["paper_2006_08435_gb300/csrc/persistent.cuh",
                   "paper_2006_08435_gb300/csrc/mbar.cuh",
                   "paper_2006_08435_gb300/csrc/rowfft.cuh",
                   "paper_2006_08435_gb300/csrc/codelets.cuh",
                   "paper_2006_08435_gb300/csrc/sizes.h"]
KERNEL_SOURCES = {128: ["paper_2006_08435_gb300/csrc/splity.cuh"] + _COMMON_SOURCES,
                  64: ["paper_2006_08435_gb300/csrc/rowfft2.cuh"] + _COMMON_SOURCES}
KERNEL_NAMES = {128: "splity_fft3d_kernel<128,-1>", 64: "rowfft2_fft3d_kernel<64,-1>",
                256: "axis_pass_kernel<-1,2> (general path, three passes)",
                96: "pairfft_fft3d_kernel<96,-1>"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device=None) -> float:
    """The largest of one per-rank duration over all ranks (an all-reduce
    MAX on the default process group); ws == 1 returns it unchanged."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: int, steps: int, ms: float) -> float:
    """Units per second over the whole job: every rank processes
    `units_per_rank` units per step, the job takes `ms` (max over ranks)."""
    return ws * units_per_rank * steps / (ms / 1e3)


def timed_ms(fn, steps: int, stream) -> float:
    """Mean milliseconds per call of `fn` over `steps` back-to-back calls,
    CUDA events on `stream` (the stream the library launches on), with a
    synchronize on both sides."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def batched_inputs(n: int, batch: int, seed: int, dev):
    """The bench's seeded Gaussian-sum batch: up to four generated grids,
    repeated, each copy times its own phase exp(0.37 i b), so every grid of
    the batch differs."""
    import torch
    from paper_2006_08435_gb300 import synth
    base = synth.gaussian_sum_grids(n, min(batch, 4), seed=seed)
    xb = torch.from_numpy(base).to(dev)
    reps = (batch + xb.shape[0] - 1) // xb.shape[0]
    x = xb.repeat(reps, 1, 1, 1)[:batch].contiguous()
    ph = torch.exp(1j * 0.37 * torch.arange(batch, device=dev, dtype=torch.float32))
    return (x * ph.view(-1, 1, 1, 1).to(torch.complex64)).contiguous()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(n: int) -> str:
    """Hash of the kernel's sources without // comments and blank lines (a
    change of the documentation alone keeps the recorded traffic)."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[n]:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(n: int, batch: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"fft3d_{n}cubed_dram_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash(n):
            return None
        per_grid = float(kv["dram_bytes_per_grid"])
        return per_grid * batch
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n: int, budget_s: float = 15.0):
    """The FP64 oracle, as it stands, on one n^3 grid of the workload,
    repeated until about `budget_s` seconds of CPU work."""
    import numpy as np
    from oracle import oracle
    from paper_2006_08435_gb300 import synth
    x = synth.gaussian_sum_grids(n, 1, seed=0).astype(np.complex128)
    oracle.dft3d(x[:, :8, :8, :8])         # load / build outside the timing
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.dft3d(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 100000:
            break
    return {"value": reps / el, "unit": "transforms/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{reps} forward transform(s) of one {n}^3 grid of the workload "
                      f"(FP64 separable direct DFT, {el:.1f} s)"}


def run_reference(args, ws, rank):
    n, batch = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle
    from paper_2006_08435_gb300 import synth
    x = synth.gaussian_sum_grids(n, 1, seed=0).astype(np.complex128)
    oracle.dft3d(x[:, :8, :8, :8])
    for _ in range(args.warmup):
        oracle.dft3d(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dft3d(x)
    el = time.perf_counter() - t0
    value = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fft3d_c2c_fwd_{n}cubed_batch{batch}", "n": n, "batch": batch,
                   "note": "each step is one grid of the batch (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"one {n}^3 grid per step, FP64 separable direct DFT"},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import torch
    from paper_2006_08435_gb300 import Plan, synth
    from paper_2006_08435_gb300 import build as B

    n, batch = WORKLOADS[args.workload]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.build()

    # seeded Gaussian-sum inputs; distinct grids from one generated grid set
    x = batched_inputs(n, batch, rank, dev)
    y = torch.empty_like(x)
    plan = Plan(n, n, n, batch)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        plan.execute(x, y, stream)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for i in range(args.steps):
        starts[i].record(stream)
        plan.execute(x, y, stream)
        ends[i].record(stream)
    t_all1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(t_all0.elapsed_time(t_all1), ws, dev)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(ws, batch, args.steps, total_ms)
    assert plan.device_status() == 0, "device-side wait timed out"

    # end to end through the public API with pinned host buffers
    e2e = None
    if args.no_e2e:
        hx = None
    else:
        # fft3d_execute_host: chunks copied in, transformed and copied out on
        # the plan's three streams, both copy directions overlapping
        hx = x.cpu().pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        plan.enable_host_io()
        e_steps = max(2, min(args.steps, 10))
        for _ in range(2):
            plan.execute_host(hx, hy, stream)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            plan.execute_host(hx, hy, stream)
        e1.record(stream)
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e_steps, ws, dev)
        e2e = {"value": whole_job_rate(ws, batch, 1, e2e_ms), "unit": "transforms/s",
               "h2d_bytes_per_step": hx.numel() * hx.element_size(),
               "d2h_bytes_per_step": hy.numel() * hy.element_size()}

    # the same workload through the split-FP16 tensor-core kind (the metric
    # compares FP32 with split FP16); timed like the FP32 steps, fewer of them
    split = None
    if not args.no_split:
        plan16 = Plan(n, n, n, batch, precision="split_fp16")
        for _ in range(3):
            plan16.execute(x, y, stream)
        barrier()
        k16 = max(1, args.steps // 4)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(k16):
            plan16.execute(x, y, stream)
        s1.record(stream)
        barrier()
        ms16 = max_over_ranks(s0.elapsed_time(s1) / k16, ws, dev)
        assert plan16.device_status() == 0
        split = {"value": whole_job_rate(ws, batch, 1, ms16), "unit": "transforms/s", "steps": k16,
                 "ms_per_step": ms16}

    # the other tensor-core operand kinds on the same batch (accuracy in the
    # error study of the GPU tests): throughput of each, timed like the
    # split leg
    kinds = None
    if not args.no_split:
        kinds = {}
        for kind in ("split_bf16", "fp16", "bfp16", "split_fp8", "fp8"):
            pk = Plan(n, n, n, batch, precision=kind)
            for _ in range(3):
                pk.execute(x, y, stream)
            barrier()
            kk = max(1, args.steps // 4)
            msk = max_over_ranks(timed_ms(lambda: pk.execute(x, y, stream), kk, stream), ws, dev)
            assert pk.device_status() == 0
            kinds[kind] = {"value": whole_job_rate(ws, batch, 1, msk), "ms_per_step": msk,
                           "steps": kk, "variant": pk.variant}
            del pk

    # real grids (the real parts of the same batch): forward R2C to half
    # spectra and inverse C2R back, each one kernel of the real-grid path
    # after a counter reset (128^3 FP32)
    real = real16 = None
    if not args.no_real:
        from paper_2006_08435_gb300 import RealPlan
        xr = x.real.contiguous()
        yr = torch.empty((batch, n, n, n // 2 + 1), dtype=torch.complex64, device=dev)
        br = torch.empty_like(xr)
        real = {}
        for name, rplan, src, dst in (("r2c", RealPlan(n, batch), xr, yr),
                                      ("c2r", RealPlan(n, batch, inverse=True), yr, br)):
            for _ in range(3):
                rplan.execute(src, dst, stream)
            barrier()
            kr = max(1, args.steps // 8)
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            for _ in range(kr):
                rplan.execute(src, dst, stream)
            r1.record(stream)
            barrier()
            msr = max_over_ranks(r0.elapsed_time(r1) / kr, ws, dev)
            assert rplan.device_status() == 0
            real[name] = {"value": whole_job_rate(ws, batch, 1, msr), "unit": "transforms/s",
                          "steps": kr, "ms_per_step": msr, "launches_per_step": 1,
                          "bytes_per_transform": 4 * n ** 3 + 8 * n * n * (n // 2 + 1)}
            del rplan
        del xr, yr, br
        # the paper's smallest edge as real grids: 16^3 x 16384 (268 MB of
        # reals in, 302 MB of half spectra out, larger than L2), one block
        # per grid
        n16, b16 = 16, 16384
        gen = torch.Generator(device=dev).manual_seed(16 + rank)
        x16 = torch.randn((b16, n16, n16, n16), generator=gen, device=dev, dtype=torch.float32)
        y16 = torch.empty((b16, n16, n16, n16 // 2 + 1), dtype=torch.complex64, device=dev)
        o16 = torch.empty_like(x16)
        real16 = {"workload": "real_16cubed_batch16384", "n": n16, "batch_per_gpu": b16,
                  "bytes_per_transform": 4 * n16 ** 3 + 8 * n16 * n16 * (n16 // 2 + 1)}
        for name, rplan, src, dst in (("r2c", RealPlan(n16, b16), x16, y16),
                                      ("c2r", RealPlan(n16, b16, inverse=True), y16, o16)):
            for _ in range(3):
                rplan.execute(src, dst, stream)
            barrier()
            kr = max(1, args.steps // 8)
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            for _ in range(kr):
                rplan.execute(src, dst, stream)
            r1.record(stream)
            barrier()
            msr = max_over_ranks(r0.elapsed_time(r1) / kr, ws, dev)
            assert rplan.device_status() == 0
            real16[name] = {"value": whole_job_rate(ws, b16, 1, msr), "unit": "transforms/s",
                            "steps": kr, "ms_per_step": msr, "launches_per_step": 1}
            del rplan
        del x16, y16, o16

    peak, peak_kind = measured_peaks()

    # the metric's other size: 64^3 x 256 grids (537 MB, larger than L2),
    # FP32 and split FP16, each through its default kernel, timed like the
    # split leg
    w64 = None
    if not args.no_64 and (n, batch) != (64, 256):
        del x, y
        n6, b6 = 64, 256
        x6 = batched_inputs(n6, b6, rank, dev)
        y6 = torch.empty_like(x6)
        w64 = {"workload": f"fft3d_c2c_fwd_{n6}cubed_batch{b6}", "n": n6, "batch_per_gpu": b6,
               "bytes_per_transform": 16 * n6 ** 3}
        for prec in ("fp32", "split_fp16"):
            p6 = Plan(n6, n6, n6, b6, precision=prec)
            for _ in range(3):
                p6.execute(x6, y6, stream)
            barrier()
            k6 = max(1, args.steps)
            ms6 = max_over_ranks(timed_ms(lambda: p6.execute(x6, y6, stream), k6, stream), ws, dev)
            assert p6.device_status() == 0
            w64[prec] = {"value": whole_job_rate(ws, b6, 1, ms6), "unit": "transforms/s",
                         "steps": k6, "ms_per_step": ms6, "variant": p6.variant,
                         "roofline_frac": 16.0 * n6 ** 3 * b6 / (ms6 / 1e3) / 1e9 / peak}
            del p6
        del x6, y6

    # the mixed-edge batch: 64 grids with edges drawn from {32, 48, 64, 80,
    # 96, 128}, forward then inverse captured in one CUDA graph and replayed
    # (a replay = 128 transforms; bytes = one read and one write of every
    # grid per direction)
    mixed = None
    if not args.no_mixed:
        import numpy as np
        from paper_2006_08435_gb300 import MixedPlan
        sizes = synth.mixed_sizes(64, seed=0)
        fwd, inv = MixedPlan(sizes), MixedPlan(sizes, inverse=True)
        packed = np.concatenate([g.ravel() for g in synth.mixed_grids(sizes, seed=1 + rank)])
        xm = torch.from_numpy(packed).to(dev)
        ym, bm = torch.empty_like(xm), torch.empty_like(xm)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            fwd.execute(xm, ym)
            inv.execute(ym, bm)
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            fwd.execute(xm, ym)
            inv.execute(ym, bm)
        for _ in range(3):
            graph.replay()
        barrier()
        km = max(1, args.steps)
        msm = max_over_ranks(timed_ms(graph.replay, km, stream), ws, dev)
        assert fwd.device_status() == 0 and inv.device_status() == 0
        pts = sum(e ** 3 for e in sizes)
        mixed = {"workload": "fft3d_c2c_mixed64_fwd_inv_graph", "edges": sorted(set(sizes)),
                 "grids": len(sizes), "points": pts, "variant_fwd": fwd.variant,
                 "value": whole_job_rate(ws, 2 * len(sizes), 1, msm), "unit": "transforms/s",
                 "steps": km, "ms_per_replay": msm, "l2": "inputs larger than L2 (no flush)",
                 "roofline_frac": 2 * 16.0 * pts / (msm / 1e3) / 1e9 / peak}
        del xm, ym, bm, graph, fwd, inv

    # the Hartree energy and its gradient on real densities (the
    # differentiation workload: 128^3, cell of 10 bohr, densities of 64
    # Gaussians): forward = real-grid transform + FP64 reduction over the
    # half spectrum, backward = seed on the half spectrum + real-grid
    # inverse; a batch of `batch` densities per step, and one density alone
    hartree = None
    if not args.no_hartree and n % 2 == 0:
        import numpy as np
        from paper_2006_08435_gb300 import hartree_energy
        rho1 = synth.hartree_density(n, seed=1 + rank)[0].astype(np.float32)
        hartree = {"cell_bohr": 10.0, "l2": "inputs larger than L2 (no flush)"}
        for hb in (batch, 1):
            rho = torch.from_numpy(rho1).to(dev).expand(hb, n, n, n).contiguous()
            rho = (rho * (1.0 + 0.01 * torch.arange(hb, device=dev).view(-1, 1, 1, 1))).contiguous()

            def step(rho=rho):
                r = rho.detach().requires_grad_(True)
                e = hartree_energy(r, 10.0)
                e.sum().backward()
                return r.grad

            with torch.cuda.stream(stream):
                for _ in range(3):
                    step()
            barrier()
            kh = max(2, args.steps // 4)
            with torch.cuda.stream(stream):  # the binding launches on the current stream
                msh = timed_ms(step, kh, stream)
            msh = max_over_ranks(msh, ws, dev)
            half = n * n * (n // 2 + 1) * 8
            # algorithmic bytes per density: R2C (4 n^3 + half), reduction
            # (half), seed (2 half), C2R (half + 4 n^3)
            hbytes = 8 * n ** 3 + 5 * half
            hartree[f"batch{hb}"] = {
                "value": whole_job_rate(ws, hb, 1, msh), "unit": "densities/s (energy + gradient)",
                "steps": kh, "ms_per_step": msh, "bytes_per_density": hbytes,
                "roofline_frac": hbytes * hb / (msh / 1e3) / 1e9 / peak}
            if hb == 1:
                # one density is bound by the host (autograd and the binding's
                # calls take longer than the GPU work): the same step captured
                # once in a CUDA graph (forward, energy, backward) and replayed
                # (captured on a side stream, whose plans and workspaces the
                # warm-up steps create: plans are kept per stream)
                gs = torch.cuda.Stream()
                gs.wait_stream(stream)
                with torch.cuda.stream(gs):
                    for _ in range(3):
                        step()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=gs):
                    step()
                with torch.cuda.stream(gs):  # replays launch on the current stream
                    for _ in range(3):
                        graph.replay()
                barrier()
                with torch.cuda.stream(gs):
                    msg = timed_ms(graph.replay, kh, gs)
                stream.wait_stream(gs)
                msg = max_over_ranks(msg, ws, dev)
                hartree["batch1_graph"] = {
                    "value": whole_job_rate(ws, 1, 1, msg), "unit": "densities/s (energy + gradient)",
                    "steps": kh, "ms_per_step": msg, "bytes_per_density": hbytes,
                    "roofline_frac": hbytes / (msg / 1e3) / 1e9 / peak}
                del graph
            del rho

    # the general path (any edge up to 512, non-cubic grids): 256^3 x 4 and
    # a non-cubic batch, one pencil pass per axis (three launches per chunk
    # of grids); roofline fractions of the 16 n^3 bytes and of the passes'
    # own traffic (three reads and writes of the grid, 48 n^3 bytes)
    general = None
    if not args.no_general:
        general = {}
        for shape, bg in (((256, 256, 256), 4), ((96, 128, 64), 64)):
            nz_, ny_, nx_ = shape
            xg = torch.randn((bg, nz_, ny_, nx_), dtype=torch.complex64, device=dev)
            yg = torch.empty_like(xg)
            pg = Plan(nx_, ny_, nz_, bg)
            for _ in range(3):
                pg.execute(xg, yg, stream)
            barrier()
            kg = max(1, args.steps // 4)
            msg = max_over_ranks(timed_ms(lambda: pg.execute(xg, yg, stream), kg, stream), ws, dev)
            assert pg.device_status() == 0
            pts_g = nx_ * ny_ * nz_ * bg
            general[f"{nz_}x{ny_}x{nx_}x{bg}"] = {
                "value": whole_job_rate(ws, bg, 1, msg), "unit": "transforms/s", "steps": kg,
                "ms_per_step": msg, "variant": pg.variant,
                "roofline_frac": 16.0 * pts_g / (msg / 1e3) / 1e9 / peak,
                "frac_of_pass_traffic": 48.0 * pts_g / (msg / 1e3) / 1e9 / peak}
            del xg, yg, pg

    # the paper's setting: one grid per transform (Table 1), latency of
    # one execute with L2 flushed before each timed launch
    batch1 = None
    if not args.no_batch1:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        batch1 = {"l2": "flushed (256 MB write) before each timed launch", "launches": 25,
                  "paper_context_us": {"fpga_kernel": {"16": 110, "32": 220, "64": 740},
                                       "fftw_40_cores": {"16": 10, "32": 30, "64": 140}}}
        for e in (16, 32, 64, 128):
            x1 = batched_inputs(e, 1, rank, dev)
            y1 = torch.empty_like(x1)
            p1 = Plan(e, e, e, 1)
            for _ in range(3):
                p1.execute(x1, y1, stream)
            us = []
            for i in range(25):
                flush.fill_(i & 255)
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                p1.execute(x1, y1, stream)
                a1.record(stream)
                a1.synchronize()
                us.append(1e3 * a0.elapsed_time(a1))
            assert p1.device_status() == 0
            us_med = max_over_ranks(statistics.median(us), ws, dev)
            batch1[str(e)] = {"us_median": us_med, "us_min": min(us), "variant": p1.variant,
                              "roofline_frac_median": 16.0 * e ** 3 / (us_med / 1e6) / 1e9 / peak}
        del flush

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    bytes_per_launch = 16.0 * n ** 3 * batch
    avg_launch_ms = statistics.mean(launch_ms)
    achieved = bytes_per_launch / (avg_launch_ms / 1e3) / 1e9
    traffic = recorded_traffic(n, batch)
    line = {
        "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": ws,
        "steps": args.steps, "warmup": warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian-sum complex64 grids)",
        "config": {"workload": f"fft3d_c2c_fwd_fp32_{n}cubed_batch{batch}", "n": n,
                   "batch_per_gpu": batch, "precision": "fp32", "direction": "forward",
                   "parallelism": f"replicas{ws}", "l2": "inputs larger than L2 (no flush)",
                   "gflops_nominal": value * 5 * n ** 3 * 3 * math.log2(n) / 1e9},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": KERNEL_NAMES.get(n, "fused_fft3d_kernel"),
                     "bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": avg_launch_ms,
                     "median_launch_ms": statistics.median(launch_ms),
                     "min_launch_ms": min(launch_ms)},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if split is not None:
        split["roofline_frac"] = 16.0 * n ** 3 * batch / (split["ms_per_step"] / 1e3) / 1e9 / peak
        line["split_fp16"] = split
    if kinds is not None:
        for v in kinds.values():
            v["roofline_frac"] = 16.0 * n ** 3 * batch / (v["ms_per_step"] / 1e3) / 1e9 / peak
        line["tensor_core_kinds"] = kinds
    if real is not None:
        for name, r in real.items():
            r["roofline_frac"] = (r["bytes_per_transform"] * batch / (r["ms_per_step"] / 1e3)
                                  / 1e9 / peak)
            line[f"real_{name}_fp32"] = r
    if real16 is not None:
        for name in ("r2c", "c2r"):
            r = real16[name]
            r["roofline_frac"] = (real16["bytes_per_transform"] * real16["batch_per_gpu"]
                                  / (r["ms_per_step"] / 1e3) / 1e9 / peak)
        line["real_16cubed_fp32"] = real16
    if w64 is not None:
        line["w64x256"] = w64
    if mixed is not None:
        line["mixed_c2"] = mixed
    if general is not None:
        line["general_path"] = general
    if hartree is not None:
        line["hartree"] = hartree
    if batch1 is not None:
        line["batch1"] = batch1
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="128x32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-real", action="store_true")
    ap.add_argument("--no-64", action="store_true", help="skip the 64^3 x 256 sub-leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-edge graph sub-leg")
    ap.add_argument("--no-batch1", action="store_true", help="skip the batch-1 latency sub-leg")
    ap.add_argument("--no-general", action="store_true", help="skip the general-path sub-leg")
    ap.add_argument("--no-hartree", action="store_true", help="skip the Hartree sub-leg")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
