#!/usr/bin/env python
"""Benchmark of the FHV hot path on GB300. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fhv|reference] [--workload ...]

Default (headline) line: the stress workload, the largest single-GPU
configuration: one step = three-axis fragment capture of 16.3M triangles,
POFA compaction at depth 11 (about 5e8 fragments, complete octree index) and
16 novel views at 3840x2160 in one batched call, with inputs resident in HBM.
Sub-lines `c2` (the 1M-triangle terrain step: PPFL, POFL, POFA, 3 views),
`batched` (many views of many scenes per call) and `learned` (splat +
gap-filler at 1080p, PSNR against direct capture) follow, each timed on its
own. --impl reference times the CPU oracle (single thread) on the same
workload (a bounded triangle sample per step for the stress workload); under
torchrun only rank 0 runs it. Multi-GPU runs are weak scaling: every rank
builds its own seeded scene of the same size, no data is exchanged.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FHV build Gfrag/s + novel-view frames/s (plain vs batched/learned @ stated PSNR)"
# DRAM bytes (read + write) per launch from ncu captures of the current kernels,
# keyed by (kernel, workload); None where no capture of the current code exists
TRAFFIC = {
    # leaf_scan at depth 9 (1.205 GB read + written per launch, ncu), scaled by
    # the 8x leaves of depth 10; the kernel is a pure stream over the leaves
    ("leaf_scan", "terrain1M_1080p_d10"): (39_897_344 + 1_165_176_064) * 8,
    # the leaf pass at depth 11, one full-size capture of the timed step (one ncu pass)
    ("leaf_scan", "stress16M_axis3_d11_4k"): 1_940_000_000 + 78_490_000_000,
    # the batched splat of the 16 4K views (views per item 16, 2048 records per
    # item, splat mode 4), one full-size capture of the timed step (one ncu pass)
    ("batch_splat", "stress16M_axis3_d11_4k", (16, 2048, 8192, 0, 4)): 8_361_361_408 + 246_524_416,
}
# L2 sectors per launch of that splat (ncu lts__t_sectors_op_read / _atom)
STRESS_SPLAT_L2 = {(16, 2048, 8192, 0, 4): (1_251_612_583, 296_404_069)}
HBM_FALLBACK_GBS = 6800.0
# L2 atomic sectors (ncu lts__t_sectors_op_red.sum) per launch: the splat of
# the terrain views (the same 1.53M POFA records at any octree depth; mean of
# the three views), and the atomic probe at 64 operations per thread.
SPLAT_RED_SECTORS = {"terrain1M_1080p": (1_265_748 + 1_233_993 + 1_200_480) / 3}
PROBE_RED_SECTORS_64 = (30_436_899 + 30_445_337) / 2


# ------------------------------------------------------------------ helpers

L2_BYTES = 129 * 10 ** 6  # GB300 L2 size


def host_cpu() -> dict:
    """The host the CPU baseline runs on: logical cores and CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    model = v.strip() if k.strip() == "model name" else f"{k.strip()} {v.strip()}"
                    if k.strip() == "model name":
                        break
    except OSError:
        pass
    import platform

    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model or platform.processor()}


# float32 operations the splat's projection takes per fragment and view
# (each rounded on its own: 3 subtractions for the offset, two dot products
# of 5 with a scale and an offset each, 2 floors for the pixel, a dot
# product, subtraction, scale and floor for the depth code), and per record
# per view group for its decoded position (3 x add, multiply, add).
SPLAT_OPS_PER_FRAGMENT_VIEW = 27
SPLAT_OPS_PER_RECORD = 9
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(max_mhz):
    """FP32 peak without FMA (one operation per lane per clock): SMs x 128
    lanes x the maximum SM clock (the NVML maximum sampled with the run,
    else 2070 MHz)."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP32_LANES_PER_SM * (max_mhz or 2070.0) * 1e6 / 1e12, sms


def peaks():
    """HBM copy bandwidth for the roofline: the measured figure if present, else the fallback, and which."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def workload(name: str, rank: int = 0, depth: int = None):
    """The named workload, seeded per rank (every rank of a weak-scaling run has its own scene)."""
    from paper_2211_15460_gb300 import scenes

    if name == "terrain":
        w = scenes.workload_terrain_1080p(seed=2 + 1000 * rank)
    elif name == "spheres":
        w = scenes.workload_spheres_256(seed=1 + 1000 * rank)
    else:
        raise ValueError(name)
    if depth is not None:
        w.depth = depth
        w.name = w.name.rsplit("_d", 1)[0] + f"_d{depth}"
    return w


class ClockSampler:
    """Samples SM clock, power and clock-event reasons through NVML (the
    driver's libnvidia-ml) in a background thread while active."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting", 0x1: "gpu_idle"}

    def __init__(self, cuda_index: int = 0, period_s: float = 0.005):
        self.period = period_s
        self.samples = []
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            bus = None
            try:
                import torch

                pr = torch.cuda.get_device_properties(cuda_index)
                bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            except Exception:
                bus = None
            rc = 1
            if bus is not None:
                rc = self.nvml.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.h))
            if rc != 0:
                rc = self.nvml.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(cuda_index), ctypes.byref(self.h))
            if rc != 0:
                return
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = int(mx.value)
            self.ok = True
        except OSError:
            self.ok = False

    def _sample(self):
        c, r, p = ctypes.c_uint(), ctypes.c_ulonglong(), ctypes.c_uint()
        if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) != 0:
            return
        fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.h, ctypes.byref(r))
        self.nvml.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(p))
        self.samples.append((int(c.value), int(r.value), int(p.value) / 1000.0))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self._sample()
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *exc):
        if self.ok:
            self._stop.set()
            self._t.join()
            self._sample()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "note": "NVML unavailable"}
        mhz = [s[0] for s in self.samples]
        bits = 0
        for s in self.samples:
            bits |= s[1]
        reasons = sorted({name for b, name in self.REASONS.items() if bits & b and b != 0x1})
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(self.samples), "power_w_max": max(s[2] for s in self.samples)}


def aggregate(frags_local: int, ms_local: float, dist):
    """(total fragments over ranks, max per-step time over ranks)."""
    if dist is None:
        return frags_local, ms_local
    import torch

    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    f = torch.tensor([float(frags_local)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return int(f.item()), float(t.item())


# -------------------------------------------------------- algorithmic bytes

def algorithmic_bytes(kernel: str, p) -> float:
    """Bytes the method must move per launch of `kernel` (averaged over the
    kernel's launches in one step where they differ)."""
    d = p.depth
    leaves = 8 ** d
    T = d - 4 if d > 4 else 0
    coarse_in_tile = sum(8 ** l for l in range(T + 1 if T > 0 else 0, d))  # levels the leaf pass writes
    n_pofl, n_ppfl = p.n_pofl, p.n_ppfl
    views = p.w.views
    if kernel == "leaf_scan":
        # occupancy bitmap in (1 bit), offset and count out (4 + 4 bytes) per
        # leaf, (off, cnt) of the coarse levels inside the tiles
        return leaves * (4 + 4 + 0.125) + coarse_in_tile * 8
    if kernel == "fill":
        # per step: tile-parent counters, one visibility buffer per view (list
        # heads are reset by the setup launch; headers and counters negligible)
        b = [(8 ** T) * 4] + [v.width * v.height * 8 for v in views]
        return sum(b) / len(b)
    if kernel == "bitmap_clear":
        return leaves / 8.0
    if kernel == "mark":
        return 8.0 * n_pofl
    if kernel == "raster":
        # per fragment a 16-byte record (+ the 4-byte parked pixel of PPFL); per
        # triangle 12 bytes of indices and 48 of vertex data (setup fused in)
        T = p.w.scene.n_tri
        return (20.0 * n_ppfl + 16.0 * n_pofl) / 2.0 + 60.0 * T
    if kernel == "link":
        return 12.0 * (n_ppfl + n_pofl) / 2.0  # 4-byte link + 8-byte head exchange
    if kernel == "count":
        return 16.0 * n_pofl
    if kernel == "scatter":
        return 32.0 * n_pofl
    if kernel == "seg_sort":
        return 32.0 * n_pofl
    if kernel == "splat":
        return 16.0 * n_pofl
    if kernel == "shade":
        return sum(v.width * v.height * (8 + 32 + 16) for v in views) / len(views)
    return 0.0


# ------------------------------------------------------------------- arms

def time_kernels(p, names, steps):
    """Average per-launch duration (ms) and launches per step of each kernel,
    from CUDA events recorded around its launches over `steps` steps."""
    import torch

    from paper_2211_15460_gb300 import fhv

    out = {}
    for name in names:
        n = 64 * steps
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        torch.cuda.synchronize()
        fhv.fhv_set_kernel_events(name, starts, stops)
        for _ in range(steps):
            p.step(concurrent=False)
        torch.cuda.synchronize()
        used = fhv.fhv_kernel_events_recorded()
        fhv.fhv_set_kernel_events(None, None, None)
        if used == 0:
            continue
        ms = [starts[i].elapsed_time(stops[i]) for i in range(used)]
        out[name] = {"avg_ms": sum(ms) / len(ms), "launches_per_step": used / steps, "ms_per_step": sum(ms) / steps}
    return out


def oracle_step(w):
    """One step of the workload by the oracle (PPFL, POFL, POFA, every view): (fragments, seconds)."""
    import oracle

    cap = w.capture.width * w.capture.height * 8
    t0 = time.perf_counter()
    n1 = oracle.ppfl(w.scene, w.capture, cap)[0]
    n2, _, _, rec, _ = oracle.pofl(w.scene, oracle.NORMAL, None, w.normal_pitch, w.depth, cap)
    pofa, off, cnt = oracle.pofa(rec[:n2], w.depth)
    for v in w.views:
        oracle.render(pofa, w.scene, v, w.lights, w.footprint_k)
    return n1 + n2, time.perf_counter() - t0


def atomic_peak(ops: int = 64, mode: int = 0, reps: int = 5):
    """Live L2 throughput from the library's probe on a 32 MB L2-resident
    buffer (mode 0: 64-bit atomicMin reductions, 1: returning atomics, 2:
    volatile reads): (ms per launch, operations per launch)."""
    import torch

    from paper_2211_15460_gb300 import fhv

    buf = torch.full((4 << 20,), -1, dtype=torch.int64, device="cuda")
    n = fhv.fhv_atomic_probe(buf, buf.numel(), ops, mode)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fhv.fhv_atomic_probe(buf, buf.numel(), ops, mode)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, n


def run_atomics(args, rank):
    """The L2 microbenchmark alone: reductions, returning atomics and volatile reads."""
    import torch

    from paper_2211_15460_gb300 import fhv

    if rank != 0:
        return None
    buf = torch.full((4 << 20,), -1, dtype=torch.int64, device="cuda")
    out = {}
    for ret in (0, 1, 2):
        for ops in (16, 64):
            n = fhv.fhv_atomic_probe(buf, buf.numel(), ops, ret)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(max(1, args.steps)):
                fhv.fhv_atomic_probe(buf, buf.numel(), ops, ret)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / max(1, args.steps)
            out[f"{('red', 'atom', 'read')[ret]}_ops{ops}"] = {"ms": ms, "ops": n, "g_ops_per_s": n / ms / 1e6}
    return {"metric": "L2 64-bit atomicMin throughput (microbenchmark)", "value": out["red_ops64"]["g_ops_per_s"],
            "unit": "G atomics/s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True,
            "config": {"workload": "atomic_probe_32MB"}, "runs": out, "device": torch.cuda.get_device_name()}


def run_reference(args, rank):
    """The reference arm: the oracle timed on the host cores, rank 0 only, on
    the workload of the fhv arm's line: for the default (stress) line each
    step is the bounded triangle sample of `stress_sample`, for the terrain
    line one full step."""
    if rank != 0:
        return None
    import oracle

    oracle.build()
    if args.workload == "headline":
        from paper_2211_15460_gb300 import scenes

        w = scenes.workload_stress()
        step = lambda i: stress_sample(w, offset=i)  # noqa: E731
        sample = STRESS_SAMPLE_NOTE
        config = {"workload": w.name, "n_tri": w.scene.n_tri, "capture": "three axes (3-Pass/1-Way)",
                  "capture_resolution": scenes.STRESS_RESOLUTION, "depth": w.depth, "views": len(w.views),
                  "view_size": "3840x2160", "lights": int(w.lights.shape[0])}
    else:
        w = workload(args.workload, 0, args.depth)
        step = lambda i: oracle_step(w)  # noqa: E731
        sample = ("the full workload, every step: PPFL capture, POFL build, POFA compaction, "
                  f"{len(w.views)} views (plain single-threaded C oracle)")
        config = None
    for i in range(args.warmup):
        step(i)
    frags, total = 0, 0.0
    for i in range(args.steps):
        f, t = step(args.warmup + i)
        frags += f
        total += t
    value = frags / total / 1e9
    if config is None:
        config = config_of(w, frags // args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gfrag/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64/f32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "Gfrag/s", "cores": 1, "host": host_cpu(),
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gfrag/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def config_of(w, frags_per_step):
    """The `config` object of the JSON line, with how the L2 is kept out of the timing."""
    dense = ((8 ** (w.depth + 1)) // 7 * 8 + (8 ** w.depth) // 7 * 4 + (8 ** w.depth) / 8) / 1e9
    if dense * 1e9 > L2_BYTES:
        l2 = ("inputs larger than L2: each step rewrites the dense depth-%d octree arrays (%.1f GB: offsets and "
              "counts of every octant, occupancy levels, leaf bitmap)" % (w.depth, dense))
    else:
        l2 = ("not flushed: the whole working set (dense depth-%d arrays %.4f GB, %d fragments) fits in L2, as it "
              "would in use" % (w.depth, dense, frags_per_step))
    return {"workload": w.name, "n_tri": w.scene.n_tri,
            "capture": f"{w.capture.width}x{w.capture.height}", "depth": w.depth, "views": len(w.views),
            "lights": int(w.lights.shape[0]), "footprint_k": w.footprint_k, "fragments_per_step": frags_per_step,
            "l2": l2}


def run_fhv(args, rank, world, dist):
    """The default benchmark: K timed steps of the plain path, roofline of the leaf pass, CPU baseline,
    end-to-end steps through the API with host copies, and clocks during the timed region."""
    import numpy as np
    import torch

    from paper_2211_15460_gb300 import fhv
    from paper_2211_15460_gb300.pipeline import PlainFHV

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    w = workload(args.workload, rank, args.depth)
    p = PlainFHV(w)
    frags = p.n_ppfl + p.n_pofl
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        p.step()
    torch.cuda.synchronize()

    # timed region: exactly K steps; the roofline kernel's launches are
    # bracketed by CUDA events on its own stream while they run
    roof_kernel = "leaf_scan"
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fhv.fhv_set_kernel_events(roof_kernel, k_start, k_stop)
    sampler = ClockSampler(local)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = fhv.fhv_launch_count()
    with sampler:
        start.record(stream)
        for _ in range(args.steps):
            p.step()
        stop.record(stream)
        torch.cuda.synchronize()
    launches = fhv.fhv_launch_count() - launches0
    if dist is not None:
        dist.barrier()
    k_used = fhv.fhv_kernel_events_recorded()
    fhv.fhv_set_kernel_events(None, None, None)
    roof_ms = [k_start[i].elapsed_time(k_stop[i]) for i in range(k_used)]
    ms = start.elapsed_time(stop) / args.steps
    total_frags, ms_max = aggregate(frags, ms, dist)
    value = total_frags / (ms_max * 1e-3) / 1e9
    if args.profile:  # only the timed steps (for profiler launch lists)
        return {"metric": METRIC, "value": value, "unit": "Gfrag/s", "ms_per_step": ms_max, "profile": True} \
            if rank == 0 else None

    # stage split (same step, separately timed)
    def timed(fn, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    k2 = max(3, min(args.steps, 50))
    def build_all():
        p.capture_ppfl()
        p.build()

    build_ms = timed(build_all, k2)
    render_ms = timed(p.render_all, k2)
    stage_ms = {"capture_ppfl": timed(p.capture_ppfl, k2), "build_pofl": timed(p.build_pofl, k2),
                "compact_pofa": timed(p.compact_pofa, k2), "render_view": render_ms / len(w.views)}

    # per-kernel durations (events around each launch) and the roofline
    names = ["fill", "reset", "raster", "big_scan", "raster_big", "link", "bitmap_clear", "mark", "count",
             "level_scan", "reduce_levels", "leaf_scan", "scatter", "seg_sort", "huge_sort", "splat", "shade"]
    kt = time_kernels(p, names, max(3, min(args.steps, 10)))  # sequential pass, one kernel name at a time
    dom = max(kt, key=lambda k: kt[k]["ms_per_step"])
    hbm, src = peaks()
    ab = algorithmic_bytes(roof_kernel, p)
    roof_avg = sum(roof_ms) / len(roof_ms)
    achieved = ab / (roof_avg * 1e-3) / 1e9
    roofline = {"kernel": roof_kernel, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": TRAFFIC.get((roof_kernel, w.name)), "peak_source": src,
                "algorithmic_bytes_per_launch": ab, "avg_launch_ms": roof_avg, "launches_timed": k_used,
                "dominant_kernel": dom}
    # the visibility pass against L2 atomic throughput: atomic sectors per
    # splat launch (ncu) over its live duration, against the library's probe
    atomics = None
    base = w.name.rsplit("_d", 1)[0]
    if base in SPLAT_RED_SECTORS and "splat" in kt:
        pms, pops = atomic_peak(64)
        peak_s = PROBE_RED_SECTORS_64 / (pms * 1e-3) / 1e9
        got_s = SPLAT_RED_SECTORS[base] / (kt["splat"]["avg_ms"] * 1e-3) / 1e9
        atomics = {"kernel": "splat", "achieved": got_s, "peak": peak_s, "unit": "G atomic sectors/s",
                   "frac": got_s / peak_s, "sectors_per_launch": SPLAT_RED_SECTORS[base],
                   "peak_probe": {"ms": pms, "ops": pops, "g_ops_per_s": pops / pms / 1e6}}

    # end to end through the public API: every step uploads the scene from pinned host memory and reads
    # the images and the fragment count back, beside the neighbouring steps' computation (StreamingSteps)
    from paper_2211_15460_gb300.pipeline import StreamingSteps

    ss = StreamingSteps(p)
    h2d, d2h = ss.h2d_bytes, ss.d2h_bytes
    for _ in range(2):
        ss.step()
    ss.finish()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ss.step()
    ss.finish()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps
    tf, e2e_max = aggregate(frags, e2e_ms, dist)
    e2e = {"value": tf / (e2e_max * 1e-3) / 1e9, "unit": "Gfrag/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max}

    # correctness of what was timed: counts unchanged, no device status bits
    st = [fhv.fhv_read_status(ws)[1] for ws in (p.ws_capture, p.ws_ppfl, p.ws_compact, *p.ws_views)]
    ok = fhv.fhv_get_count(p.ppfl)[1] == p.n_ppfl and fhv.fhv_get_count(p.pofl)[1] == p.n_pofl and not any(st)

    # the same steps with the sparse octree index in place of the complete one
    dense_pofa = p.pofa[: 2 * p.n_pofl].clone()
    p.use_sparse_index()
    for _ in range(2):
        p.step()
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler_sp = ClockSampler(local)
    with sampler_sp:
        sa.record(stream)
        for _ in range(args.steps):
            p.step()
        sb.record(stream)
        torch.cuda.synchronize()
    sp_ms = sa.elapsed_time(sb) / args.steps
    sp_cmp = timed(p.compact_pofa, k2)
    lb = p.level_base[: p.depth + 2].cpu().tolist()
    sparse = {"value": frags / (sp_ms * 1e-3) / 1e9, "unit": "Gfrag/s", "ms_per_step": sp_ms, "compact_ms": sp_cmp,
              "index_entries": lb[-1], "index_bytes": 16 * lb[-1],
              "records_equal_dense": bool(torch.equal(p.pofa[: 2 * p.n_pofl], dense_pofa)),
              "device_status": fhv.fhv_read_status(p.ws_sparse)[1], "clocks": sampler_sp.summary()}
    p.use_sparse_index(False)
    del dense_pofa

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cf, ct = oracle_step(w)
        cpu = {"kind": "oracle", "value": cf / ct / 1e9, "unit": "Gfrag/s", "cores": 1, "host": host_cpu(),
               "sample": "one full step of the same workload (PPFL + POFL + POFA + %d views), plain "
                         "single-threaded C oracle, %.1f s" % (len(w.views), ct)}

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": "Gfrag/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64/f32", "data": "synthetic", "config": config_of(w, frags),
        "novel_view_frames_per_s": 1000.0 / stage_ms["render_view"],
        "build_gfrag_s": frags / (build_ms * 1e-3) / 1e9,
        "stage_ms": stage_ms, "kernels": kt, "roofline": roofline, "atomics": atomics, "sparse": sparse,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches, "clocks": sampler.summary(),
        "fragments": {"ppfl": p.n_ppfl, "pofl": p.n_pofl}, "checks_ok": bool(ok),
        "device": torch.cuda.get_device_name(local),
    }
    return line


def run_batched(args, rank):
    """Many views of many scenes: fhv_render_views (one call, CUDA graph,
    autotuned decomposition) against one fhv_render_view call per view."""
    import numpy as np
    import torch

    from paper_2211_15460_gb300 import batched, fhv, scenes

    if rank != 0:
        return None
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws = batched.batched_workloads(n_scenes=args.batch_scenes, n_views=args.batch_views)
    t0 = time.perf_counter()
    sources = batched.build_sources(ws)
    build_s = time.perf_counter() - t0
    lights = np.stack([scenes.directional_light((1.0, 1.0, 1.0), (0.8, 0.8, 0.8)),
                       scenes.point_light((0.5, 1.5, 0.5), (0.3, 0.3, 0.3))])
    bv = batched.BatchedViews(sources, [w.views for w in ws], lights, 1)
    cfg, tune_ms, table = batched.autotune(bv, reps=2)
    bv.capture_graph()

    def timed(fn, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(k):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    k = max(1, min(args.steps, 10))
    plain_ms = timed(bv.render_one_by_one, k)
    ref = [(v.clone(), r.clone()) for v, r in zip(bv.vis, bv.rgba)]
    sampler = ClockSampler(0)
    with sampler:
        batch_ms = timed(bv.replay, k)
    same = all(torch.equal(v, rv) and bool(((r - rr).abs().max() < 1e-6).item())
               for v, r, (rv, rr) in zip(bv.vis, bv.rgba, ref))
    kt = {}
    for name in ("batch_clear", "batch_plan", "batch_splat", "batch_shade"):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        sp = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        fhv.fhv_set_kernel_events(name, st, sp)
        for _ in range(4):
            bv.render()
        torch.cuda.synchronize()
        u = fhv.fhv_kernel_events_recorded()
        fhv.fhv_set_kernel_events(None, None, None)
        kt[name] = sum(st[i].elapsed_time(sp[i]) for i in range(u)) / max(u, 1)
    frags = sum(s.n for s in sources)
    pixels = sum(c.width * c.height for c in bv.cams)
    hbm, src = peaks()
    covered = sum(int((v != -1).sum().item()) for v in bv.vis)
    shade_bytes = pixels * (8 + 16) + covered * 32  # vis in, rgba out; one 32-byte record sector per covered pixel
    clear_bytes = pixels * 8
    return {
        "metric": "novel-view frames/s, batched (many views x many scenes per call)", "value": bv.n_views / (batch_ms * 1e-3),
        "unit": "views/s", "n_gpus": 1, "steps": k, "warmup": args.warmup, "ms_per_step": batch_ms,
        "higher_is_better": True, "dtype": "i64/f32", "data": "synthetic",
        "config": {"workload": f"batched{len(ws)}x{args.batch_views}_1280x720", "scenes": len(ws),
                   "triangles": [w.scene.n_tri for w in ws], "depths": [w.depth for w in ws],
                   "views": bv.n_views, "fragments": frags, "view_pixels": pixels, "covered_pixels": covered},
        "plain_views_per_s": bv.n_views / (plain_ms * 1e-3), "plain_ms": plain_ms,
        "speedup_vs_plain": plain_ms / batch_ms, "identical_to_plain": bool(same),
        "tuned_config": {"views_per_item": cfg[0], "frags_per_item": cfg[1], "pixels_per_item": cfg[2],
                         "ctas_per_sm": cfg[3], "splat_mode": cfg[4] if len(cfg) > 4 else 0},
        "tuning_candidates": len(table),
        "kernels_ms": kt, "splats_per_s": frags * args.batch_views / (kt["batch_splat"] * 1e-3),
        "roofline_shade": {"bound": "hbm", "achieved": shade_bytes / (kt["batch_shade"] * 1e-3) / 1e9, "peak": hbm,
                           "unit": "GB/s", "frac": shade_bytes / (kt["batch_shade"] * 1e-3) / 1e9 / hbm,
                           "peak_source": src},
        "roofline_clear": {"achieved": clear_bytes / (kt["batch_clear"] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s"},
        "build_s": build_s, "clocks": sampler.summary(), "device": torch.cuda.get_device_name(),
    }


STRESS_SAMPLE_STRIDE = 1024  # the oracle's sample of the stress workload: every 1024th triangle


def stress_sample(w, offset: int = 0, stride: int = STRESS_SAMPLE_STRIDE, threads: int = 1):
    """One step of the stress workload by the oracle on a bounded sample:
    triangles offset, offset + stride, ... (about 16k of 16.3M), captured
    along the three axes, sorted into POFA order and splatted and shaded in
    all 16 novel views at 3840x2160. The dense depth-11 index (9.8e9
    octants) is left out: the host cannot hold it. threads > 1 runs the
    oracle's unchanged functions on that many host threads (capture by
    triangle ranges, one view per thread; identical results). Returns
    (fragments, seconds)."""
    import numpy as np

    import oracle
    from paper_2211_15460_gb300 import scenes

    sc = w.scene
    sel = np.arange(offset % stride, sc.n_tri, stride)
    sub = scenes.Scene(pos=sc.pos, nrm=sc.nrm, idx=sc.idx[sel], tri_material=sc.tri_material[sel], albedo=sc.albedo,
                       cube_min=sc.cube_min, cube_side=sc.cube_side)
    t0 = time.perf_counter()
    if threads > 1:
        from oracle import threads as othreads

        rec = othreads.fragments(sub, oracle.AXIS3, None, w.normal_pitch, threads)
        pofa = oracle.pofa_sort(rec)
        othreads.render_views(pofa, sub, w.views, w.lights, w.footprint_k, threads)
    else:
        rec, _, _ = oracle.fragments(sub, oracle.AXIS3, None, w.normal_pitch)
        pofa = oracle.pofa_sort(rec)
        for v in w.views:
            oracle.render(pofa, sub, v, w.lights, w.footprint_k)
    return int(rec.size), time.perf_counter() - t0


STRESS_SAMPLE_NOTE = ("every 1024th triangle of the stress scene (about 16k of 16.3M), one subset per step: three-axis "
                      "capture, POFA order, and all 16 novel views at 3840x2160 splatted and shaded, by the plain "
                      "single-threaded C oracle; the dense depth-11 octree index is not built (it does not fit the "
                      "host)")

# kernels of one headline step, in launch order
STRESS_KERNELS = ["fill", "raster", "big_scan", "raster_big", "bitmap_clear", "mark", "count", "level_scan",
                  "reduce_levels", "leaf_scan", "scatter", "seg_sort", "huge_sort", "batch_clear", "batch_plan",
                  "batch_splat", "batch_shade"]


def stress_algorithmic_bytes(kernel: str, p) -> float:
    """Bytes the method must move per launch of `kernel` in the headline step
    (per-unit figures in the design notes): the capture writes a 16-byte
    record per fragment and reads 12 bytes of indices and 48 bytes of vertex
    data per triangle; the compaction's passes move their records; the leaf
    pass writes (off, cnt) of every leaf and coarse octant of its tiles and
    reads the occupancy bitmap; the views read each record once per view
    group and write 8 + 16 bytes per pixel."""
    d, n, T = p.depth, p.n, p.w.scene.n_tri
    leaves = 8 ** d
    Tl = d - 4 if d > 4 else 0
    coarse_in_tile = sum(8 ** l for l in range(Tl + 1 if Tl > 0 else 0, d))
    pixels = sum(v.width * v.height for v in p.w.views)
    if kernel == "raster":
        return 16.0 * n + 60.0 * T
    if kernel == "leaf_scan":
        return leaves * (4 + 4 + 0.125) + coarse_in_tile * 8
    if kernel in ("scatter", "seg_sort"):
        return 32.0 * n
    if kernel == "count":
        return 16.0 * n
    if kernel == "mark":
        return 8.0 * n
    if kernel == "bitmap_clear":
        return leaves / 8.0
    if kernel == "batch_splat":
        return 16.0 * n * max(1, -(-len(p.w.views) // p.views.config_tuple[0])) + 8.0 * pixels
    if kernel == "batch_shade":
        return pixels * (8 + 16) + 32.0 * pixels
    return 0.0


SPARSE_KERNELS = ["fill", "bucket_count", "bucket_chunk", "bucket_chunk_scan", "bucket_offsets", "bucket_scatter", "tile_sort",
                  "bucket_sort", "huge_range_sort", "index_count", "index_scan", "index_write", "index_cnt"]


def run_sparse_steps(p, K, local):
    """The same steps with the sparse-index compaction in place of the dense
    one (capture, fhv_compact_pofa_sparse, the views): step time, the
    compaction's kernels, and its records checked equal to the dense
    compaction's on the device."""
    import torch

    from paper_2211_15460_gb300 import fhv

    p.alloc_sparse()
    stream = torch.cuda.current_stream()

    def step():
        p.capture()
        p.compact_sparse()
        p.render()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    kt = {}
    for name in SPARSE_KERNELS:
        st = [torch.cuda.Event(enable_timing=True) for _ in range(64)]
        sp = [torch.cuda.Event(enable_timing=True) for _ in range(64)]
        fhv.fhv_set_kernel_events(name, st, sp)
        p.compact_sparse()
        torch.cuda.synchronize()
        u = fhv.fhv_kernel_events_recorded()
        fhv.fhv_set_kernel_events(None, None, None)
        if u:
            kt[name] = sum(st[i].elapsed_time(sp[i]) for i in range(u))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(local)
    launches0 = fhv.fhv_launch_count()
    with sampler:
        for e in ev:
            e[0].record(stream)
            p.capture()
            e[1].record(stream)
            p.compact_sparse()
            e[2].record(stream)
            p.render()
            e[3].record(stream)
        torch.cuda.synchronize()
    launches = fhv.fhv_launch_count() - launches0
    ms = sum(e[0].elapsed_time(e[3]) for e in ev) / K
    cmp_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    p.compact()  # the dense compaction of the same records, for the byte comparison
    torch.cuda.synchronize()
    same = bool(torch.equal(p.sparse_pofa[: 2 * p.n], p.pofa[: 2 * p.n]))
    st = fhv.fhv_read_status(p.ws_sparse)[1]
    lb = p.level_base[: p.depth + 2].cpu().tolist()
    return {"value": p.n / (ms * 1e-3) / 1e9, "unit": "Gfrag/s", "ms_per_step": ms, "compact_ms": cmp_ms,
            "build_gfrag_s": p.n / ((ms - sum(e[2].elapsed_time(e[3]) for e in ev) / K) * 1e-3) / 1e9,
            "kernels_ms": kt, "index_entries": lb[-1],
            "occupied_octants_per_level": [lb[i + 1] - lb[i] for i in range(p.depth + 1)],
            "index_bytes": 16 * lb[-1], "records_equal_dense": same, "device_status": st, "gpu_launches": launches,
            "clocks": sampler.summary()}


def run_stress(args, rank, world=1, dist=None):
    """The headline: the stress workload (16.3M triangles captured along the
    three axes into one POFA at depth 11, about 5e8 fragments, then 16 novel
    views at 3840x2160 in one batched call). One step = fragment capture +
    POFA compaction (complete octree index) + the 16 views. Inputs resident
    in HBM, far larger than L2. Per-kernel times, the dominant kernel's
    roofline, the oracle on a bounded sample, end-to-end steps through the
    API with host copies, and clocks during the timed region.
    `--workload stress_small` runs the same step on the scaled-down stress
    scene (3.1M triangles, depth 9, 16 views at 1080p) for profiles."""
    import torch

    from paper_2211_15460_gb300 import fhv, scenes
    from paper_2211_15460_gb300.pipeline import PofaViews, StreamingPofaSteps

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    w = (scenes.workload_stress_small if args.workload == "stress_small" else scenes.workload_stress)(
        seed=5 + 1000 * rank)
    if args.capture_res:  # axis-capture resolution (pitch cube_side / res) instead of the workload's
        w.normal_pitch = float(w.scene.cube_side) / args.capture_res
        w.name = f"{w.name}_res{args.capture_res}"
    p = PofaViews(w)
    n = p.n
    stream = torch.cuda.current_stream()
    p.capture()
    p.compact()
    tuned = p.tune_views()
    for _ in range(args.warmup):
        p.step()
    torch.cuda.synchronize()

    # per-kernel durations: events around every launch of one kernel name per step
    kt = {}
    if not args.profile:
        for name in STRESS_KERNELS:
            st = [torch.cuda.Event(enable_timing=True) for _ in range(64)]
            sp = [torch.cuda.Event(enable_timing=True) for _ in range(64)]
            fhv.fhv_set_kernel_events(name, st, sp)
            p.step()
            torch.cuda.synchronize()
            u = fhv.fhv_kernel_events_recorded()
            fhv.fhv_set_kernel_events(None, None, None)
            if u:
                ms = [st[i].elapsed_time(sp[i]) for i in range(u)]
                kt[name] = {"avg_ms": sum(ms) / u, "launches_per_step": u, "ms_per_step": sum(ms)}
    dom = max(kt, key=lambda k: kt[k]["ms_per_step"]) if kt else "raster"

    # timed region: exactly K steps; the dominant kernel's launches bracketed by events on its stream
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    ks = [torch.cuda.Event(enable_timing=True) for _ in range(4 * K)]
    kp = [torch.cuda.Event(enable_timing=True) for _ in range(4 * K)]
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    fhv.fhv_set_kernel_events(dom, ks, kp)
    launches0 = fhv.fhv_launch_count()
    with sampler:
        for e in ev:
            e[0].record(stream)
            p.capture()
            e[1].record(stream)
            p.compact()
            e[2].record(stream)
            p.render()
            e[3].record(stream)
        torch.cuda.synchronize()
    launches = fhv.fhv_launch_count() - launches0
    k_used = fhv.fhv_kernel_events_recorded()
    fhv.fhv_set_kernel_events(None, None, None)
    if dist is not None:
        dist.barrier()
    cap_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    cmp_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    ren_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / K
    ms = sum(e[0].elapsed_time(e[3]) for e in ev) / K
    total_frags, ms_max = aggregate(n, ms, dist)
    value = total_frags / (ms_max * 1e-3) / 1e9
    if args.profile:
        return {"metric": METRIC, "value": value, "unit": "Gfrag/s", "ms_per_step": ms_max, "profile": True} \
            if rank == 0 else None
    dom_ms = [ks[i].elapsed_time(kp[i]) for i in range(k_used)]
    dom_avg = sum(dom_ms) / max(len(dom_ms), 1)
    hbm, src = peaks()
    ab = stress_algorithmic_bytes(dom, p)
    achieved = ab / (dom_avg * 1e-3) / 1e9 if dom_avg > 0 else 0.0
    cfg = tuple(p.views.config_tuple)
    traffic = TRAFFIC.get((dom, w.name, cfg)) if dom.startswith("batch") else TRAFFIC.get((dom, w.name))
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_source": src,
                "algorithmic_bytes_per_launch": ab, "avg_launch_ms": dom_avg, "launches_timed": k_used,
                "dominant_kernel": dom}
    roofline_hbm = None
    clk = sampler.summary()
    if dom == "batch_splat" and dom_avg > 0:
        # the splat is issue-bound on its arithmetic, not on memory: its roofline is the float32
        # work of the projection against the FP32 peak; the HBM figure is kept beside it
        n_views = len(w.views)
        groups = -(-n_views // p.views.config_tuple[0])
        ops = float(SPLAT_OPS_PER_FRAGMENT_VIEW) * n * n_views + float(SPLAT_OPS_PER_RECORD) * n * groups
        peak_t, sms = fp32_peak_tflops(clk.get("sm_max_mhz"))
        ach_t = ops / (dom_avg * 1e-3) / 1e12
        roofline_hbm = dict(roofline)
        roofline = {"kernel": dom, "bound": "alu", "achieved": ach_t, "peak": peak_t, "unit": "TFLOP/s",
                    "frac": ach_t / peak_t, "traffic": traffic,
                    "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                   f"{clk.get('sm_max_mhz') or 2070} MHz, one float32 operation per lane per clock",
                    "algorithmic_ops_per_launch": ops, "ops_per_fragment_view": SPLAT_OPS_PER_FRAGMENT_VIEW,
                    "avg_launch_ms": dom_avg, "launches_timed": k_used, "dominant_kernel": dom}
    # the splat against the L2's own ceilings: its read-first probes and record reads (L2 read sectors)
    # and its atomics per launch (ncu, this decomposition) over the event-timed launch, against the
    # library's L2 probe (volatile reads / reductions on an L2-resident buffer)
    l2 = None
    if cfg in STRESS_SPLAT_L2 and "batch_splat" in kt:
        rd, at = STRESS_SPLAT_L2[cfg]
        t_splat = kt["batch_splat"]["avg_ms"] * 1e-3
        prd_ms, prd_ops = atomic_peak(64, 2)
        pat_ms, pat_ops = atomic_peak(64, 1)
        l2 = {"kernel": "batch_splat", "unit": "G sectors/s",
              "read": {"achieved": rd / t_splat / 1e9, "peak": prd_ops / (prd_ms * 1e-3) / 1e9,
                       "frac": (rd / t_splat) / (prd_ops / (prd_ms * 1e-3)), "sectors_per_launch": rd},
              "atomic": {"achieved": at / t_splat / 1e9, "peak": pat_ops / (pat_ms * 1e-3) / 1e9,
                         "frac": (at / t_splat) / (pat_ops / (pat_ms * 1e-3)), "sectors_per_launch": at},
              "note": "peaks: one word per 32-byte sector per probe operation (returning atomics for the atomic peak)"}
    leaf = None
    if "leaf_scan" in kt:
        lb = stress_algorithmic_bytes("leaf_scan", p)
        la = lb / (kt["leaf_scan"]["avg_ms"] * 1e-3) / 1e9
        leaf = {"kernel": "leaf_scan", "bound": "hbm", "achieved": la, "peak": hbm, "unit": "GB/s", "frac": la / hbm,
                "traffic": TRAFFIC.get(("leaf_scan", w.name)), "algorithmic_bytes_per_launch": lb}
    status = [fhv.fhv_read_status(x)[1] for x in (p.ws_capture, p.ws_compact, p.views.ws)]
    ok = fhv.fhv_get_count(p.frags)[1] == n and not any(status)

    # end to end through the public API: scene arrays uploaded from pinned host memory and every image and the
    # fragment count read back every step, beside the neighbouring steps' computation
    ss = StreamingPofaSteps(p)
    h2d, d2h = ss.h2d_bytes, ss.d2h_bytes
    for _ in range(2):
        ss.step()
    ss.finish()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        ss.step()
    ss.finish()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / K
    tf, e2e_max = aggregate(n, e2e_ms, dist)
    e2e = {"value": tf / (e2e_max * 1e-3) / 1e9, "unit": "Gfrag/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max}
    del ss
    sparse = run_sparse_steps(p, K, local)
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        cf, ct = 0, 0.0
        for i in range(4):
            f, t = stress_sample(w, offset=i)
            cf, ct = cf + f, ct + t
        cpu = {"kind": "oracle", "value": cf / ct / 1e9, "unit": "Gfrag/s", "cores": 1, "host": host_cpu(),
               "sample": STRESS_SAMPLE_NOTE + "; 4 subsets, %d fragments, %.1f s" % (cf, ct)}
        from oracle import threads as othreads

        nt = othreads.default_threads()
        af, at = 0, 0.0
        for i in range(4, 12):
            f, t = stress_sample(w, offset=i, threads=nt)
            af, at = af + f, at + t
        cpu_all = {"kind": "oracle", "value": af / at / 1e9, "unit": "Gfrag/s", "cores": nt, "host": host_cpu(),
                   "sample": STRESS_SAMPLE_NOTE.replace("single-threaded", "unchanged") + "; its functions on %d "
                             "host threads (capture by triangle ranges, one view per thread); 8 subsets, %d "
                             "fragments, %.1f s" % (nt, af, at)}
    if rank != 0:
        return None
    leaves = 8 ** w.depth
    return {
        "metric": METRIC, "value": value, "unit": "Gfrag/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i64/f32", "data": "synthetic",
        "config": {"workload": w.name, "n_tri": w.scene.n_tri, "capture": "three axes (3-Pass/1-Way)",
                   "capture_resolution": scenes.STRESS_RESOLUTION, "depth": w.depth, "views": len(w.views),
                   "view_size": "3840x2160", "lights": int(w.lights.shape[0]), "fragments_per_step": n,
                   "l2": "inputs far larger than L2: %.1f GB of records, %.1f GB of octree index rewritten every step"
                         % (n * 16 / 1e9, (8 * leaves * 8 // 7) / 1e9)},
        "build_gfrag_s": n / ((cap_ms + cmp_ms) * 1e-3) / 1e9,
        "novel_view_frames_per_s": len(w.views) / (ren_ms * 1e-3),
        "stage_ms": {"capture": cap_ms, "compact_pofa": cmp_ms, "render_16_views": ren_ms},
        "views_config": dict(zip(("views_per_item", "frags_per_item", "pixels_per_item", "ctas_per_sm", "splat_mode"),
                                 p.views.config_tuple), candidates_ms=[[list(c), m] for c, m in tuned[2]]),
        "kernels": kt, "roofline": roofline, "roofline_hbm": roofline_hbm, "roofline_leaf_pass": leaf, "l2": l2,
        "sparse": sparse,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
        "gpu_launches": launches, "clocks": sampler.summary(), "checks_ok": bool(ok), "device_status": status,
        "device": torch.cuda.get_device_name(local),
    }


class ReadBack:
    """Results of repeated frames read back to pinned host memory on a copy
    stream beside the next frame's work: the device results alternate
    between two sets, and a set is written again only after its copy ended."""

    def __init__(self, like):
        import torch

        self.sets = [list(like), [torch.empty_like(t) for t in like]]
        self.host = [[torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in like] for _ in range(2)]
        self.copy = torch.cuda.Stream()
        self.copied = [None, None]
        self.k = 0

    @property
    def bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.host[0])

    def begin(self):
        """The device set this frame writes (the current stream waits until it is free)."""
        import torch

        s = self.k % 2
        if self.copied[s] is not None:
            torch.cuda.current_stream().wait_event(self.copied[s])
        return self.sets[s]

    def end(self):
        import torch

        s = self.k % 2
        done = torch.cuda.Event()
        done.record(torch.cuda.current_stream())
        self.copy.wait_event(done)
        with torch.cuda.stream(self.copy):
            for h, d in zip(self.host[s], self.sets[s]):
                h.copy_(d.view(-1), non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.copy)
        self.copied[s] = ev
        self.k += 1

    def finish(self):
        import torch

        torch.cuda.current_stream().wait_stream(self.copy)
        self.copy.synchronize()


def run_raycast(args, rank):
    """Ray casting through the POFA of the terrain workload (Section 3.3,
    Table 3): opaque (R), transparent exact (R/T, t_stop 0) and with the
    early-out (t_stop 0.01), beside the 1 x 1 splat of the same views. The
    FHV is built once (the paper's frames 1+); each timed frame is preceded by
    an L2 flush outside its events."""
    import numpy as np
    import torch

    from paper_2211_15460_gb300 import fhv
    from paper_2211_15460_gb300.pipeline import PlainFHV

    if rank != 0:
        return None
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = workload("terrain", 0, args.depth)
    p = PlainFHV(w)
    p.build()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    alpha_h = np.random.default_rng(11).uniform(0.3, 0.8, w.scene.albedo.shape[0]).astype(np.float32)
    alpha = torch.from_numpy(alpha_h).cuda()
    cams = w.views
    W, H = cams[0].width, cams[0].height
    vis = torch.empty(W * H, dtype=torch.int64, device="cuda")
    rgba = torch.empty(W * H * 4, dtype=torch.float32, device="cuda")
    ws = fhv.workspace(fhv.FHV_RAYCAST_WS_BYTES)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def cast(cam, al, t_stop, out=None):
        v_, r_ = (vis, rgba) if out is None else out
        fhv.fhv_raycast_pofa(p.pofa, n, p.off, p.cnt, w.depth, p.scene, p.scene.albedo, al, t_stop, p.lights,
                             p.n_lights, cam, v_, r_, ws)

    def splat(cam):
        fhv.fhv_render_view(p.pofa, n, None, p.scene, p.scene.albedo, p.lights, p.n_lights, cam, 1, vis, rgba, ws)

    modes = {"R": lambda c: cast(c, None, 0.0), "RT": lambda c: cast(c, alpha, 0.0),
             "RT_early": lambda c: cast(c, alpha, 0.01), "splat1": splat}
    k = max(1, args.steps)
    res, kern, each = {}, {}, {}
    sampler = ClockSampler(0)
    with sampler:
        for name, fn in modes.items():
            for _ in range(args.warmup):
                for c in cams:
                    fn(c)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k * len(cams))]
            kname = "splat" if name == "splat1" else "raycast"
            ks = [torch.cuda.Event(enable_timing=True) for _ in range(k * len(cams))]
            kp = [torch.cuda.Event(enable_timing=True) for _ in range(k * len(cams))]
            torch.cuda.synchronize()
            fhv.fhv_set_kernel_events(kname, ks, kp)
            i = 0
            for _ in range(k):
                for c in cams:
                    flush.fill_(i & 255)
                    ev[i][0].record(stream)
                    fn(c)
                    ev[i][1].record(stream)
                    i += 1
            torch.cuda.synchronize()
            used = fhv.fhv_kernel_events_recorded()
            fhv.fhv_set_kernel_events(None, None, None)
            res[name] = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
            kern[name] = sum(ks[j].elapsed_time(kp[j]) for j in range(used)) / max(used, 1)
            each[name] = [round(a.elapsed_time(b), 4) for a, b in ev]
    status = fhv.fhv_read_status(ws)[1]
    covered = int((vis != -1).sum().item())

    # end to end through the public API: the camera in (a by-value struct),
    # the image and visibility out to pinned host memory, every frame (read-back beside the next frame)
    rb = ReadBack([vis, rgba])

    def e2e_frame(c):
        cast(c, alpha, 0.0, rb.begin())
        rb.end()

    for c in cams:
        e2e_frame(c)
    rb.finish()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        for c in cams:
            e2e_frame(c)
    rb.finish()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / (k * len(cams))

    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        frag_o, _, _ = oracle.fragments(w.scene, oracle.NORMAL, None, w.normal_pitch)
        pofa_o = oracle.pofa_sort(frag_o)
        t0 = time.perf_counter()
        oracle.raycast(pofa_o, w.scene, cams[1], w.lights, alpha_h)
        ct = time.perf_counter() - t0
        cpu = {"kind": "oracle", "value": 1.0 / ct, "unit": "frames/s", "cores": 1, "host": host_cpu(),
               "sample": "one R/T frame of view 1 by the single-threaded brute-force oracle (%.2f s)" % ct}
    px = W * H
    return {
        "metric": "ray-cast novel view through the POFA, R/T (transparent, exact) frames/s", "value": 1000.0 / res["RT"],
        "unit": "frames/s", "n_gpus": 1, "steps": k, "warmup": args.warmup, "ms_per_step": res["RT"],
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{w.name}_raycast", "width": W, "height": H, "views": len(cams), "depth": w.depth,
                   "fragments": n, "l2": "flushed (256 MiB write) before every timed frame, outside its events"},
        "frame_ms": res, "kernel_ms": kern, "frame_ms_each": each, "rays_per_s_RT": px / (kern["RT"] * 1e-3),
        "rays_per_s_R": px / (kern["R"] * 1e-3), "covered_pixels_last_frame": covered,
        "e2e": {"value": 1000.0 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": rgba.numel() * 4 + vis.numel() * 8, "ms_per_step": e2e_ms,
                "note": "camera passed by value; R/T image and visibility copied to pinned host memory every frame, beside the next frame"},
        "cpu_baseline": cpu, "gpu_launches": 2 * k * len(cams), "device_status": status,
        "clocks": sampler.summary(), "device": torch.cuda.get_device_name(),
    }


def run_learned(args, rank):
    """Learned gap-filler (config 4): train on 20k 128x128 crops of
    (PPFL splat, direct capture) pairs from 8-sphere scenes at orbit offsets
    +-U[10, 60] degrees, then at 1920x1080 on held-out scenes compare plain
    1 x 1 splatting with splat + gap-filler: frames/s and PSNR against the
    direct capture of the same view."""
    import numpy as np
    import torch

    from paper_2211_15460_gb300 import fhv, gapfill, scenes

    if rank != 0:
        return None
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    feat, tgt = gapfill.make_dataset(args.crops, seed=1)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    net = gapfill.GapFiller(seed=0)
    t0 = time.perf_counter()
    hist = gapfill.train(net, feat, tgt, epochs=args.epochs, batch=64, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    steps = args.epochs * (feat.shape[0] // 64)
    # where a training step's time goes (events around every launch of the kind)
    split = {}
    bf, bt = feat[:64].contiguous(), tgt[:64].contiguous()
    for name, per in (("conv_fwd", 11), ("conv_wgrad", 6), ("gapfill_loss", 1)):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(3 * per)]
        sp = [torch.cuda.Event(enable_timing=True) for _ in range(3 * per)]
        fhv.fhv_set_kernel_events(name, st, sp)
        for _ in range(3):
            net.train_step(bf, bt, 64, 128, 128, 0.0)
        torch.cuda.synchronize()
        used = fhv.fhv_kernel_events_recorded()
        fhv.fhv_set_kernel_events(None, None, None)
        split[name] = sum(st[i].elapsed_time(sp[i]) for i in range(used)) / 3
    del feat, tgt, bf, bt
    torch.cuda.empty_cache()

    W, H = 1920, 1080
    P = W * H
    stream = torch.cuda.current_stream()
    vis = torch.empty(P, dtype=torch.int64, device="cuda")
    rgba = torch.empty(P * 4, dtype=torch.float32, device="cuda")
    fts = torch.empty(P * 8, dtype=torch.int16, device="cuda")
    img = torch.empty(P * 4, dtype=torch.float32, device="cuda")
    tgt_img = torch.empty(P * 4, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    lossd = torch.zeros(1, dtype=torch.float64, device="cuda")
    zero16 = torch.zeros(P * 16, dtype=torch.int16, device="cuda")
    evals = []
    plain_ms, learned_ms, conv_ms, flops = [], [], [], 0
    sampler = ClockSampler(0)
    with sampler:
        for si, seed in enumerate((901, 902)):
            sc = scenes.spheres_scene(seed)
            cap = scenes.orbit_camera(sc, W, H)
            pm = gapfill.PairMaker(sc, cap, 6, gapfill.spheres_light())
            p = pm.p
            for deg in (20.0, -35.0, 50.0):
                cam = scenes.orbit_camera(sc, W, H, orbit_deg=deg)
                pm.make(cam, fts, tgt_img, vis, rgba)  # target: direct capture of the view

                def plain():
                    fhv.fhv_render_view(p.ppfl.rec, p.ppfl.capacity, p.ppfl.count, p.scene, p.scene.albedo,
                                        pm.lights, p.n_lights, cam, 1, vis, rgba, ws)

                def learned(out=None):
                    plain()
                    fhv.fhv_splat_features(vis, rgba, p.ppfl.rec, cam, fts)
                    acts = net.forward(fts, 1, H, W)
                    fhv.fhv_gapfill_compose(acts[-1], fts, P, img if out is None else out)

                for fn, acc in ((plain, plain_ms), (learned, learned_ms)):
                    for _ in range(args.warmup):
                        fn()
                    for _ in range(args.steps):
                        flush.fill_(1)
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        fn()
                        b.record(stream)
                        torch.cuda.synchronize()
                        acc.append(a.elapsed_time(b))
                # convolution time inside the learned frame (events around each conv launch)
                st = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                sp = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                fhv.fhv_set_kernel_events("conv_fwd", st, sp)
                flush.fill_(2)
                learned()
                torch.cuda.synchronize()
                used = fhv.fhv_kernel_events_recorded()
                fhv.fhv_set_kernel_events(None, None, None)
                conv_ms.append(sum(st[i].elapsed_time(sp[i]) for i in range(used)))
                flops = sum(2 * 9 * ci * co for ci, co in gapfill.LAYERS) * P
                # PSNR of both images against the direct capture
                lossd.zero_()
                fhv.fhv_gapfill_loss(zero16, fts, tgt_img, P, 1.0, lossd, None)
                torch.cuda.synchronize()
                mse_plain = lossd.item() / (3 * P)
                lossd.zero_()
                acts = net.forward(fts, 1, H, W)
                fhv.fhv_gapfill_loss(acts[-1], fts, tgt_img, P, 1.0, lossd, None)
                torch.cuda.synchronize()
                mse_learned = lossd.item() / (3 * P)
                evals.append({"scene_seed": seed, "orbit_deg": deg, "psnr_plain_db": gapfill.psnr(mse_plain),
                              "psnr_learned_db": gapfill.psnr(mse_learned)})
    status = fhv.fhv_read_status(net.ws)[1]
    plain_avg = sum(plain_ms) / len(plain_ms)
    learned_avg = sum(learned_ms) / len(learned_ms)
    conv_avg = sum(conv_ms) / len(conv_ms)
    from statistics import mean

    hbm, src = peaks()
    bf16_peak, bf16_src = None, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak, bf16_src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        bf16_peak = 1900.0
    achieved = flops / (conv_avg * 1e-3) / 1e12
    # every layer reads its input and writes its output once (weights: a few KB);
    # at 58-145 FLOP per byte all six sit below the bf16/HBM balance point, so
    # the memory roof is the one that binds
    conv_bytes = sum((ci + co) * 2 for ci, co in gapfill.LAYERS) * P
    achieved_gbs = conv_bytes / (conv_avg * 1e-3) / 1e9
    # DRAM bytes read + written by the frame's six conv_fwd launches, one ncu capture (one pass) of
    # `python -m paper_2211_15460_gb300.gapfill --network --reps 2`
    conv_traffic = 721_863_424 + 430_181_888

    # end to end: the learned frame with the image read back to pinned host memory (beside the next frame)
    rb = ReadBack([img])
    for _ in range(2):
        learned(rb.begin()[0])
        rb.end()
    rb.finish()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        learned(rb.begin()[0])
        rb.end()
    rb.finish()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps

    cpu = None
    if not args.no_cpu_baseline:
        from oracle import gapfill as G

        x = G.from_bf16_bits(fts.view(H, W, 8)[:128, :256].cpu().numpy().view(np.uint16))[None]
        ws_ = [G.from_bf16_bits(t.cpu().numpy().view(np.uint16)).reshape(co, 3, 3, ci)
               for t, (ci, co) in zip(net.w16, gapfill.LAYERS)]
        bs_ = [t.cpu().numpy().astype(np.float64) for t in net.b32]
        t0 = time.perf_counter()
        a_ = x
        for li in range(6):
            a_ = G.conv3x3(a_, ws_[li], bs_[li], relu=li < 5)
        ct = time.perf_counter() - t0
        cpu = {"kind": "oracle", "value": (128 * 256) / ct / P, "unit": "frames/s", "cores": 1, "host": host_cpu(),
               "sample": "the network's forward pass (fp64 numpy oracle) on a 256x128 tile of a 1920x1080 frame, "
                         "%.2f s, scaled to a full frame" % ct}
    return {
        "metric": "novel-view frames/s at 1920x1080, plain 1x1 splat vs splat + learned gap-filler, @ PSNR against "
                  "direct capture", "value": 1000.0 / learned_avg, "unit": "frames/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": learned_avg, "higher_is_better": True,
        "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
        "config": {"workload": "gapfill_8spheres_1920x1080", "layers": gapfill.LAYERS, "train_crops": args.crops,
                   "crop": 128, "epochs": args.epochs, "eval_views": len(evals),
                   "l2": "flushed (256 MiB write) before every timed frame, outside its events"},
        "plain_frames_per_s": 1000.0 / plain_avg, "plain_ms": plain_avg, "learned_ms": learned_avg,
        "conv_ms_per_frame": conv_avg,
        "psnr_plain_db": mean(e["psnr_plain_db"] for e in evals),
        "psnr_learned_db": mean(e["psnr_learned_db"] for e in evals), "evals": evals,
        "train": {"crops": args.crops, "epochs": args.epochs, "steps": steps, "seconds": train_s,
                  "ms_per_step": train_s * 1000.0 / max(1, steps), "data_seconds": data_s,
                  "mse_per_epoch": hist, "kernel_ms_per_step": split},
        "roofline": {"kernel": "conv_fwd", "bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": achieved_gbs / hbm, "traffic": conv_traffic, "traffic_per": "frame (six launches)",
                     "peak_source": src,
                     "algorithmic_bytes_per_frame": conv_bytes,
                     "tensor": {"achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                                "frac": achieved / bf16_peak, "peak_source": bf16_src,
                                "algorithmic_flops_per_frame": flops}},
        "e2e": {"value": 1000.0 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": P * 16, "ms_per_step": e2e_ms},
        "cpu_baseline": cpu, "gpu_launches": (3 + 1 + 6 + 1) * args.steps, "device_status": status,
        "clocks": sampler.summary(), "device": torch.cuda.get_device_name(),
    }


def run_headline(args, rank, world, dist):
    """The default line: the stress workload (the largest single-GPU
    configuration) as `value`, with the terrain step (`c2`), the batched
    views (`batched`) and the learned gap-filler (`learned`) as sub-lines,
    each with its own timing and clocks. Sub-lines run on rank 0 after the
    headline's memory is released."""
    import copy

    import torch

    line = run_stress(args, rank, world, dist)
    if rank != 0 or args.profile:
        return line
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    sub = copy.copy(args)
    sub.steps = max(3, min(args.steps, 20))
    sub.workload = "terrain"
    line["c2"] = run_fhv(sub, 0, 1, None)
    torch.cuda.empty_cache()
    sub.steps = max(3, min(args.steps, 10))
    line["batched"] = run_batched(sub, 0)
    torch.cuda.empty_cache()
    sub.steps = max(3, min(args.steps, 10))
    line["learned"] = run_learned(sub, 0)
    return line


def main():
    """Parse the arguments, run the chosen arm and workload, print one JSON line on rank 0."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fhv", "reference"], default="fhv")
    ap.add_argument("--workload", choices=["headline", "terrain", "spheres", "batched", "raycast", "learned", "atomics",
                                           "stress", "stress_small"], default="headline")
    ap.add_argument("--crops", type=int, default=20000, help="learned: training crops")
    ap.add_argument("--epochs", type=int, default=4, help="learned: training epochs")
    ap.add_argument("--batch-scenes", type=int, default=16)
    ap.add_argument("--batch-views", type=int, default=64)
    ap.add_argument("--depth", type=int, default=None, help="override the workload's octree depth")
    ap.add_argument("--capture-res", type=int, default=None,
                    help="stress workloads: axis-capture resolution (pitch = cube side / res)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="run warm-up and timed steps only")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank)
    elif args.workload == "batched":
        line = run_batched(args, rank)
    elif args.workload == "raycast":
        line = run_raycast(args, rank)
    elif args.workload == "learned":
        line = run_learned(args, rank)
    elif args.workload == "atomics":
        line = run_atomics(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as tdist

            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            tdist.init_process_group("nccl")
            dist = tdist
        if args.workload in ("headline", "stress", "stress_small"):
            line = run_headline(args, rank, world, dist) if args.workload == "headline" else \
                run_stress(args, rank, world, dist)
        else:
            line = run_fhv(args, rank, world, dist)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
