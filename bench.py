#!/usr/bin/env python
"""Throughput benchmark of the Splotch frame render (particles/s per GB300).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one frame of the whole hot path -- rasterise, bin, tile pass, large
pass -- over the workload's particle set, which is resident in HBM before the
timed region starts.  `value` is particles rendered per second over all
ranks; `e2e` is the same metric through the C ABI with host buffers (particle
upload and image download inside the timed region).  Under torchrun every
rank renders its own copy of the workload (independent frames, weak scaling,
no collective on the data path); timing is the max over ranks.

`--impl reference` times the FP64 CPU oracle (the correctness reference) on
the host cores, each step a random sample of the same workload.
`--subsample M` renders a random M-particle subset of the workload (same camera
and image): a small case of the same kernels for profiler captures, labelled
as such in the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "clustered": {"scene": "clustered", "label": "clustered-10M-1024sq-f32",
                  "desc": "10M particles, 70% in 500 Plummer haloes + 30% uniform background, "
                          "density-derived h, FP32 attributes, 1024x1024 RGB FP32"},
    "precision": {"scene": "precision", "label": "clustered-100M-2048sq-f16attr", "fp16": "all",
                  "desc": "100M clustered particles, h/I/s stored FP16, 2048x2048 RGB FP32"},
    "precision-mixed": {"scene": "precision", "label": "clustered-100M-2048sq-f16IS", "fp16": "is",
                        "desc": "100M clustered particles, I/s stored FP16, h FP32, 2048x2048 RGB FP32"},
    "precision-logh": {"scene": "precision", "label": "clustered-100M-2048sq-logh16", "fp16": "logh",
                       "desc": "100M clustered particles, I/s stored FP16, h as a 16-bit logarithmic "
                               "code (1/4096 octave), 2048x2048 RGB FP32"},
    "precision32": {"scene": "precision", "label": "clustered-100M-2048sq-f32",
                    "desc": "100M clustered particles, FP32 attributes, 2048x2048 RGB FP32"},
    "precision32-support": {"scene": "precision", "label": "clustered-100M-2048sq-f32-support",
                            "params": {"sigma_per_h": 1.0 / 3.0},
                            "desc": "100M clustered particles, FP32 attributes, 2048x2048 RGB "
                                    "FP32, smoothing length read as the support radius "
                                    "(sigma = h / chi: 9x fewer covered pixels)"},
    "absorb": {"scene": "clustered", "label": "clustered-10M-1024sq-f32-absorb",
               "params": {"mode": 2, "absorption": 1.0},
               "desc": "the clustered 10M / 1024x1024 workload rendered with Eq. 1's general "
                       "absorption (grey absorption A = I, coloured emission): tile lists "
                       "radix-sorted by depth, front-to-back compositing"},
    "uniform": {"scene": "uniform", "label": "uniform-200k-256sq-f32",
                "desc": "200k uniform particles, log-normal h, 256x256 RGB FP32"},
    "pareto": {"scene": "pareto", "label": "pareto-400M-4096sq-f32", "sched": True,
               "desc": "400M clustered particles, heavy-tailed smoothing lengths (Pareto alpha 1.5), "
                       "4096x4096 RGB FP32, work items in tile order (the frame with items "
                       "ordered by the count heuristic and by the tile-cost network timed beside it)"},
    "stream": {"scene": "precision", "label": "stream-100M-2048sq-f32-chunks12.5M", "stream": 12_500_000,
               "desc": "100M clustered particles kept in page-locked host memory, FP32 attributes, "
                       "streamed through the GPU in 8 chunks of 12.5M (copy of chunk k+1 overlaps "
                       "the render of chunk k), 2048x2048 RGB FP32"},
    "orbit": {"scene": "orbit", "label": "orbit-20M-64views-512-2048", "batch": True,
              "desc": "20M clustered particles, 64 views on an azimuth orbit (5.625 deg steps), "
                      "resolutions cycling 512^2/1024^2/2048^2, one batched graph-replayed render"},
}
METRIC = "particles/s per GB300 at stated error vs FP64 oracle; % of HBM roofline"
E2E_STREAM_MIN = 16_000_000   # end-to-end through the out-of-core call from this size on
E2E_CHUNKS = 8
FLOPS_PER_PAIR = 7      # separable weight product (1 mul) + 3 multiply-adds
FLOPS_PER_POINT = 3     # 3 adds
# absorption: tau (2 mul), 1 - exp(-tau) (1 transcendental + 1), T (1 - e^-tau)
# (1 mul), 3 multiply-adds into C, the transmittance update (1)
FLOPS_PER_ABSORB = 11
FP32_LANES_PER_SM = 128


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the first query initialises NVML, which can hold driver calls for a
            # while: let it finish before the timed region begins
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# the source files a kernel is compiled from (its counters stay valid while
# these are unchanged)
KERNEL_SOURCES = {
    "item_kernel": ("spl_tile.cu", "spl_tile.cuh", "spl_geom.cuh", "spl_internal.cuh"),
    "absorb_kernel": ("spl_absorb.cu", "spl_tile.cuh", "spl_geom.cuh", "spl_internal.cuh"),
}


def _code_only(text: str) -> str:
    """Source text without comments and blank space: the code a kernel is
    compiled from (an edited comment leaves its counters valid)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_hash(files=None) -> str:
    """Hash of the kernel sources' code (the named files of csrc/, else all of them)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1309_1114_gb300", "csrc")
    names = sorted(files) if files else sorted(
        n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh")))
    for name in names:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_entry(kernel: str, label: str):
    """The committed ncu figures of this kernel on this workload
    (profiles/traffic.json), if its sources are unchanged since (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(f"{kernel}@{label}")
    if not e or e.get("source_hash") != source_hash(KERNEL_SOURCES.get(kernel.split("<")[0])):
        return None
    return e


def profiled_traffic(kernel: str, label: str):
    """DRAM bytes per launch from the committed ncu figures (else None)."""
    e = profiled_entry(kernel, label)
    return e.get("dram_bytes_per_launch") if e else None


def profiled_limiter(kernel: str, label: str):
    """The pipe that bounds the kernel in the committed ncu figures (else None)."""
    e = profiled_entry(kernel, label)
    return e.get("limiter") if e else None


def tile_kernel_name(tile_px: int, large: bool) -> str:
    """Name of the tile (or large) pass kernel that renders tiles of this side."""
    return f"item_kernel<{int(tile_px)}, {int(large)}>"


def oracle_par(wl: dict) -> dict:
    keys = ("mode", "absorption", "sigma_per_h")
    return {k: v for k, v in wl.get("params", {}).items() if k in keys}


# error bars per attribute layout: the FP32 path against the FP64 oracle, and
# the binary16 layouts against the oracle run on the original FP32 values
ERROR_TOL = {None: 1e-4, "is": 2e-3, "logh": 2e-3, "all": 4e-3}


def stated_error(scene, cam, g, par, tol, n_windows=1, n_bright=64, n_random=448):
    """Max relative pixel error of the timed frame g (H x W x 3, float64) against
    the FP64 oracle at >= 1024 sampled pixels: a whole 32 x 32 window over the
    seams of the four tiles nearest the brightest pixel (a halo core), the
    brightest pixels and random pixels, each computed one by one by the oracle
    from the original FP32 particles (mode 2 with its ambiguity mass)."""
    import oracle
    from tests._metrics import pick_pixels, rel_pixel_error
    px, py = pick_pixels(g, tile=32, n_windows=n_windows, n_bright=n_bright, n_random=n_random)
    t0 = time.perf_counter()
    mass = par.get("mode") == 2
    res = oracle.render_pixels(scene.parts, scene.palette, cam, par, px, py,
                               nthreads=os.cpu_count() or 1, with_mass=mass)
    o, B = res if mass else (res, None)
    M = np.abs(g).reshape(-1, 3).max(0)
    err = rel_pixel_error(g[py, px], o, B, M=M)
    return {"max_rel": err, "tol": tol, "n_pixels": int(px.size), "within_tol": bool(err <= tol),
            "vs": "FP64 oracle on the original FP32 particles",
            "picks": f"{n_windows} whole 32x32 tile-corner window(s) (first at the brightest pixel), "
                     f"{n_bright} brightest, {n_random} random",
            "metric": "max over pixels and channels of max(0, |g - o| - B) / max(|o|, 1e-3 max|o_c|)",
            "oracle_s": time.perf_counter() - t0}


def oracle_sample_rate(scene, cam, target_s: float, seed: int = 0, par=None, threads=None):
    """Time the FP64 oracle (all host cores unless threads is given; one for the
    depth-ordered absorption mode, which the oracle runs serially) on a random
    sample of the scene, sized to take about target_s seconds.  Returns
    (particles/s, sample, cores, secs)."""
    import oracle
    par = dict(par or {})
    cores = 1 if par.get("mode") == 2 else (threads or os.cpu_count() or 1)
    rng = np.random.default_rng(seed)
    m = min(scene.n, 20000)
    for _ in range(4):
        idx = np.sort(rng.choice(scene.n, m, replace=False))
        sub = {k: v[idx] for k, v in scene.parts.items()}
        t0 = time.perf_counter()
        oracle.render(sub, scene.palette, cam, par, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or m == scene.n:
            return m / dt, m, cores, dt
        m = int(min(scene.n, max(m * 2, m * target_s / max(dt, 1e-3))))
    return m / dt, m, cores, dt


def make_scene(wl: dict, subsample: int = 0):
    """The workload's scene; with subsample > 0 a random subset of that many
    of its particles (same camera and image: a small case of the same kernels
    for profiler captures, never a bench line of the workload itself)."""
    from paper_1309_1114_gb300 import scenes
    sc = scenes.make(wl["scene"])
    if subsample and subsample < sc.n:
        keep = np.sort(np.random.default_rng(0).choice(sc.n, subsample, replace=False))
        sc.parts = {k: v[keep] for k, v in sc.parts.items()}
        if sc.fp16 is not None:
            sc.fp16 = {k: v[keep] for k, v in sc.fp16.items()}
    return sc


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    scene = make_scene(wl)
    cam = scene.cams[0]
    # size one step to ~2 s of oracle work on all cores
    rate, m, cores, _ = oracle_sample_rate(scene, cam, 2.0, par=oracle_par(wl))
    import oracle
    rng = np.random.default_rng(1)
    times = []
    for k in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(scene.n, m, replace=False))
        sub = {kk: v[idx] for kk, v in scene.parts.items()}
        t0 = time.perf_counter()
        oracle.render(sub, scene.palette, cam, oracle_par(wl), nthreads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = m / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "description": wl["desc"],
                   "n_particles": scene.n, "image": [cam["width"], cam["height"]]},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{m} particles drawn at random per step from the "
                                   f"{scene.n}-particle workload, full {cam['width']}x"
                                   f"{cam['height']} image, FP64, OpenMP over {cores} threads"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, wl):
    """Batched multi-view workload: a step renders every view of the orbit."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1309_1114_gb300.splotch import Renderer

    scene = make_scene(wl)
    cams = scene.cams
    V = len(cams)
    stream = torch.cuda.current_stream()
    r = Renderer(local, stream.cuda_stream)
    r.load(scene.parts)
    r.set_colormap(scene.palette)
    r.set_params()
    imgs = [torch.empty((c["height"], c["width"], 3), device="cuda") for c in cams]
    tuned, tuned_ms = r.autotune(cams, imgs, reps=1)      # picks tile and class radii
    work = [0, 0, 0, 0]
    for c in cams:
        r.set_camera(c)
        work = [a + b for a, b in zip(work, r.count_work())]
    for _ in range(args.warmup):
        r.render_batch(cams, imgs)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.render_batch(cams, imgs)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    graph_kernels = int(r.stats()["launches"])      # kernel nodes of the replayed graph
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * V * scene.n / (ms * 1e-3)

    # stage times of the same batch rendered eagerly (graph replay times only the total)
    r.set_graph(False)
    r.set_timing(True)
    nst = max(2, min(args.steps, 5))
    for _ in range(nst):
        r.render_batch(cams, imgs)
    st = r.stats()
    r.set_timing(False)
    r.set_graph(True)
    nfr = max(st["timed_frames"], 1)
    stage = dict(zip(["raster", "bin", "tile", "large", "epilogue", "total"],
                     [v / nfr for v in st["sum_ms"]]))

    # the plain form: one spl_render per view with default parameters
    r.set_params()
    for c, im in zip(cams[:3], imgs[:3]):
        r.set_camera(c)
        r.render(im)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for c, im in zip(cams, imgs):
        r.set_camera(c)
        r.render(im)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    keep = {k: tuned[k] for k in ("tile_px", "r_small", "r_large")}
    r.set_params(**keep)

    # the same batch under each scheduler (graph replays, CUDA events): the
    # work items of all views taken in order, longest-first by the count
    # heuristic, and longest-first by the tile-cost network
    by_sched = None
    from paper_1309_1114_gb300 import scheduler, train_scheduler
    if os.path.exists(train_scheduler.DEFAULT_OUT):
        theta, heur = scheduler.load(train_scheduler.DEFAULT_OUT)
        r.set_model(theta, heur)
        by_sched = {}
        for name, mode in (("none", 0), ("count", 1), ("network", 2)):
            r.set_params(sched=mode, **keep)
            r.render_batch(cams, imgs)          # eager render + graph capture
            r.render_batch(cams, imgs)
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(3):
                r.render_batch(cams, imgs)
            q1.record(stream)
            torch.cuda.synchronize()
            by_sched[name] = q0.elapsed_time(q1) / 3
        r.set_params(**keep)

    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    dom = "tile" if stage["tile"] >= stage["large"] else "large"
    flops = (FLOPS_PER_POINT * work[0] + FLOPS_PER_PAIR * (work[1] + work[2]) if dom == "tile"
             else FLOPS_PER_PAIR * work[3])
    achieved = flops / (stage[dom] * 1e-3) / 1e12 if stage[dom] > 0 else 0.0
    kname = tile_kernel_name(tuned["tile_px"], dom != "tile")
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": profiled_traffic(kname, wl["label"]),
                "limiter": profiled_limiter(kname, wl["label"]),
                "kernel": kname, "kernel_ms": stage[dom],
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                              f"{sm_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
                "work": {"point_deposits": work[0], "small_pairs": work[1],
                         "medium_pairs": work[2], "large_pairs": work[3],
                         "flops_per_pair": FLOPS_PER_PAIR},
                "stage_basis": "eager batch with per-stage CUDA events"}
    pix = sum(c["width"] * c["height"] for c in cams)
    alg_bytes = scene.n * 24 + 12 * pix
    hbm = float(peaks.get("hbm_gbs", 6771.1))

    # end to end: upload the particles, render the batch, download every image
    host_parts = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
                  for k, v in scene.parts.items()}
    host_imgs = [torch.empty(tuple(im.shape), dtype=torch.float32).pin_memory() for im in imgs]
    e2e_steps = 3
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r.load(host_parts)
        r.render_batch(cams, imgs)
        for im, h in zip(imgs, host_imgs):
            h.copy_(im, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": ws * V * scene.n / e2e_s, "unit": "particles/s",
           "h2d_bytes_per_step": scene.n * 24, "d2h_bytes_per_step": 12 * pix,
           "ms_per_step": 1e3 * e2e_s}

    cpu = None
    error = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU leg: the oracle states the error of one 1024^2 view of the last
        # batch, then is timed
        r.render_batch(cams, imgs)
        torch.cuda.synchronize()
        error = stated_error(scene, cams[1], imgs[1].cpu().numpy().astype(np.float64), {},
                             ERROR_TOL[None], n_random=256)
        error["view"] = 1
        rate, m, cores, secs = oracle_sample_rate(scene, cams[1], 10.0)
        cpu = {"value": rate, "unit": "particles/s", "cores": cores, "kind": "oracle",
               "sample": f"{m} particles drawn at random from the workload, one 1024x1024 view of "
                         f"the orbit, FP64, OpenMP over {cores} threads, {secs:.1f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["label"], "description": wl["desc"],
                       "n_particles": scene.n, "n_views": V, "units": "particle-views",
                       "autotuned": {k: tuned[k] for k in ("tile_px", "r_small", "r_large")},
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (20M particles = 480 MB); no flush"},
            "plain_form": {"ms_per_step": plain_ms, "value": V * scene.n / (plain_ms * 1e-3),
                           "note": "one spl_render per view, default parameters"},
            "batch_ms_by_scheduler": by_sched,
            "roofline": roofline,
            "hbm_roofline_frac": alg_bytes / (ms * 1e-3) / (hbm * 1e9),
            "hbm_alg_bytes_per_step": alg_bytes,
            "stage_ms": stage,
            "e2e": e2e,
            "gpu_launches": graph_kernels * args.steps,
            "clocks": clocks,
            "error": error,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    r.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_ours(args, wl):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1309_1114_gb300.splotch import Renderer

    scene = make_scene(wl, args.subsample)
    cam = scene.cams[0]
    W, H = cam["width"], cam["height"]
    fp16 = None
    h_log2_min = None
    if wl.get("fp16") == "all":
        fp16 = scene.fp16
    elif wl.get("fp16") == "is":
        fp16 = {k: scene.fp16[k] for k in ("I", "s")}
    stream = torch.cuda.current_stream()
    r = Renderer(local, stream.cuda_stream)
    if wl.get("fp16") == "logh":
        # the library encodes the 18 B layout (I, s binary16, h a 16-bit log code)
        from paper_1309_1114_gb300 import splotch as _S
        h_log2_min = -14.0
        dev = {k: torch.from_numpy(scene.parts[k]).cuda() for k in ("h", "I", "s")}
        coded = r.encode_attrs(dev["h"], dev["I"], dev["s"], _S.SPL_ATTR_LOGH16, h_log2_min)
        torch.cuda.synchronize()
        fp16 = {"h": coded["h"].cpu().numpy().view(np.uint16), "I": coded["I"].cpu().numpy(),
                "s": coded["s"].cpu().numpy()}
        del dev, coded
    r.load(scene.parts, fp16, h_log2_min)
    r.set_colormap(scene.palette)
    r.set_camera(cam)
    r.set_params(**wl.get("params", {}))
    # the timed frame takes the work items in tile order (measured fastest);
    # with "sched" the frame under the count heuristic and the tile-cost
    # network is timed beside it
    sched_mode = 0
    model_info = None
    have_model = False
    if wl.get("sched"):
        from paper_1309_1114_gb300 import scheduler, train_scheduler
        if os.path.exists(train_scheduler.DEFAULT_OUT):
            theta, heur = scheduler.load(train_scheduler.DEFAULT_OUT)
            r.set_model(theta, heur)
            have_model = True
            with open(train_scheduler.DEFAULT_OUT) as fh:
                model_info = {k: v for k, v in json.load(fh).items() if k not in ("theta", "heur")}
    img = torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
    work = r.count_work()

    for _ in range(args.warmup):
        r.render(img)
    torch.cuda.synchronize()
    r.set_timing(True)
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.render(img)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = r.stats()
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * scene.n / (ms * 1e-3)

    # per-stage device times over the timed frames (CUDA events on the render stream)
    nfr = max(st["timed_frames"], 1)
    stage = dict(zip(["raster", "bin", "tile", "large", "epilogue", "total"],
                     [v / nfr for v in st["sum_ms"]]))
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12    # TFLOP/s
    absorbing = wl.get("params", {}).get("mode") == 2
    per_pair = FLOPS_PER_ABSORB if absorbing else FLOPS_PER_PAIR
    per_point = FLOPS_PER_ABSORB if absorbing else FLOPS_PER_POINT
    tile_flops = per_point * work[0] + per_pair * (work[1] + work[2])
    large_flops = per_pair * work[3]
    dom = "tile" if stage["tile"] >= stage["large"] else "large"
    flops = tile_flops if dom == "tile" else large_flops
    achieved = flops / (stage[dom] * 1e-3) / 1e12 if stage[dom] > 0 else 0.0
    kname = (f"absorb_kernel<{st['tile_px']}>" if absorbing else
             tile_kernel_name(st["tile_px"], dom != "tile"))
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": profiled_traffic(kname, wl["label"]),
                "limiter": profiled_limiter(kname, wl["label"]),
                "kernel": kname, "kernel_ms": stage[dom],
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                              f"{sm_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
                "work": {"point_deposits": work[0], "small_pairs": work[1],
                         "medium_pairs": work[2], "large_pairs": work[3],
                         "flops_per_pair": per_pair}}
    schedulers = None
    if wl.get("sched"):
        # the same frame with each scheduler (CUDA-event frame times, 5 frames each)
        schedulers = {}
        for name, mode in (("none", 0), ("count", 1), ("network", 2)):
            if mode == 2 and not have_model:
                continue
            r.set_params(sched=mode)
            r.render(img)
            r.set_timing(True)
            for _ in range(5):
                r.render(img)
            sst = r.stats()
            r.set_timing(False)
            schedulers[name] = sst["sum_ms"][5] / max(sst["timed_frames"], 1)
        r.set_params(sched=sched_mode, **wl.get("params", {}))
    bytes_per_particle = {None: 24, "all": 18, "is": 20, "logh": 18}[wl.get("fp16")]
    alg_bytes = scene.n * bytes_per_particle + 12 * W * H
    hbm = float(peaks.get("hbm_gbs", 6771.1))
    hbm_frac = alg_bytes / (ms * 1e-3) / (hbm * 1e9)

    # end to end through the C ABI with host buffers (upload + render + download)
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
           for k, v in (dict(scene.parts, **fp16) if fp16 is not None else scene.parts).items()}
    host_parts = {k: v.numpy() for k, v in pin.items()}
    host_img = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    r.set_timing(False)
    if ws > 1:
        torch.distributed.barrier()
    xyz = {k: host_parts[k] for k in ("x", "y", "z")}
    attrs = {k: host_parts[k] for k in ("h", "I", "s")}
    host_np = host_img.numpy()
    f32_parts = dict(xyz, **{k: attrs[k] for k in attrs if fp16 is None or k not in fp16})
    half_parts = None if fp16 is None else {k: attrs[k] for k in fp16}
    # large sets: the out-of-core call, whose chunk uploads overlap the render
    # of the previous chunk (the call a caller with host arrays makes); small
    # ones: upload, then render into host memory
    stream_chunk = -(-scene.n // E2E_CHUNKS) if scene.n >= E2E_STREAM_MIN else 0
    img_e2e = torch.empty_like(img) if stream_chunk else None

    def e2e_step():
        if stream_chunk:
            r.render_stream(f32_parts, stream_chunk, img_e2e, half_parts, h_log2_min=h_log2_min)
            host_img.copy_(img_e2e)
        else:
            r.load(f32_parts, half_parts, h_log2_min)
            r.render_host(host_np)

    e2e_step()                        # untimed: the chunk buffers are allocated once
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        t = torch.tensor([e2e_s], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": ws * scene.n / e2e_s, "unit": "particles/s",
           "h2d_bytes_per_step": scene.n * bytes_per_particle, "d2h_bytes_per_step": 12 * W * H,
           "ms_per_step": 1e3 * e2e_s,
           "api": (f"spl_render_stream from page-locked host arrays, {E2E_CHUNKS} chunks of "
                   f"{stream_chunk} particles, image read back" if stream_chunk else
                   "spl_load_particles from page-locked host arrays + spl_render_host")}
    del img_e2e

    cpu = None
    error = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU leg: the oracle states the timed frame's error, then is timed
        g = img.cpu().numpy().astype(np.float64)
        error = stated_error(scene, cam, g, dict(oracle_par(wl)), ERROR_TOL[wl.get("fp16")],
                             n_random=128 if scene.n > 200_000_000 else 448)
        del g
        rate, m, cores, secs = oracle_sample_rate(scene, cam, 10.0, par=oracle_par(wl))
        cpu = {"value": rate, "unit": "particles/s", "cores": cores, "kind": "oracle",
               "sample": f"{m} particles drawn at random from the workload, full {W}x{H} image, "
                         f"FP64, OpenMP over {cores} threads, {secs:.1f} s"}
        if cores > 1:
            r1, m1, _, s1 = oracle_sample_rate(scene, cam, 3.0, seed=1, par=oracle_par(wl),
                                               threads=1)
            cpu["single_thread"] = {"value": r1, "unit": "particles/s",
                                    "sample": f"{m1} particles at random, one thread, {s1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["label"], "description": wl["desc"],
                       "n_particles": scene.n, "image": [W, H],
                       "attributes": {None: "f32", "all": "h,I,s f16", "is": "I,s f16; h f32",
                                      "logh": "I,s f16; h 16-bit log code"}[wl.get("fp16")],
                       "tile_px": 32, "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (particles + per-frame records > 129 MB); no flush"},
            "roofline": roofline,
            "hbm_roofline_frac": hbm_frac,
            "hbm_alg_bytes_per_step": alg_bytes,
            "stage_ms": stage,
            "scheduler": {"mode": ["none", "count", "network"][sched_mode],
                          "frame_ms_by_scheduler": schedulers, "model": model_info}
            if wl.get("sched") else None,
            "stats": {k: st[k] for k in ("n_active", "n_point", "n_small", "n_medium", "n_large")}
            | {"n_entries": st["n_entries"], "n_tiles": st["n_tiles"]},
            "e2e": e2e,
            "gpu_launches": int(st["launches"]) * args.steps,
            "clocks": clocks,
            "error": error,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    r.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_stream(args, wl):
    """Out-of-core workload: a step streams the whole host-resident set through
    the GPU (spl_render_stream), so the host-to-device copy is inside every step."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1309_1114_gb300.splotch import Renderer

    scene = make_scene(wl)
    cam = scene.cams[0]
    W, H = cam["width"], cam["height"]
    stream = torch.cuda.current_stream()
    r = Renderer(local, stream.cuda_stream)
    r.set_colormap(scene.palette)
    r.set_camera(cam)
    r.set_params()
    # covered pairs of the whole set (diagnostic render of the loaded set), then
    # drop the device copy: the timed steps read host memory only
    r.load(scene.parts)
    work = r.count_work()
    r.load({k: v[:0] for k, v in scene.parts.items()})
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in scene.parts.items()}
    img = torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
    chunk = wl["stream"]
    for _ in range(args.warmup):
        r.render_stream(pin, chunk, img)
    torch.cuda.synchronize()
    r.set_timing(True)
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.render_stream(pin, chunk, img)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = r.stats()
    r.set_timing(False)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    n = int(pin["x"].shape[0])
    value = ws * n / (ms * 1e-3)
    nch = (n + chunk - 1) // chunk
    stage = dict(zip(["raster", "bin", "tile", "large", "epilogue", "total"],
                     [v / max(args.steps, 1) for v in st["sum_ms"]]))
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    dom = "tile" if stage["tile"] >= stage["large"] else "large"
    flops = (FLOPS_PER_POINT * work[0] + FLOPS_PER_PAIR * (work[1] + work[2])) if dom == "tile" \
        else FLOPS_PER_PAIR * work[3]
    achieved = flops / (stage[dom] * 1e-3) / 1e12 if stage[dom] > 0 else 0.0
    kname = tile_kernel_name(st["tile_px"], dom != "tile")
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": profiled_traffic(kname, wl["label"]),
                "limiter": profiled_limiter(kname, wl["label"]),
                "kernel": kname, "kernel_ms": stage[dom] / nch,
                "note": f"the dominant kernel runs once per chunk ({nch} per step); achieved = "
                        "algorithmic flops of the whole set / summed launch time",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                              f"{sm_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"}
    h2d = n * 24
    # end to end: the same call plus the image download into page-locked host memory
    host_img = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r.render_stream(pin, chunk, img)
        host_img.copy_(img, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": ws * n / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": 12 * W * H, "ms_per_step": 1e3 * e2e_s}
    error = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU leg: the oracle states the error of the streamed frame
        error = stated_error(scene, cam, host_img.numpy().astype(np.float64), {},
                             ERROR_TOL[None])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["label"], "description": wl["desc"], "n_particles": n,
                       "image": [W, H], "attributes": "f32", "chunk": chunk, "chunks": nch,
                       "tile_px": int(st["tile_px"]), "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (2.4 GB streamed per step); no flush"},
            "roofline": roofline,
            "h2d_gbs": h2d / (ms * 1e-3) / 1e9,
            "stage_ms": stage,
            "stats": {k: st[k] for k in ("n_active", "n_point", "n_small", "n_medium", "n_large")}
            | {"n_entries": st["n_entries"]},
            "e2e": e2e,
            "gpu_launches": int(st["launches"]) * nch * args.steps,
            "clocks": clocks,
            "error": error,
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    r.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="precision32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--subsample", type=int, default=0,
                    help="render a random subset of this many particles (profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    if args.subsample:
        if wl.get("batch") or wl.get("stream") or args.impl == "reference":
            ap.error("--subsample applies to single-frame workloads of this implementation")
        wl = dict(wl, label=f"{wl['label']}-subsample{args.subsample}")
    if args.impl == "reference":
        return run_reference(args, wl)
    if wl.get("batch"):
        return run_batch(args, wl)
    if wl.get("stream"):
        return run_stream(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
