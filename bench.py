"""Benchmark: rasterize throughput of the grouped FP16 tensor-core 3DGS path on GB300.

Workload (default): the 1.5M-Gaussian mixture scene (256 clusters, SH degree 3) rendered at
1600x1064 from 8 orbit cameras. One step = the whole hot path (preprocess, bin + sort,
rasterize) for all 8 cameras. `value` = megapixels per second over the timed steps with the scene
resident in HBM; `e2e` = the same metric with the scene copied host -> device and the 8 images
copied back every step, through the public API.

Also reported: p50/p99 frame latency, the FP32 CUDA-core rasterizer (1x1 tiles, the plain tile
rasterizer) on the same GPU, the per-stage split, the roofline of the dominant kernel (the
tensor-core rasterizer) and, on rank 0 at N=1, the FP64 CPU oracle on a bounded sample (which also
gives the PSNR of the sampled pixels against the oracle).

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (launched with torch.distributed.run): every rank renders the 8 cameras of its own copy
of the scene (independent frames, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rasterize Mpx/s & p99 frame ms, FP16-TC vs FP32-core, PSNR>=45dB vs oracle"
DTYPE = {"fp16_tc": "f16 products, f32 accumulate/blend", "bf16_tc": "bf16 products, f32 accumulate/blend",
         "fp32": "f32"}
UNIT = "Mpx/s"
SM_MAX_MHZ = 2070.0


def _unit_peaks(device: int):
    """Measured ex2 and FFMA rates of this GPU (the microbenchmark library) and its SM count."""
    import ctypes as C

    import torch
    from paper_2605_17855_gb300 import build as _b
    _b.build()
    lib = C.CDLL(_b.MICROBENCH_LIB)
    lib.tgs_microbench_peaks.restype = C.c_int
    lib.tgs_microbench_peaks.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    scratch = torch.empty(8 * sms * 512, dtype=torch.float32, device="cuda")
    ex2, ffma = C.c_double(0), C.c_double(0)
    torch.cuda.synchronize()
    if lib.tgs_microbench_peaks(C.c_void_p(scratch.data_ptr()), sms, C.byref(ex2), C.byref(ffma)) != 0:
        raise RuntimeError("microbenchmark failed")
    return {"sm_count": sms, "ex2_per_s": ex2.value, "ffma_per_s": ffma.value}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest of every rank's value (the time of the slowest replica); the value itself
    without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size: int, pixels_per_step_per_rank: int, ms_per_step: float) -> float:
    """Mpx/s of the whole job: every rank renders its own frames (weak scaling), the step time is
    the slowest rank's."""
    return world_size * pixels_per_step_per_rank / (ms_per_step * 1e-3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample of the same workload.

def cpu_baseline(scene, cam, tc_image=None, target_s=12.0, seed=0):
    """Oracle preprocess + bin sort of the whole frame, and the blend of a sample of tile groups
    (random groups, grown until about `target_s` of blending); frame time is extrapolated by pixel
    count. Returns (record, psnr_of_gpu_image_on_the_sample)."""
    import oracle
    t0 = time.perf_counter()
    pr = oracle.preprocess(scene, cam)
    t1 = time.perf_counter()
    bins = oracle.bin_sort(pr.mean2d, pr.radius, pr.depth, cam.width, cam.height, 2, 2, conic=pr.conic,
                           opacity=pr.opacity)
    t2 = time.perf_counter()
    TX, TY, GX, GY = oracle.group_grid(cam.width, cam.height, 2, 2)
    rng = np.random.default_rng(seed)
    order = rng.permutation(GX * GY)
    pix_done, blend_s, k = 0, 0.0, 0
    ref_list, pix_list = [], []
    batch = 8
    while k < len(order) and blend_s < target_s:
        gs = order[k: k + batch]
        k += len(gs)
        pix = []
        for g in gs:
            gx, gy = g % GX, g // GX
            xs = np.arange(gx * 32, min(gx * 32 + 32, cam.width))
            ys = np.arange(gy * 32, min(gy * 32 + 32, cam.height))
            X, Y = np.meshgrid(xs, ys)
            pix.append(np.stack([X.ravel(), Y.ravel()], 1))
        pix = np.concatenate(pix)
        tb = time.perf_counter()
        img = oracle.blend(cam.width, cam.height, pr.mean2d, pr.conic, pr.opacity, pr.rgb, bins, pixels=pix)
        blend_s += time.perf_counter() - tb
        pix_done += len(pix)
        ref_list.append(img.rgb)
        pix_list.append(pix)
        batch = min(batch * 2, 256)
    frame_s = (t1 - t0) + (t2 - t1) + blend_s * (cam.width * cam.height) / max(pix_done, 1)
    psnr = None
    if tc_image is not None:
        pix = np.concatenate(pix_list)
        ref = np.concatenate(ref_list)
        got = tc_image[:, pix[:, 1], pix[:, 0]].T
        import oracle as _o
        psnr = _o.psnr(got, ref)
    rec = {"value": round(cam.width * cam.height / frame_s / 1e6, 6), "unit": UNIT,
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": (f"1 frame of camera 0: full preprocess ({(t1 - t0):.2f}s) + bin sort ({(t2 - t1):.2f}s)"
                      f" of {scene.n} splats; blend of {k} random 2x2 tile groups ({pix_done} px, "
                      f"{blend_s:.2f}s) extrapolated to {cam.width}x{cam.height}")}
    return rec, psnr


# ------------------------------------------------------------------------------------------------

def _time_renderer(rend, ncams, steps, warmup):
    """Mean frame ms of a Renderer over `steps` passes of its cameras (CUDA events)."""
    import torch
    for _ in range(warmup):
        for i in range(ncams):
            rend.render(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        for i in range(ncams):
            rend.render(i)
    rend.join()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / (steps * ncams)


def run_dense4k(args):
    """6M Gaussians (64 tight clusters, 5% needles, SH degree 3) from 4 cameras at 3840x2160: every
    grouping (1x1, 2x2, 4x2, 2x4, 4x4) in FP16 and BF16 and the FP32 CUDA-core path, timed with the
    whole frame (preprocess, bin sort, rasterize) in CUDA graphs; the fastest grouping per precision
    is reported (the autotune), with a per-image error report of its camera-0 image against the
    oracle on sampled tile groups."""
    import torch
    import paper_2605_17855_gb300 as tgs
    from paper_2605_17855_gb300 import scenes
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    scene, cams = scenes.clusters_6m_3840x2160()
    H, W = cams[0].height, cams[0].width
    ds = tgs.DeviceScene.from_host(scene)
    steps = max(2, min(args.steps, 10))
    table = {}
    for prec in ("fp16_tc", "bf16_tc"):
        for tl in ((1, 1), (2, 2), (4, 2), (2, 4), (4, 4)):
            rend = tgs.Renderer(ds, cams, tl, prec)
            table[f"{prec}_{tl[0]}x{tl[1]}"] = round(_time_renderer(rend, len(cams), steps, 3), 4)
            if rend.overflowed():
                raise RuntimeError("bin capacity overflow")
            del rend
            torch.cuda.empty_cache()
    # the plain FP32 tile rasterizer (AABB-range lists), and FP32 on the membership lists
    rend = tgs.Renderer(ds, cams, (1, 1), "fp32", membership=False)
    table["fp32_1x1"] = round(_time_renderer(rend, len(cams), steps, 3), 4)
    del rend
    rend = tgs.Renderer(ds, cams, (1, 1), "fp32")
    table["fp32_1x1_membership"] = round(_time_renderer(rend, len(cams), steps, 3), 4)
    del rend
    best = {p: min((v, k) for k, v in table.items() if k.startswith(p)) for p in ("fp16_tc", "bf16_tc")}
    torch.cuda.empty_cache()
    errors = {}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        pix, ref = _oracle_sample(scene, cams[0], target_s=args.cpu_sample_s)
        for prec, (_, key) in best.items():
            tl = tuple(int(v) for v in key.split("_")[-1].split("x"))
            rgb, _, _, _, _ = tgs.render(ds, cams[0], tl, prec)
            torch.cuda.synchronize()
            got = rgb.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T
            errors[prec] = {"tiling": key.split("_")[-1], "pixels": int(len(pix)),
                            "psnr_db": round(oracle.psnr(got, ref), 2),
                            "max_abs": float(np.abs(got - ref).max())}
    px = len(cams) * W * H
    del ds
    torch.cuda.empty_cache()
    out = {"metric": "rasterize Mpx/s, grouping x precision autotune (6M Gaussians, 3840x2160)",
           "value": round(W * H / (best["fp16_tc"][0] * 1e-3) / 1e6, 2), "unit": "Mpx/s", "n_gpus": ws,
           "higher_is_better": True, "dtype": DTYPE["fp16_tc"], "data": "synthetic",
           "config": {"workload": "6M Gaussians, 64 clusters (std 0.15), 5% needles 100:1, SH degree 3; "
                                  "4 orbit cameras at 3840x2160", "steps": steps, "pixels_per_step": px},
           "frame_ms": table,
           "autotune": {p: {"tiling": k.split("_")[-1], "frame_ms": v} for p, (v, k) in best.items()},
           "speedup_vs_fp32_core": round(table["fp32_1x1"] / best["fp16_tc"][0], 3),
           "error_vs_oracle": errors}
    if getattr(args, "return_dict", False):
        return out
    if rank == 0:
        print(json.dumps(out))
    return 0


def run_backward(args):
    """Forward (FP32 rasterize with n_contrib) + backward of the blend for 500k Gaussians (the box
    generator) from 8 jittered cameras at 1024x1024, L = sum(image * G) with a fixed random G."""
    import torch
    import paper_2605_17855_gb300 as tgs
    from paper_2605_17855_gb300 import scenes
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    scene, cams = scenes.box_500k_1024_8cams()
    ds = tgs.DeviceScene.from_host(scene)
    frames = []
    for cam in cams:
        proj = tgs.preprocess(ds, cam)
        bins = tgs.bin_sort(proj, cam.width, cam.height, (2, 2))
        G = torch.randn((3, cam.height, cam.width), device="cuda")
        frames.append((cam, proj, bins, G))
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step():
        for cam, proj, bins, G in frames:
            rgb, T, nc = tgs.rasterize(proj, bins, cam.width, cam.height, "fp32")
            tgs.rasterize_backward(proj, bins, cam.width, cam.height, T, nc, G)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 20))
    a, b = ev(), ev()
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # backward alone
    cam, proj, bins, G = frames[0]
    rgb, T, nc = tgs.rasterize(proj, bins, cam.width, cam.height, "fp32")
    a.record()
    for _ in range(steps):
        tgs.rasterize_backward(proj, bins, cam.width, cam.height, T, nc, G)
    b.record()
    torch.cuda.synchronize()
    bwd_ms = a.elapsed_time(b) / steps
    px = sum(c.width * c.height for c in cams)
    out = {"metric": "forward+backward Mpx/s (500k Gaussians, 8 cameras at 1024x1024)",
           "value": round(px / (ms * 1e-3) / 1e6, 2), "unit": "Mpx/s", "n_gpus": ws, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "500k Gaussians (box generator, SH degree 0), 8 yaw-jittered cameras at "
                                  "1024x1024, 2x2 groups", "steps": steps},
           "ms_per_step": round(ms, 4), "backward_ms_per_frame": round(bwd_ms, 4)}
    del frames, ds
    torch.cuda.empty_cache()
    if getattr(args, "return_dict", False):
        return out
    if rank == 0:
        print(json.dumps(out))
    return 0


def _oracle_sample(scene, cam, target_s=10.0, seed=0):
    """The oracle's colours of random 2x2 tile groups of a frame (grown until about target_s of
    oracle blending): (pixels [P,2] as (x, y), rgb [P,3])."""
    import oracle
    pr = oracle.preprocess(scene, cam)
    bins = oracle.bin_sort(pr.mean2d, pr.radius, pr.depth, cam.width, cam.height, 2, 2, conic=pr.conic,
                           opacity=pr.opacity)
    TX, TY, GX, GY = oracle.group_grid(cam.width, cam.height, 2, 2)
    rng = np.random.default_rng(seed)
    order = rng.permutation(GX * GY)
    pix_list, ref_list = [], []
    k, spent, batch = 0, 0.0, 8
    while k < len(order) and spent < target_s:
        gs = order[k:k + batch]
        k += len(gs)
        pix = []
        for g in gs:
            gx, gy = g % GX, g // GX
            xs = np.arange(gx * 32, min(gx * 32 + 32, cam.width))
            ys = np.arange(gy * 32, min(gy * 32 + 32, cam.height))
            X, Y = np.meshgrid(xs, ys)
            pix.append(np.stack([X.ravel(), Y.ravel()], 1))
        pix = np.concatenate(pix)
        t = time.perf_counter()
        ref = oracle.blend(cam.width, cam.height, pr.mean2d, pr.conic, pr.opacity, pr.rgb, bins, pixels=pix)
        spent += time.perf_counter() - t
        pix_list.append(pix)
        ref_list.append(ref.rgb)
        batch = min(batch * 2, 256)
    return np.concatenate(pix_list), np.concatenate(ref_list)


def serve_sweep(rates, seconds, precision="fp16_tc", tiling=(2, 2), local=0, slots=8):
    """The rendering service on four resident scenes (200k / 800k / 1.5M / 3M Gaussians, SH degree 3)
    under a 120 GB budget: for each offered rate, open-loop Poisson arrivals for `seconds`, each
    request a random scene at a random resolution of 640x480, 1280x720, 1920x1080 and a 4096x2048
    stereo pair. Returns, per rate, completed frames/s and the per-resolution p50/p99 of
    submit-to-completion latency (measured by the server)."""
    import torch
    import paper_2605_17855_gb300 as tgs
    from paper_2605_17855_gb300 import scenes
    sc = scenes.resident_scenes_200k_800k_1p5m_3m()
    cams = [scenes.identity_camera(w, h) for (w, h) in scenes.SERVING_RESOLUTIONS]
    max_inflight = 64
    # output buffers: one per admitted request at most, per resolution
    pool = {k: [torch.empty((3, c.height, c.width), device="cuda") for _ in range(max_inflight)]
            for k, c in enumerate(cams)}
    rng = np.random.default_rng(0)
    results = {}
    for rate in rates:
        # a fresh server per rate keeps each rate's latency ring to its own requests
        srv = tgs.Server(120 << 30, max_inflight=max_inflight, slots=slots, device=local, precision=precision,
                         tiling=tiling, max_gaussians=max(s.n for s in sc), max_size=(4096, 2048),
                         max_entries=160 << 20)
        ids = [srv.add_scene(tgs.DeviceScene.from_host(s)) for s in sc]
        for sid in ids:  # warm-up: every scene at every resolution once
            for k, c in enumerate(cams):
                st = srv.wait(srv.submit(sid, c, pool[k][0]), 60000)
                if st != tgs.TGS_OK:
                    raise RuntimeError(f"serving warm-up failed with status {st}")
        base = srv.stats()
        free = {k: list(range(max_inflight)) for k in pool}
        n_arr = int(rng.poisson(rate * seconds))
        times = np.sort(rng.uniform(0.0, seconds, n_arr))
        picks = rng.integers(0, len(ids), n_arr), rng.integers(0, len(cams), n_arr)
        pending = []  # (ticket, resolution, buffer index)
        rejected_busy = rejected_nobuf = 0
        t0 = time.perf_counter()
        for j in range(n_arr):
            while True:
                now = time.perf_counter() - t0
                still = []
                for (t, k, b) in pending:  # reap finished requests to return their buffers
                    r = srv.poll(t)
                    if r is None:
                        still.append((t, k, b))
                    else:
                        free[k].append(b)
                pending = still
                if now >= times[j]:
                    break
                time.sleep(min(2e-4, times[j] - now))
            k = int(picks[1][j])
            if not free[k]:
                rejected_nobuf += 1
                continue
            b = free[k].pop()
            t = srv.try_submit(ids[int(picks[0][j])], cams[k], pool[k][b])
            if t is None:
                rejected_busy += 1
                free[k].append(b)
            else:
                pending.append((t, k, b))
        for (t, k, b) in pending:
            srv.wait(t, 60000)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
        done = st["completed"] - base["completed"]
        lat = {f"{r['width']}x{r['height']}": {"p50": round(r["p50_ms"], 3), "p99": round(r["p99_ms"], 3),
                                               "mean": round(r["mean_ms"], 3), "completed": int(r["completed"])}
               for r in st["resolutions"]}
        results[str(rate)] = {"offered": n_arr, "frames_per_s": round(done / elapsed, 2), "completed": int(done),
                              "failed": int(st["failed"] - base["failed"]), "rejected_busy": rejected_busy,
                              "rejected_no_buffer": rejected_nobuf, "latency_ms": lat}
        hbm = int(st["hbm_bytes"])
        srv.close()
    return results, hbm


def run_serve(args):
    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    tiling = tuple(int(v) for v in args.tiling.split("x"))
    rates = [float(r) for r in args.rates.split(",")] if args.rates else [args.rate]
    results, hbm = serve_sweep(rates, args.seconds, args.precision, tiling, local)
    best = max(v["frames_per_s"] for v in results.values())
    out = {"metric": "serve frames/s & p99 latency per resolution (4 resident scenes)",
           "value": best, "unit": "frames/s", "n_gpus": ws, "higher_is_better": True,
           "dtype": DTYPE[args.precision], "data": "synthetic",
           "config": {"workload": "4 resident scenes of 200k/800k/1.5M/3M Gaussians (SH degree 3), "
                                  "Poisson arrivals, resolutions 640x480/1280x720/1920x1080/4096x2048",
                      "seconds_per_rate": args.seconds, "tiling": args.tiling, "precision": args.precision,
                      "slots": 8, "max_inflight": 64, "hbm_budget_gb": 120,
                      "rasterization": "binned requests rasterized together by batched persistent launches"},
           "rates": results, "hbm_bytes": hbm,
           "note": "latency = submit to completion seen by the server's worker (warm-up excluded: a new "
                   "server per rate)"}
    if rank == 0:
        print(json.dumps(out))
    return 0


def run_reference(args):
    """The reference arm: the FP64 CPU oracle timed on the host cores (bounded sample per step)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2605_17855_gb300 import scenes
    scene, cams = scenes.mixture_1p5m_1600x1064()
    cam = cams[0]
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state
    vals, times = [], []
    for k in range(args.steps):
        t = time.perf_counter()
        rec, _ = cpu_baseline(scene, cam, target_s=args.ref_sample_s, seed=k)
        times.append(time.perf_counter() - t)
        vals.append(rec["value"])
    value = float(np.mean(vals))
    frame_ms = cam.width * cam.height / (value * 1e6) * 1e3
    # ms_per_step is what a step ran (one bounded sample of a frame: full preprocess and bin sort,
    # a sample of the blend); the rate is that sample's, extrapolated to the whole frame
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(times)), 3),
           "frame_ms_extrapolated": round(frame_ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _config(scene, cams, args),
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": rec["cores"], "kind": "oracle",
                            "sample": rec["sample"]},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of camera 0 of
# the 1.5M-Gaussian workload, keyed by the kernel and the SHA-1 of the sources it is built from;
# reported only while those sources are unchanged (the profile summary gives the command).
TRAFFIC = {("k_raster_tc", "2x2"): {"bytes": 67730944,
                                   "sha1": "855099e9d3b785864c0687b71b1bc7d5c4c17b93"}}
# Pipe utilizations of the dominant kernel from the same kind of capture (ncu --set full), keyed by
# the kernel; reported only while its sources hash to the recorded value.
NCU_FRACTIONS = {"k_raster_tc": {"sha1": "855099e9d3b785864c0687b71b1bc7d5c4c17b93",
                                  "tensor_pipe_pct": 3.1, "xu_mufu_pct": 11.1, "issue_active_pct": 69.9,
                                  "alu_pipe_pct": 47.6, "fma_pipe_pct": 23.7, "warps_active_pct": 60.1,
                                  "warp_instructions": 214615715}}


def _kernel_sources_sha1(kernel):
    files = {"k_raster_tc": ["raster_tc_impl.cuh", "tgs_internal.cuh"],
             "k_raster_fp32": ["raster_fp32.cu", "tgs_internal.cuh"]}[kernel]
    h = hashlib.sha1()
    for f in files:  # code only: comments and blank lines do not change the kernel
        with open(os.path.join(ROOT, "paper_2605_17855_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in src.splitlines():
            line = line.split("//", 1)[0].rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()


def _traffic(kernel, args):
    rec = TRAFFIC.get((kernel, args.tiling))
    if rec is None or rec["sha1"] != _kernel_sources_sha1(kernel):
        return None
    return rec["bytes"]


def _config(scene, cams, args):
    return {"workload": f"mixture scene, {scene.n} Gaussians (256 clusters, SH degree 3), "
                        f"{len(cams)} orbit cameras at {cams[0].width}x{cams[0].height}",
            "splats": scene.n, "cameras": len(cams), "width": cams[0].width, "height": cams[0].height,
            "tiling": args.tiling, "precision": args.precision,
            "l2": "inputs larger than L2 (scene %.0f MB read every frame)" % (scene.nbytes / 1e6)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tgs", choices=["tgs", "reference"])
    ap.add_argument("--precision", default="fp16_tc", choices=["fp16_tc", "bf16_tc", "fp32"])
    ap.add_argument("--tiling", default="2x2")
    ap.add_argument("--splats", type=int, default=1_500_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the 4K autotune, backward and serving workloads appended to the headline line")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--ref-sample-s", type=float, default=8.0)
    ap.add_argument("--workload", default="frames", choices=["frames", "dense4k", "backward"],
                    help="frames: the headline frame benchmark; dense4k: 6M Gaussians at 3840x2160, grouping "
                         "and precision autotune with a per-image error report; backward: forward + "
                         "backward, 500k Gaussians at 1024x1024")
    ap.add_argument("--serve", action="store_true",
                    help="benchmark the rendering service on four resident scenes instead")
    ap.add_argument("--rate", type=float, default=1000.0, help="--serve: offered requests per second")
    ap.add_argument("--rates", default="200,300,500,1000,2000",
                    help="--serve: comma-separated offered rates to sweep (overrides --rate)")
    ap.add_argument("--seconds", type=float, default=5.0, help="--serve: length of the arrival process")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.serve:
        return run_serve(args)
    if args.workload == "dense4k" and args.impl != "reference":
        return run_dense4k(args)
    if args.workload == "backward" and args.impl != "reference":
        return run_backward(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_2605_17855_gb300 as tgs
    from paper_2605_17855_gb300 import scenes

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tiling = tuple(int(v) for v in args.tiling.split("x"))

    scene, cams = scenes.mixture_1p5m_1600x1064(n=args.splats)
    H, W = cams[0].height, cams[0].width
    ds = tgs.DeviceScene.from_host(scene)
    stream = torch.cuda.current_stream()
    ncam = len(cams)
    px_per_step = ncam * W * H
    tc = args.precision != "fp32"
    # The renderers: one pair of CUDA graphs per camera (preprocess + bin sort, rasterize), a frame
    # is two launches. Pipelined (the next frame's preprocess + bin sort overlaps the previous
    # frame's rasterize) for frame rates, unpipelined for the per-stage times and the rasterize
    # kernel's own launch time. The plain FP32 CUDA-core rasterizer uses the original tile
    # organization: 1x1 tiles and every tile of each Gaussian's AABB range.
    R = {}

    def make(key, tl, prec, membership=True, cull=True):
        R[key] = (tgs.Renderer(ds, cams, tl, prec, membership=membership, cull=cull),
                  tgs.Renderer(ds, cams, tl, prec, membership=membership, cull=cull, pipeline=False))

    make("main", tiling, args.precision)
    make("fp32_plain", (1, 1), "fp32", membership=False)
    make("fp32_membership", (1, 1), "fp32")
    if tc:
        make("tc_range_skip", tiling, args.precision, membership=False)
        make("tc_range_noskip", tiling, args.precision, membership=False, cull=False)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(r, steps, warmup):
        for _ in range(warmup):
            for i in range(ncam):
                r.render(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [[(ev(), ev(), ev()) for _ in cams] for _ in range(steps)]
        t0, t1 = ev(), ev()
        t0.record(stream)
        torch.cuda.nvtx.range_push(f"timed_{r.precision}_{r.tiling[0]}x{r.tiling[1]}" + ("" if r.cull else "_noskip")
                                   + ("" if r.membership else "_range"))
        for k in range(steps):
            for i in range(ncam):
                r.render(i, evs[k][i])
        r.join()
        torch.cuda.nvtx.range_pop()
        t1.record(stream)
        torch.cuda.synchronize()
        total_ms = max_over_ranks(t0.elapsed_time(t1), dist, "cuda")
        if dist:
            dist.barrier()
        # frame time = interval between consecutive frame completions (what a viewer of the
        # frame sequence sees); latency = from a frame's first kernel to its last
        ends = [c for row in evs for _, _, c in row]
        frames = np.array([t0.elapsed_time(ends[0])] +
                          [ends[q - 1].elapsed_time(ends[q]) for q in range(1, len(ends))])
        timed.latency = np.array([a.elapsed_time(c) for row in evs for a, _, c in row])
        prep = np.array([a.elapsed_time(m) for row in evs for a, m, _ in row])
        raster = np.array([m.elapsed_time(c) for row in evs for _, m, c in row])
        return total_ms, frames, prep, raster

    # clocks are sampled over every timed phase (the headline loop alone is a fraction of a second)
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, frames_ms, _, _ = timed(R["main"][0], args.steps, args.warmup)
    latency_ms = timed.latency
    launches = int(args.steps * sum(R["main"][0].kernels_per_frame))
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(ws, px_per_step, ms_per_step)
    steps2 = max(3, args.steps // 2)
    paths = {}
    for key, (rp, rs) in R.items():
        totp, framesp, _, _ = timed(rp, steps2, 3)
        tots, _, prep, raster = timed(rs, steps2, 3)
        if rp.overflowed() or rs.overflowed():
            raise RuntimeError("bin capacity overflow during the benchmark")
        paths[key] = {"value": round(whole_job_rate(ws, px_per_step, totp / steps2), 3), "unit": UNIT,
                      "frame_ms_p99": round(float(np.percentile(framesp, 99)), 4),
                      "value_without_pipeline": round(whole_job_rate(ws, px_per_step, tots / steps2), 3),
                      "preprocess_plus_bin_sort_ms": round(float(prep.mean()), 4),
                      "rasterize_ms": round(float(raster.mean()), 4)}
    # the other grouping / precision combinations of the paper's comparison (Table 3, Table 5)
    variants = {}
    for prec, tl, memb in (("fp32", (2, 2), False), ("fp16_tc", (1, 1), True)):
        rv = tgs.Renderer(ds, cams, tl, prec, membership=memb)
        totv, framesv, _, _ = timed(rv, steps2, 3)
        if rv.overflowed():
            raise RuntimeError("bin capacity overflow during the benchmark")
        variants[f"{prec}_{tl[0]}x{tl[1]}" + ("" if memb else "_range")] = {
            "value": round(whole_job_rate(ws, px_per_step, totv / steps2), 3), "unit": UNIT,
            "frame_ms_p99": round(float(np.percentile(framesv, 99)), 4)}
        del rv

    # split of the preprocess + bin sort stage for one frame (direct calls)
    rs = R["main"][1]
    e = [ev() for _ in range(3)]
    e[0].record(stream)
    tgs.preprocess(ds, cams[0], out=rs.proj)
    e[1].record(stream)
    tgs.bin_sort(rs.proj, W, H, tiling, bins=rs.bins, sync=False)
    e[2].record(stream)
    torch.cuda.synchronize()
    stages = {"note": "the headline path without the frame pipeline (CUDA events between the stages)",
              "value_without_pipeline": paths["main"]["value_without_pipeline"],
              "preprocess_plus_bin_sort_ms": paths["main"]["preprocess_plus_bin_sort_ms"],
              "rasterize_ms": paths["main"]["rasterize_ms"],
              "preprocess_ms_direct": round(e[0].elapsed_time(e[1]), 4),
              "bin_sort_ms_direct": round(e[1].elapsed_time(e[2]), 4)}

    # algorithmic work of the dominant kernel per launch. The plain algorithm's pairs: (pixel,
    # entry) pairs evaluated before termination on the original tile lists (every tile of the AABB
    # range, no skip); the pairs the headline path evaluates (membership lists, producer skip);
    # the pairs that pass 1/255 (one exponential each).
    cnt_plain = torch.zeros(3, dtype=torch.int64, device="cuda")
    cnt_main = torch.zeros(3, dtype=torch.int64, device="cuda")
    ent_plain = ent_main = 0
    for i, cam in enumerate(cams):
        tgs.preprocess(ds, cam, out=rs.proj)
        for c, memb, cull in ((cnt_plain, False, False), (cnt_main, True, True)):
            bins = tgs.bin_sort(rs.proj, W, H, tiling, membership=memb)
            tgs.rasterize(rs.proj, bins, W, H, args.precision, out=(rs.out[i][0], rs.out[i][1], None),
                          want_n_contrib=False, counters=c, cull=cull)
            if memb:
                ent_main += bins.entries
            else:
                ent_plain += bins.entries
    torch.cuda.synchronize()
    pairs, exps, _ = [int(v) / ncam for v in cnt_plain.cpu().tolist()]
    pairs_main, _, slots = [int(v) / ncam for v in cnt_main.cpu().tolist()]

    # end to end through the C ABI with host buffers: every step is one tgs_frames_render call that
    # uploads the scene from pinned host memory and renders the eight cameras into pinned host images
    # (the copies overlap the kernels: two device scene copies, three frame buffer sets in flight)
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).pin_memory()
            for k in ("means", "scales", "quats", "opacities", "sh")}
    host_scene = types.SimpleNamespace(sh_degree=scene.sh_degree, **host)
    host_imgs = torch.empty((ncam, 3, H, W), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 4 for t in host.values())
    d2h = host_imgs.numel() * 4
    frames = tgs.Frames(scene.n, max_size=(W, H), max_entries=int(max(ent_main, 1) / ncam * 1.5) + 4096,
                        tiling=tiling, precision=args.precision, sets=3, max_sh_degree=scene.sh_degree,
                        device=local)

    def e2e_step():
        frames.render(host_scene, cams, host_imgs, stream=stream)

    for _ in range(2):
        e2e_step()
    frames.wait()
    e2e_steps = max(3, args.steps // 2)
    a, b = ev(), ev()
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    frames.wait()  # raises on a capacity overflow or a bin-sort time-out
    frames.close()
    clocks = sampler.stop()
    e2e_ms = max_over_ranks(a.elapsed_time(b) / e2e_steps, dist, "cuda")
    e2e_value = whole_job_rate(ws, px_per_step, e2e_ms)

    # roofline of the dominant kernel: the plain algorithm evaluates one ex2 per pair on the
    # special-function units (the scarcest unit it uses), so its pair rate is bounded by the
    # measured ex2 rate of this GPU
    peaks, peak_kind = _peaks()
    unit_peaks = _unit_peaks(local)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", SM_MAX_MHZ)
    mufu_peak = unit_peaks["ex2_per_s"] / 1e9
    raster_avg_ms = paths["main"]["rasterize_ms"]
    achieved = pairs / (raster_avg_ms * 1e-3) / 1e9
    kernel = "k_raster_tc" if tc else "k_raster_fp32"
    roofline = {"bound": "alu", "kernel": kernel,
                "achieved": round(achieved, 2), "peak": round(mufu_peak, 1), "unit": "Gpair/s",
                "frac": round(achieved / mufu_peak, 4), "traffic": _traffic(kernel, args),
                "peak_source": f"measured: ex2.approx.f32 microbenchmark on this GPU ({unit_peaks['sm_count']} SMs; "
                               f"{unit_peaks['ex2_per_s'] / unit_peaks['sm_count'] / (sm_mhz * 1e6):.1f} ex2/clk/SM at "
                               f"the {sm_mhz:.0f} MHz sampled during the timed phases); one ex2 per evaluated "
                               "(pixel, entry) pair of the plain algorithm",
                "work_per_launch": {"evaluated_pairs_plain": pairs, "evaluated_pairs_headline_path": pairs_main,
                                    "pixel_slots_stepped": slots, "exp_evaluations": exps,
                                    "group_entries": ent_main / ncam, "group_entries_plain": ent_plain / ncam},
                "avg_launch_ms": round(raster_avg_ms, 4),
                "exp_rate_gexps": round(exps / (raster_avg_ms * 1e-3) / 1e9, 2),
                "ffma_peak_per_s": unit_peaks["ffma_per_s"],
                "sm_mhz_during_timing": sm_mhz}
    rec = NCU_FRACTIONS.get(kernel)
    if rec is not None and rec["sha1"] == _kernel_sources_sha1(kernel):
        roofline["ncu"] = {k: v for k, v in rec.items() if k != "sha1"}

    plain = paths["fp32_plain"]
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPE[args.precision],
           "data": "synthetic", "config": _config(scene, cams, args),
           "frame_ms": {"mean": round(float(frames_ms.mean()), 4), "p50": round(float(np.percentile(frames_ms, 50)), 4),
                        "p99": round(float(np.percentile(frames_ms, 99)), 4),
                        "definition": "interval between consecutive frame completions"},
           "frame_latency_ms": {"p50": round(float(np.percentile(latency_ms, 50)), 4),
                                "p99": round(float(np.percentile(latency_ms, 99)), 4),
                                "definition": "first kernel of the frame to its last (includes waiting for "
                                              "the previous frame's rasterize)"},
           "fps": round(1000.0 / float(frames_ms.mean()), 2),
           "fp32_core_1x1": dict(plain, note="the plain FP32 CUDA-core tile rasterizer: 1x1 tiles, every tile of "
                                             "each Gaussian's AABB range (the original organization)"),
           "ablations": {
               "fp32_core_1x1_with_membership": dict(paths["fp32_membership"], note="FP32 CUDA cores on the same "
                                                     "membership lists as the headline path (skip for skip)"),
               **({"fp16_tc_range_lists": dict(paths["tc_range_skip"], note="tensor cores, AABB-range lists, the "
                                               "rasterizer's own per-(Gaussian, tile) skip"),
                   "fp16_tc_range_lists_no_skip": dict(paths["tc_range_noskip"], note="tensor cores, AABB-range lists, "
                                                       "no skip at all (the paper's organization)")} if tc else {}),
               "headline": {k: paths["main"][k] for k in ("value", "value_without_pipeline", "rasterize_ms",
                                                          "preprocess_plus_bin_sort_ms")}},
           "variants": variants,
           "speedup_vs_fp32_core": round(value / plain["value"], 3),
           "rasterize_speedup_vs_fp32_core": round(plain["rasterize_ms"] / raster_avg_ms, 3),
           "rasterize_speedup_skip_for_skip": round(paths["fp32_membership"]["rasterize_ms"] / raster_avg_ms, 3),
           "stages": stages,
           "evals_per_s": round(pairs * ncam / (ms_per_step * 1e-3), 1),
           "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4),
                   "how": "per step: one tgs_frames_render call (C ABI, host buffers): the scene uploaded "
                          "from pinned host memory, preprocess -> bin sort -> rasterize per camera, every image "
                          "downloaded into pinned host memory; copies overlapped with the kernels (two device "
                          "scene copies, three frame buffer sets in flight)"},
           "gpu_launches": launches,
           "kernels_per_frame": R["main"][0].kernels_per_frame[0],
           "graphs": "one CUDA graph pair per camera (preprocess + bin sort, rasterize); the preprocess + "
                     "bin sort of a frame runs on a second stream of the highest priority, overlapping the previous "
                     "frame's rasterize",
           "clocks": clocks,
           "roofline": roofline}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        for k, t in host.items():  # restore the scene (the e2e loop copied the same values back)
            getattr(ds, k).copy_(t)
        rend = R["main"][0]
        rgb, _ = rend.render(0)
        rend.join()
        torch.cuda.synchronize()
        rec, psnr = cpu_baseline(scene, cams[0], tc_image=rgb.cpu().numpy(), target_s=args.cpu_sample_s)
        out["cpu_baseline"] = rec
        out["psnr_vs_oracle_sampled"] = round(psnr, 3) if psnr is not None and math.isfinite(psnr) else psnr
    if ws == 1 and not args.no_extra_workloads:
        # the other workloads of the evaluation, in the same run: 6M Gaussians at 3840x2160 (grouping
        # x precision autotune with its error against the oracle), forward + backward, and the
        # rendering service under a sweep of offered rates
        del R, rs, frames, ds
        torch.cuda.empty_cache()
        import argparse as _ap
        sub = _ap.Namespace(**vars(args))
        sub.return_dict = True
        sub.steps = 5
        sub.cpu_sample_s = 6.0
        extra = {"dense4k": run_dense4k(sub)}
        torch.cuda.empty_cache()
        extra["backward"] = run_backward(sub)
        torch.cuda.empty_cache()
        rates = [float(r) for r in args.rates.split(",")]
        # 4 s of arrivals per rate: a p99 per resolution then rests on 200-500 requests below
        # saturation (at 2 s it was set by the two largest latencies of ~100)
        res, hbm = serve_sweep(rates, 4.0, args.precision, tiling, local)
        extra["serve"] = {"metric": "serve frames/s & p50/p99 latency per resolution (4 resident scenes)",
                          "seconds_per_rate": 4.0, "rates": res, "hbm_bytes": hbm}
        out["workloads"] = extra
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
