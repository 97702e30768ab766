#!/usr/bin/env python
"""Benchmark: forward + backward throughput of the Gaussian Mesh Renderer hot
path (mesh-to-Gaussian conversion, EWA projection, tile binning and sorting,
alpha compositing, and the backward to vertices and face colours/opacity).

Metric: Mpixel-views/s = (pixels over all views) / (fwd + bwd time) / 1e6 for
one step, where a step renders every view of the workload, computes the L2
loss against fixed target images and runs the full backward. The headline
value is the batched form (all views in one call, captured in a CUDA graph);
the per-view form (one call per view) is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmr|reference]
Under torchrun (N > 1) every rank runs an independent replica of the
workload (the path is not sharded); value = pixels of all ranks / slowest rank.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gmr_inputs as gi  # noqa: E402

METRIC = "fwd+bwd Mpixel-views/s and ms/iter, batched vs per-view, at ≤1e-5 img err"
UNIT = "Mpixel-views/s"
DEFAULT_WORKLOAD = "icosphere6_noise_64xuneven"
WORKLOADS = {
    "icosphere5_sin_8x512": gi.scene_ring,
    "icosphere3_1x128": gi.scene_single_view,
    "icosphere6_noise_64xuneven": gi.scene_fibonacci_uneven,
    "icosphere8_perlin_16x1024": gi.scene_large,
    "icosphere7_fit_4x512": gi.scene_fit,
    # the level-8 mesh in 2 views: a dense case small enough (about 2 GB on
    # the device) for multi-pass profiler captures of the dense-mesh kernels
    "icosphere8_perlin_2x1024": lambda: gi.scene_large(n_views=2),
    # the first 16 of the 64 uneven views' resolution draws: the 64-view
    # workload's kernels at about a quarter of its size, for full captures
    "icosphere6_noise_16xuneven": lambda: gi.scene_fibonacci_uneven(n_views=16),
}
# the optimisation-loop workload: a step is one Adam step of the fit (render
# 4 views of 512^2, loss, backward, parameter update)
FIT_WORKLOAD = "icosphere7_fit_4x512"

# FP32 peak of the CUDA cores: 148 SMs x 128 lanes x 2 (FMA) x 2.032 GHz.
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# Algorithmic FP32 operations (FMA = 2) per evaluated (pixel, Gaussian) pair
# and per contributing pair, counted from the compositing formulas.
FLOPS_EVAL = 13
FLOPS_FWD_CONTRIB = 10
FLOPS_BWD_CONTRIB = 59
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) that
# one ncu capture measured for the dominant kernel, per workload and launch
# shape (tile, backward threads, batch, persistent, backward layout); an
# entry is removed when
# the kernel changes after its capture.
NCU_TRAFFIC = {("raster_bwd", "icosphere6_noise_64xuneven", (16, 128, 256, 0, 1)): 1857956608,
               ("raster_bwd", "icosphere8_perlin_16x1024", (8, 32, 64, 0, 2)): 8664350464,
               ("raster_bwd", "icosphere5_sin_8x512", (16, 128, 256, 0, 0)): 81138944}

L2_FLUSH_BYTES = 512 << 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clock, power and clock-event reasons with nvidia-smi while
    the benchmark runs (read-only queries)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, local_rank, period_ms=100):
        self.samples = []
        self.proc = None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.cmd = ["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    f"-lms", str(period_ms)]

    def _reader(self):
        for line in self.proc.stdout:
            t = time.perf_counter()
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                mhz, mx, pw = float(parts[0]), float(parts[1]), float(parts[2])
            except ValueError:
                continue
            active = [n for n, v in zip(self.NAMES, parts[3:]) if v.lower() == "active"]
            self.samples.append((t, mhz, mx, pw, active))

    def start(self):
        import subprocess

        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError as e:
            log(f"clock sampling unavailable: {e}")
            self.proc = None
            return
        self.th = threading.Thread(target=self._reader, daemon=True)
        self.th.start()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.th.join(timeout=5)

    def summary(self, t0, t1):
        if not self.samples:
            return None
        inside = [s for s in self.samples if t0 <= s[0] <= t1 + 0.15]
        window = "timed"
        if len(inside) < 3:
            inside = self.samples
            window = "warmup+timed"
        reasons = sorted({n for s in inside for n in s[4]})
        return {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": max(s[2] for s in inside),
                "reasons": reasons, "samples": len(inside), "window": window,
                "power_w_max": max(s[3] for s in inside)}


# ---------------------------------------------------------------- distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------- oracle timing
def oracle_sample_time(scene, n_pix, seed=0, keep=False):
    """Oracle fwd + bwd on n_pix random (distinct) pixels of the workload:
    seconds and the number of pixels; with keep=True also the pixels, the
    oracle's render and backward and the upstream gradient it used."""
    import oracle

    rng = np.random.default_rng(seed)
    pix = []
    for _ in range(n_pix):
        c = int(rng.integers(len(scene.cams)))
        pix.append((c, int(rng.integers(int(scene.cams[c]["width"]))), int(rng.integers(int(scene.cams[c]["height"])))))
    pix = np.unique(np.array(pix, dtype=np.int32), axis=0)
    t0 = time.perf_counter()
    r = oracle.render(scene, pixels=pix)  # with the ambiguity flags the parity check excludes
    g = 2.0 * (r["rgb"] - 0.5)
    g[r["flags"] != 0] = 0.0  # no gradient through pixels near a decision threshold
    b = oracle.backward(scene, g, pixels=pix)
    t = time.perf_counter() - t0
    if keep:
        return t, len(pix), (pix, r, g, b)
    return t, len(pix)


def cpu_baseline(scene, target_seconds, gpu_check=None):
    """The oracle timed on bounded samples of the workload's pixels, on every
    host core (OpenMP over pixels, records and faces; the headline value) and
    on one thread, in its binned mode (each pixel walks the faces its 16x16
    grid cell lists; bit-identical to its brute force). With gpu_check, the
    GPU's image at the all-cores sample's pixels and its gradients for the
    same upstream gradient are compared with the oracle's."""
    import oracle

    cores = oracle.set_threads(0)
    was_binned = oracle.set_binned(True)
    # calibration on all cores: one pixel (the per-call conversion,
    # projection and depth sort of every record dominate) and 64 per core
    t_a, n_a = oracle_sample_time(scene, 1)
    t_b, n_b = oracle_sample_time(scene, 64 * cores)
    per_px = max((t_b - t_a) / max(n_b - n_a, 1), 1e-7)
    fixed = max(t_a - n_a * per_px, 0.0)
    n = int(max(64, min(4000000, (target_seconds - fixed) / per_px)))
    t, n, kept = oracle_sample_time(scene, n, seed=1, keep=True)
    # the two calibration calls are single timings: when one was noisy and
    # the sample ended well short of the target, size it again from its own
    # rate (once)
    if t < 0.5 * target_seconds and n < 4000000:
        per_px_s = max((t - fixed) / n, 1e-7)
        n2 = int(min(4000000, (target_seconds - fixed) / per_px_s))
        if n2 > 1.5 * n:
            t, n, kept = oracle_sample_time(scene, n2, seed=1, keep=True)
    # one thread: its per-pixel and fixed costs are at most `cores` times the
    # all-core ones (the parallel loops scale at best linearly), so this many
    # pixels take at most about target_seconds
    per_px = max((t - fixed) / n, per_px)
    oracle.set_threads(1)
    n1_req = int(max(8, min(n, (target_seconds - fixed * cores) / (per_px * cores))))
    t1, n1 = oracle_sample_time(scene, n1_req, seed=2)
    out = {"value": n / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} random pixels of the {len(scene.cams)}-view workload, FP64 binned fwd+bwd "
                     f"on {cores} host threads (os.cpu_count() = {os.cpu_count()}), {t:.1f} s",
           "single_thread": {"value": n1 / t1 / 1e6, "unit": UNIT, "cores": 1,
                             "sample": f"{n1} random pixels, one thread, {t1:.1f} s"}}
    oracle.set_binned(was_binned)
    if gpu_check is not None:
        out["parity"] = gpu_check(*kept)
    return out


def parity_with_oracle(r, v, f, c, o, cams, scene, pix, ref, g, bref):
    """GPU image at the oracle's pixels (max abs error over the pixels no
    decision threshold is near, as the tests count it) and GPU gradients for
    the oracle's upstream gradient at those pixels (relative L2)."""
    import torch

    img, _ = r.forward(v, f, c, o, cams, want_t=False)
    widths = np.array([int(cm["width"]) for cm in scene.cams])
    heights = np.array([int(cm["height"]) for cm in scene.cams])
    off = np.concatenate([[0], np.cumsum(widths * heights)])
    lin = off[pix[:, 0]] + pix[:, 2] * widths[pix[:, 0]] + pix[:, 1]
    gimg = img[torch.from_numpy(lin).to(img.device)].double().cpu().numpy()
    amb = (ref["flags"] & 3) != 0  # alpha-skip or termination decision near its threshold
    err = np.abs(gimg - ref["rgb"]).max(1)
    gfull = torch.zeros_like(img)
    gfull[torch.from_numpy(lin).to(img.device)] = torch.from_numpy(g.astype(np.float32)).to(img.device)
    dv, dc, _ = r.backward(gfull)
    dv, dc = dv.double().cpu().numpy(), dc.double().cpu().numpy()

    def rel(a, b):
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))

    e_img = float(err[~amb].max()) if (~amb).any() else 0.0
    e_v, e_c = rel(dv, bref["dverts"]), rel(dc, bref["drgb"])
    return {"pixels": int(len(pix)), "ambiguous_pixels": int(amb.sum()), "img_max_abs_err": e_img,
            "dverts_rel_l2": e_v, "drgb_rel_l2": e_c, "ok": bool(e_img <= 1e-5 and e_v <= 1e-4 and e_c <= 1e-4)}


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle (the paper publishes no code), fwd +
    bwd of a bounded random pixel sample per step, on every host core, in
    its binned mode."""
    if rank != 0:
        return
    import oracle

    cores = oracle.set_threads(0)
    oracle.set_binned(True)
    scene = WORKLOADS[args.workload]()
    n_pix = args.ref_pixels
    for _ in range(args.warmup):
        oracle_sample_time(scene, max(8, n_pix // 8))
    runs = [oracle_sample_time(scene, n_pix, seed=k + 1) for k in range(args.steps)]
    total = sum(t for t, _ in runs)
    n_done = sum(n for _, n in runs)
    value = n_done / total / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "step": f"oracle fwd+bwd on {n_pix} random pixels"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{n_pix} random pixels per step, FP64 binned, {cores} host threads"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_fit(args, ws, rank, local):
    """The fitting loop (level-7 icosphere to a deformed shape, 4 random
    views of 512^2 per step, Adam lr 1e-3): per-step time of the batched and
    the per-view form, loss and chamfer distance before and after."""
    import torch

    from paper_2602_14493_b300 import Renderer, camera_array
    from paper_2602_14493_b300.fit import fit, render_targets

    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sampler = ClockSampler(local, period_ms=50)
    sampler.start()
    K, W = args.steps, args.warmup
    scene = gi.scene_fit(steps=K)
    r = Renderer()
    faces = torch.from_numpy(scene.faces).to(dev)
    op = torch.from_numpy(scene.opacity).to(dev)
    v0 = torch.from_numpy(scene.verts).to(dev)
    c0 = torch.from_numpy(scene.rgb).to(dev)
    cams0 = camera_array(scene.extra["view_sets"][0])
    targets = render_targets(r, torch.from_numpy(scene.extra["target_verts"]).to(dev), faces,
                             torch.from_numpy(scene.extra["target_rgb"]).to(dev), op, scene.extra["view_sets"])
    shape_choice = "default"
    if args.tile == "auto":  # launch shape tuned on the first step's views
        from paper_2602_14493_b300.autotune import shape_name, tune

        best, tuned = tune(r, v0, faces, c0, op, cams0, targets[0], use_cache=False)
        log("autotune:", {shape_name(k): round(t, 4) for k, t in sorted(tuned.items(), key=lambda kv: kv[1])[:8]})
        shape_choice = "autotuned " + shape_name(best)
    # no host synchronisation inside a step: workspace reserved with room for
    # twice the first views' pairs (an overflow would set the device status
    # reported below)
    r.forward(v0, faces, c0, op, cams0, want_t=False)
    n_pix0 = sum(int(cm.width) * int(cm.height) for cm in cams0)
    r.reserve(len(scene.faces), len(cams0), n_pix0, 2 * r.stats()["n_pairs"] + 4096)
    r.set_config(sync_check=False)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    fit(scene, steps=W, renderer=r, targets=targets[:W])  # warm-up of both forms
    fit(scene, steps=W, form="per_view", renderer=r, targets=targets[:W])
    torch.cuda.synchronize()
    barrier(ws)
    t_wall0 = time.perf_counter()
    out_b = fit(scene, steps=K, form="batched", renderer=r, targets=targets, between_steps=flush.zero_)
    out_p = fit(scene, steps=K, form="per_view", renderer=r, targets=targets, between_steps=flush.zero_)
    t_wall1 = time.perf_counter()
    sampler.stop()
    n_pix = out_b["pixels_per_step"]
    tb = max_over_ranks(float(out_b["ms"].sum()) / 1e3, ws)
    tp = max_over_ranks(float(out_p["ms"].sum()) / 1e3, ws)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(scene, args.cpu_seconds)
    out = {
        "metric": METRIC, "value": ws * n_pix * K / tb / 1e6, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": 1e3 * tb / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32", "data": "synthetic",
        "config": {"workload": FIT_WORKLOAD, "faces": len(scene.faces), "views_per_step": len(scene.cams),
                   "pixels_per_step": n_pix, "optimizer": "adam", "lr": 1e-3,
                   "step": "render 4 views + L2 loss + backward + Adam on vertices and face colours",
                   "form": "batched, one call for all views of a step, eager",
                   "shape_choice": shape_choice, "host_sync": "none inside a step (workspace reserved)",
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "per_view": {"value": ws * n_pix * K / tp / 1e6, "ms_per_step": 1e3 * tp / K,
                     "form": "one call per view, eager"},
        "fit": {"loss_first": float(out_b["loss"][0]), "loss_last": float(out_b["loss"][-1]),
                "chamfer_initial": out_b["chamfer_initial"], "chamfer_final": out_b["chamfer_final"],
                "chamfer_final_per_view": out_p["chamfer_final"]},
        "roofline": None, "cpu_baseline": cpu, "e2e": None,
        "clocks": sampler.summary(t_wall0, t_wall1),
        "device_status": out_b["status"] | out_p["status"],
    }
    print(json.dumps(out), flush=True)


def run_gmr(args, ws, rank, local):
    import torch

    from paper_2602_14493_b300 import Renderer, camera_array, copy_h2d

    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sampler = ClockSampler(local, period_ms=50)
    sampler.start()
    scene = WORKLOADS[args.workload]()
    C, F = len(scene.cams), len(scene.faces)
    n_pix = scene.n_pixels

    v = torch.from_numpy(scene.verts).to(dev)
    f = torch.from_numpy(scene.faces).to(dev)
    c = torch.from_numpy(scene.rgb).to(dev)
    o = torch.from_numpy(scene.opacity).to(dev)
    cams = camera_array(scene.cams)

    # the timed graph brackets only the dominant kernel's stage with events;
    # the breakdown of all stages comes from separate profiled replays
    r = Renderer(profile=[DOMINANT])
    # target: render of the jittered mesh
    vt = torch.from_numpy(scene.extra["target_verts"]).to(dev)
    target, _ = r.forward(vt, f, c, o, cams, want_t=False)
    target = target.clone()
    if args.tile == "auto":
        from paper_2602_14493_b300.autotune import shape_name, tune

        (tile, threads, threads_bwd, batch, persistent, layout_fwd, layout_bwd), tuned = tune(r, v, f, c, o, cams,
                                                                                              target, use_cache=False)
        log("autotune:", {shape_name(k): round(t, 4) for k, t in sorted(tuned.items(), key=lambda kv: kv[1])[:8]})
        # the fastest full-warp shape with one CTA per tile and as a persistent
        # grid, and the half-warp layouts the tuner tried
        full = min((k for k in tuned if k[4:] == (0, 0, 0)), key=tuned.get)
        scheduler = {"per_tile_grid_ms": tuned.get(full), "persistent_ms": tuned.get(full[:4] + (1, 0, 0)),
                     "layouts_ms": {shape_name(k): round(t, 4) for k, t in tuned.items() if k[5] or k[6]},
                     "layout_codes": "last two fields: forward, backward layout; 0 block-staged, 1 half-warp, "
                                     "2 warp-staged",
                     "best_ms_per_tile": {str(t): round(min(v for k, v in tuned.items() if k[0] == t), 4)
                                          for t in sorted({k[0] for k in tuned})},
                     "source": "autotuner, eager fwd + loss + bwd step, median of 15"}
    else:
        tile, threads, batch = int(args.tile), args.threads, args.batch
        threads_bwd = args.threads_bwd or threads
        persistent, layout_fwd, layout_bwd = int(args.persistent), int(args.layout_fwd), int(args.layout_bwd)
        scheduler = None
        r.set_config(tile=tile, threads=threads, threads_bwd=threads_bwd, batch=batch, persistent=bool(persistent),
                     half_fwd=layout_fwd == 1, half_bwd=layout_bwd == 1, warp_fwd=layout_fwd == 2,
                     warp_bwd=layout_bwd == 2, deterministic=bool(args.deterministic))
    img, _ = r.forward(v, f, c, o, cams, want_t=False)
    torch.cuda.synchronize()
    P = r.stats()["n_pairs"]
    r.reserve(F, C, n_pix, int(P * 1.3) + 4096)
    r.set_config(sync_check=False)
    stream = torch.cuda.Stream(dev)
    img = torch.empty((n_pix, 3), device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    dv, dc, do = torch.empty_like(v), torch.empty_like(c), torch.empty_like(o)

    def step(s):
        # forward, then the squared-error loss and the backward in one call
        # (the loss formed in the compositing backward's prologue,
        # gmr_render_bwd_l2: 1% faster than gmr_l2_loss + gmr_render_bwd;
        # the loss fused into the forward's epilogue, gmr_render_fwd_l2,
        # measured slower)
        r.forward(v, f, c, o, cams, images=img, want_t=False, stream=s)
        r.backward_l2(img, target, loss, dv, dc, do, stream=s)

    with torch.cuda.stream(stream):
        step(stream)
    stream.synchronize()
    l0 = r.stats()["launches"]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(stream)
    launches_per_step = r.stats()["launches"] - l0
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    st = r.stats()
    if r.device_status() != 0:
        raise RuntimeError("device status bits set during warm-up")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_acc = {}
    barrier(ws)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
            flush.zero_()  # L2 flush between timed steps (outside the events)
        times = r.stage_times(stream)
        for name, ms in times.items():
            if ms is not None:
                stage_acc.setdefault(name, []).append(ms)
    torch.cuda.synchronize()
    barrier(ws)
    t_wall1 = time.perf_counter()
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    total_s_max = max_over_ranks(total_s, ws)
    value = ws * n_pix * args.steps / total_s_max / 1e6
    ms_per_step = 1e3 * total_s_max / args.steps
    status = r.device_status()

    # per-view form: one call per view (eager, same workspace)
    pv_steps = max(3, min(args.steps, 30))
    cams_k = [camera_array(scene.cams[k:k + 1]) for k in range(C)]
    with torch.cuda.stream(stream):
        off = np.concatenate([[0], np.cumsum([int(cm.width) * int(cm.height) for cm in cams])])

        def per_view_step():
            for k in range(C):
                sl = slice(int(off[k]), int(off[k + 1]))
                r.forward(v, f, c, o, cams_k[k], images=img[sl], want_t=False, stream=stream)
                r.backward_l2(img[sl], target[sl], loss, dv, dc, do, accumulate=(k > 0), stream=stream)

        for _ in range(2):
            per_view_step()
        stream.synchronize()
        pv_ev = []
        for _ in range(pv_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            per_view_step()
            b.record(stream)
            flush.zero_()
            pv_ev.append((a, b))
        stream.synchronize()
        pv_ms = statistics.mean(a.elapsed_time(b) for a, b in pv_ev)
        # batched, eager (no graph)
        be_ev = []
        for _ in range(pv_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(stream)
            b.record(stream)
            flush.zero_()
            be_ev.append((a, b))
        stream.synchronize()
        be_ms = statistics.mean(a.elapsed_time(b) for a, b in be_ev)

    # end to end through the public API with host buffers. Every step copies
    # its inputs (mesh and target images) from pinned host memory and reads
    # its results (loss and gradients) back; the copies of step k + 1 run on
    # a copy stream while step k computes (double-buffered inputs), and the
    # host waits for each step's results before it goes on. The inputs are
    # copied by gmr_copy_h2d (below 64 MiB a kernel reading the pinned host
    # buffers over the bus, faster than the copy engine for such sizes on
    # these hosts; larger buffers, such as the 64-view targets, by the copy
    # engine).
    h_v = torch.from_numpy(scene.verts).pin_memory()
    h_f = torch.from_numpy(scene.faces).pin_memory()
    h_c = torch.from_numpy(scene.rgb).pin_memory()
    h_o = torch.from_numpy(scene.opacity).pin_memory()
    h_t = target.cpu().pin_memory()
    h_in = (h_v, h_f, h_c, h_o, h_t)
    d_in = [tuple(torch.empty_like(x, device=dev) for x in h_in) for _ in range(2)]
    h_out = [tuple(torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in (loss, dv, dc, do)) for _ in range(2)]
    h2d = sum(x.numel() * x.element_size() for x in h_in)
    d2h = sum(x.numel() * x.element_size() for x in h_out[0])
    e2e_steps = max(3, min(args.steps, 30))
    copy_stream = torch.cuda.Stream(dev)

    def e2e_run(n):
        copied = [torch.cuda.Event() for _ in range(n)]
        done = [torch.cuda.Event() for _ in range(n)]

        def enqueue_copy(k):
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(done[k - 2])  # slot k % 2 free again
                for d, h in zip(d_in[k % 2], h_in):
                    copy_h2d(d, h, stream=copy_stream)
                copied[k].record(copy_stream)

        def enqueue_compute(k):
            d_v, d_f, d_c, d_o, d_t = d_in[k % 2]
            with torch.cuda.stream(stream):
                stream.wait_event(copied[k])
                r.forward(d_v, d_f, d_c, d_o, cams, images=img, want_t=False, stream=stream)
                r.backward_l2(img, d_t, loss, dv, dc, do, stream=stream)
                for h, d in zip(h_out[k % 2], (loss, dv, dc, do)):
                    h.copy_(d, non_blocking=True)
                done[k].record(stream)

        enqueue_copy(0)
        for k in range(n):
            if k + 1 < n:
                enqueue_copy(k + 1)
            enqueue_compute(k)
            if k >= 1:
                done[k - 1].synchronize()  # step k - 1's loss and gradients are on the host
        done[n - 1].synchronize()

    e2e_run(3)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, ws)

    # stage breakdown: the same step captured with events around every stage
    r.set_config(profile=True)
    with torch.cuda.stream(stream):
        step(stream)  # the per-view runs changed the cameras: upload the batch's again
    stream.synchronize()
    graph_prof = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_prof, stream=stream):
        step(stream)
    prof_acc, prof_ms = {}, []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph_prof.replay()
            b.record(stream)
            flush.zero_()
        times = r.stage_times(stream)
        if k >= args.warmup:
            prof_ms.append(a.elapsed_time(b))
            for name, ms in times.items():
                if ms is not None:
                    prof_acc.setdefault(name, []).append(ms)
    r.set_config(profile=[DOMINANT])

    if rank != 0:
        return
    stats = r.stats()
    peaks, peak_kind = measured_peaks()
    stage_ms = {k: statistics.mean(vs) for k, vs in prof_acc.items()}
    kern = {k: vv for k, vv in stage_ms.items() if k != "loss"}
    if kern and max(kern, key=kern.get) != DOMINANT:
        log(f"note: the largest stage is {max(kern, key=kern.get)}, not {DOMINANT}")
    if stage_acc.get(DOMINANT):
        # duration of the dominant kernel inside the timed steps themselves
        roof = roofline_for(DOMINANT, statistics.mean(stage_acc[DOMINANT]), stats, scene, peaks, peak_kind, args,
                            shape=(tile, threads_bwd, batch, int(persistent), int(layout_bwd)))
    else:
        roof = None
        log("no stage times were recorded")
    # memory-type stages: algorithmic bytes over their live stage times
    stage_gbs = {}
    for name in ("project", "scan", "bin", "project_bwd"):
        if stage_ms.get(name):
            rf = roofline_for(name, stage_ms[name], stats, scene, peaks, peak_kind, args)
            stage_gbs[name] = {"achieved_gbs": round(rf["achieved"], 1), "frac": round(rf["frac"], 4)}
    free_b, total_b = torch.cuda.mem_get_info(dev)
    memory = {"workspace_gb": stats["workspace_bytes"] / 1e9,
              "torch_peak_gb": torch.cuda.max_memory_allocated(dev) / 1e9,
              "device_used_gb": (total_b - free_b) / 1e9}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, args.cpu_seconds,
                           lambda *kept: parity_with_oracle(r, v, f, c, o, cams, scene, *kept))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32", "data": "synthetic",
        "step_ms_spread": {"median": float(np.median(step_ms)), "p10": float(np.percentile(step_ms, 10)),
                           "p90": float(np.percentile(step_ms, 90)), "min": min(step_ms), "max": max(step_ms),
                           "source": "CUDA events around each timed graph replay (this rank)"},
        "config": {"workload": args.workload, "views": C, "faces": F, "pixels_per_step": n_pix,
                   "form": "batched, one call for all views, CUDA graph", "tile": tile, "threads": threads, "threads_bwd": threads_bwd,
                   "batch": batch, "persistent": bool(persistent), "deterministic": bool(args.deterministic),
                   "layout_fwd": ["block-staged", "half-warp", "warp-staged"][layout_fwd],
                   "layout_bwd": ["block-staged", "half-warp", "warp-staged"][layout_bwd],
                   "shape_choice": "autotuned" if args.tile == "auto" else "fixed",
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "per_view": {"value": n_pix / (pv_ms / 1e3) / 1e6, "ms_per_step": pv_ms, "form": "one call per view, eager"},
        "batched_eager": {"value": n_pix / (be_ms / 1e3) / 1e6, "ms_per_step": be_ms},
        "scheduler": scheduler,
        "stages_ms": {k: round(vv, 5) for k, vv in stage_ms.items()},
        "stages_source": "separate replays of the step captured with events around every stage "
                         f"({statistics.mean(prof_ms):.4f} ms per profiled step)",
        "roofline": roof,
        "stage_hbm": stage_gbs,
        "memory": memory,
        "cpu_baseline": cpu,
        "e2e": {"value": ws * n_pix / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s,
                "form": "public API, pinned host buffers copied by gmr_copy_h2d (kernel < 64 MiB, copy engine "
                        "above); step k+1's copies overlap "
                        "step k's compute"},
        "gpu_launches": launches_per_step * args.steps,
        "launches_per_step": launches_per_step,
        "clocks": sampler.summary(t_wall0, t_wall1),
        "counters": {"pairs": stats["n_pairs"], "evals_fwd": stats["evals_fwd"], "evals_bwd": stats["evals_bwd"],
                     "contribs": stats["contribs"]},
        "device_status": status,
    }
    print(json.dumps(out), flush=True)


DOMINANT = "raster_bwd"  # the step's largest kernel (compositing backward)


def roofline_for(stage, ms, stats, scene, peaks, peak_kind, args, shape=None):
    """Roofline entry of the dominant kernel from its live event time
    (shape: the launch shape (tile, backward threads, batch, persistent,
    backward layout), which selects the recorded DRAM traffic)."""
    E_f, E_b, K = stats["evals_fwd"], stats["evals_bwd"], stats["contribs"]
    if stage in ("raster_fwd", "raster_bwd"):
        flops = (FLOPS_EVAL * E_f + FLOPS_FWD_CONTRIB * K) if stage == "raster_fwd" else \
                (FLOPS_EVAL * E_b + FLOPS_BWD_CONTRIB * K)
        ach = flops / (ms / 1e3) / 1e12
        return {"kernel": stage, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None if args.deterministic else NCU_TRAFFIC.get((stage, args.workload, shape)),
                "peak_source": "FP32 CUDA-core peak from unit counts and max clock (148 SM x 128 x 2 x 2.032 GHz)",
                "ms": ms}
    # memory-type stages: algorithmic bytes per record, pair, tile and face
    R = stats["n_records"]
    P = stats["n_pairs"]
    # (the projection also writes the zeros of the backward's gradient sums:
    # 32 B per record, 16 B per face)
    byts = {"project": R * 96 + len(scene.faces) * 44 + P * 4, "scan": stats["n_tiles"] * 8,
            "bin": R * 16 + P * 8 * 3 + P * 4, "project_bwd": R * 48 + len(scene.faces) * 116}.get(stage, 0)
    ach = byts / (ms / 1e3) / 1e9
    pk = peaks["hbm_gbs"]
    return {"kernel": stage, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
            "traffic": None if args.deterministic else NCU_TRAFFIC.get((stage, args.workload, shape)), "peak_source": peak_kind, "ms": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gmr", choices=["gmr", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--tile", default="auto", help="8, 16, 32 or auto (autotuner)")
    ap.add_argument("--threads", type=int, default=128)
    ap.add_argument("--threads-bwd", type=int, default=0, help="backward threads per tile (0: as --threads)")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--persistent", type=int, default=0, help="with a fixed shape: 1 = persistent compositing grids")
    ap.add_argument("--layout-fwd", type=int, default=0,
                    help="with a fixed shape, forward layout: 0 block-staged, 1 half-warp, 2 warp-staged")
    ap.add_argument("--layout-bwd", type=int, default=0, help="with a fixed shape, backward layout (as --layout-fwd)")
    ap.add_argument("--deterministic", action="store_true",
                    help="with a fixed shape (block-staged backward): the fixed-order backward")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-pixels", type=int, default=65536)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == FIT_WORKLOAD:
        run_fit(args, ws, rank, local)
        return
    run_gmr(args, ws, rank, local)


if __name__ == "__main__":
    main()
