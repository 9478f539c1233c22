#!/usr/bin/env python
"""Throughput of the gaze-mapping hot path: sample x fixation pairs per second.

One step = the whole path on one synthetic workload: scene build (world transform + BVH),
area-weighted sampling, fixation prep, the fused cone/occlusion/Gaussian accumulation and the
max-normalisation, through the C ABI. `value` times steps with inputs already resident in
HBM (CUDA events, L2 flushed between steps); `e2e` times the same call from pinned host
buffers with the copies in and the map copy out inside the timed region.

  python bench.py [--gpus N --steps K --warmup W] [--impl gazemap|reference] [--workload ...]

Under torchrun (N > 1) the path is sharded by samples: every rank builds the scene, takes one
contiguous slice of the samples and accumulates it; the ranks exchange one maximum per window
(all-reduce) and normalise their slices by it (strong scaling: the workload is fixed); timing is
the max over ranks. `--impl reference` times the FP64 CPU oracle on this host's cores on a bounded sample
of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sample×fixation pairs/s at ≤1e-4 rel err"
FP32_INSTR_PER_PAIR = 18          # algorithmic FP32 work of the cone test per pair
FP32_INSTR_PER_NODE = 28          # two slab tests: 6 FMA + 6 min/max + two 3-input min/max each
FP32_INSTR_PER_TRI = 25           # watertight test: 3 x 3 sub, 6 products with 3 subtractions, U V W, det, T
FP32_INSTR_PER_INCONE = 12        # Gaussian (divide, scale, ex2, weight) and the compensated sum (4 adds)
FP32_INSTR_PER_ENTRY = 1          # eye grid: the depth-bound compare of a list entry
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_accumulate launch, from a
# one-pass ncu capture of the default bench command (paper scene, default flags and builder).
# The figure stands only while the sources that shape the kernel and its inputs are the ones it
# was taken on: their SHA-256 is stored beside it and `traffic` is null on any mismatch.
ACC_TRAFFIC = {"workload": "paper_scene_800ktri_2Msample_6000fix", "bytes": 168.055296e6,
               "sources_sha256": "23103779d73037ce45bbabf1a5134c689c5acd655942c8dcc03478fa3a1feed0"}
ACC_TRAFFIC_SOURCES = ("paper_2601_07571_gb300/csrc/gm_trace.cuh", "paper_2601_07571_gb300/csrc/gm_accum.cu",
                       "paper_2601_07571_gb300/csrc/gm_scene.cu", "paper_2601_07571_gb300/csrc/gm_sampler.cu")


def accumulate_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in ACC_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(workload: str, flags: int, builder: str, default_tree_and_segment: bool = True):
    if (ACC_TRAFFIC["bytes"] is None or workload != ACC_TRAFFIC["workload"] or flags != 0 or builder != "default"
            or not default_tree_and_segment):
        return None
    return ACC_TRAFFIC["bytes"] if accumulate_sources_sha256() == ACC_TRAFFIC["sources_sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gazemap", "reference"], default="gazemap")
    ap.add_argument("--workload", choices=["paper_scene", "tiny_sphere", "batched", "field", "city", "zbuffer",
                                           "dynamic", "sampler"],
                    default="paper_scene")
    ap.add_argument("--field-steps", type=int, default=30000, help="Adam steps of the neural field")
    ap.add_argument("--field-lr", type=float, default=1e-3, help="initial learning rate of the field")
    ap.add_argument("--field-lr-min", type=float, default=None, help="final learning rate (default lr / 100)")
    ap.add_argument("--no-field", action="store_true", help="leave the neural-field measurement out of the line")
    ap.add_argument("--field-batch", type=int, default=65536, help="training batch of the neural field")
    ap.add_argument("--queries", type=int, default=10_000_000, help="query points of the field workload")
    ap.add_argument("--sessions", type=int, default=64, help="sessions of the batched workload")
    ap.add_argument("--fixations", type=int, default=0, help="use only the first N fixations (profiling)")
    ap.add_argument("--flags", type=int, default=0, help="extra GM_F_* accumulation flags (variant A/B runs)")
    ap.add_argument("--builder", choices=["default", "lbvh", "ploc"], default="default", help="BVH builder")
    ap.add_argument("--ploc-radius", type=int, default=0, help="PLOC neighbour radius (0: library default 8)")
    ap.add_argument("--eps-rel", type=float, default=None,
                    help="occlusion segment end (1 - eps_rel of the way to the sample); default the workload's 1e-5")
    ap.add_argument("--zb-res", type=int, default=256, help="z-buffer pixels per side (zbuffer workload)")
    ap.add_argument("--zb-eps", type=float, default=0.005, help="z-buffer depth tolerance, metres (zbuffer workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    return ap.parse_args()


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """Max of a per-rank value over all ranks (identity without torch.distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, dist=None, device="cpu") -> float:
    """Sum of a per-rank value over all ranks (identity without torch.distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, slowest_s: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank / slowest_s


def make_workload(name, n_fix=0):
    import synth
    w = {"paper_scene": synth.paper_scene, "tiny_sphere": synth.tiny_sphere, "city": synth.city_block}[name]()
    if n_fix:
        w.fixations = w.fixations.subset(slice(0, n_fix))
    return w


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                if self.uuid and self.uuid not in p[1]:
                    continue
                rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------------------------
def oracle_sample_run(w, n_samples, nthreads):
    """The oracle as it stands: world triangles, areas and counts for the whole scene, then
    the sample positions and brute-force accumulation of `n_samples` evenly strided samples
    over every fixation. Returns (seconds, pairs)."""
    import oracle
    t0 = time.perf_counter()
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    n = int(off[-1])
    which = np.unique(np.linspace(0, n - 1, max(1, min(n_samples, n))).astype(np.int64))
    s = oracle.samples(tri, off, w.seed, w.session, which)
    oracle.accumulate(tri, s.xyz, s.tri, w.fixations, w.params, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return dt, len(which) * w.fixations.n


def calibrated_oracle(w, target_s, nthreads):
    n0 = nthreads
    dt, _ = oracle_sample_run(w, n0, nthreads)
    # scale the sample count so one run takes about target_s seconds (at least one per thread)
    n = int(max(n0, min(20000, n0 * target_s / max(dt, 1e-3))))
    dt, pairs = oracle_sample_run(w, n, nthreads)
    return dt, pairs, n


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload, args.fixations)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    dt, _ = oracle_sample_run(w, cores, cores)
    n = int(max(cores, min(20000, cores * per_step / max(dt, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample_run(w, n, cores)
    tot_t, tot_p = 0.0, 0
    for _ in range(args.steps):
        dt, p = oracle_sample_run(w, n, cores)
        tot_t += dt
        tot_p += p
    v = tot_p / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "fixations": w.fixations.n},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": min(cores, n), "kind": "oracle",
                             "sample": f"{n} evenly strided samples x all {w.fixations.n} fixations per step, "
                                       f"whole-scene transform/areas/counts included"},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def measured_bf16_peak():
    """Dense BF16 peak (TFLOP/s) for a kernel timed alone: the measured burst figure of
    MEASURED_PEAKS.json, else a fallback of 1.9 PFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured burst cuBLAS bf16 (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16"


def batched_arm(args):
    """64 independent sessions (5k-300k tris, 500-20k fixations, 1e3-5e4 samples/m^2, log-uniform):
    the plain form (one gm_accumulate_fixations per session, back to back on one stream) against
    the batched form (one replay of the autotuned, graph-captured persistent plan). Scenes and
    samples are built before timing; both forms include the fixation prep and normalisation."""
    import torch
    import synth
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    torch.cuda.set_device(0)
    ws = synth.batched_sessions(args.sessions)
    ctx = G.gm_create(0)
    stream = torch.cuda.current_stream()
    hs = []
    for w in ws:
        sc = G.gm_build_scene(ctx, pipeline.mesh_args(w, to_device=True), stream)
        sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session, stream)
        hs.append((sc, sm, *pipeline.fixation_args(w.fixations, to_device=True)))
    prm = pipeline.params_of(ws[0], normalize=True)
    pairs = sum(G.gm_samples_info(h[1]) * w.fixations.n for h, w in zip(hs, ws))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def plain_once():
        maps = [G.gm_accumulate_fixations(h[0], h[1], *h[2:], prm, stream) for h in hs]
        return maps

    for _ in range(args.warmup):
        for m in plain_once():
            G.gm_map_free(m)
    plain_t = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        maps = plain_once()
        e1.record(stream)
        e1.synchronize()
        plain_t.append(e0.elapsed_time(e1))
        for m in maps:
            G.gm_map_free(m)
    b = G.gm_batch_create(ctx, hs, prm, stream)
    flags, tune_ms = G.gm_batch_autotune(b, stream)
    for _ in range(args.warmup):
        G.gm_batch_run(b, stream)
    torch.cuda.synchronize()
    l0 = G.gm_ctx_launches(ctx)
    batch_t = []
    clocks = ClockSampler()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.gm_batch_run(b, stream)
        e1.record(stream)
        e1.synchronize()
        batch_t.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = G.gm_ctx_launches(ctx) - l0
    info = G.gm_batch_info(b)
    buckets = G.gm_batch_buckets(b)
    ms = sum(batch_t) / len(batch_t)
    pms = sum(plain_t) / len(plain_t)
    line = {"metric": METRIC, "value": pairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched_{len(ws)}_sessions", "sessions": len(ws), "pairs_per_step": int(pairs),
                       "work_items": info["n_work_items"], "variant_flags": flags,
                       "l2": "flushed between steps (256 MiB write)", "inputs": "device-resident"},
            "plain_form": {"value": pairs / (pms * 1e-3), "ms_per_step": pms,
                           "form": "one gm_accumulate_fixations per session"},
            "batched_over_plain": pms / ms,
            "size_buckets": [{"triangles": rng, "sessions": x["sessions"], "work_items": x["work_items"],
                              "variant_flags": x["flags"], "launch_ms": x["ms"]}
                             for rng, x in zip(("< 2^14", "2^14 .. 2^17", ">= 2^17"), buckets)],
            "gpu_launches": int(launches), "clocks": clk}
    G.gm_batch_free(b)
    for sc, sm, *_ in hs:
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)
    G.gm_destroy(ctx)
    print(json.dumps(line), flush=True)


def zbuffer_arm(args):
    """The paper's own occlusion form (Sections 3.2.2 and 3.3.2: per-fixation crop frustum, z-buffer,
    +-eps depth test) beside the exact ray form, on the paper-shaped scene with head poses within
    15 degrees of the gaze. Scene and samples are built before timing; both forms include the
    fixation prep and the normalisation. One untimed run with the ray test beside the z-buffer
    counts the in-cone pairs on which the two disagree."""
    import torch
    import synth
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    torch.cuda.set_device(0)
    w = make_workload("paper_scene", args.fixations)
    fwd, up = synth.head_frames(w.fixations)
    ctx = G.gm_create(0)
    stream = torch.cuda.current_stream()
    sc = G.gm_build_scene(ctx, pipeline.mesh_args(w, to_device=True), stream)
    sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session, stream)
    fix = pipeline.fixation_args(w.fixations, to_device=True)
    d_fwd, d_up = torch.from_numpy(fwd).cuda(), torch.from_numpy(up).cuda()
    prm = pipeline.params_of(w, normalize=True)
    zbp = G.zbuffer_params(args.zb_res, 0.05, 100.0, args.zb_eps)
    ns = G.gm_samples_info(sm)
    pairs = ns * w.fixations.n
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            G.gm_map_free(fn())
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            G.gm_map_free(m)
        return sum(ts) / len(ts)

    clocks = ClockSampler()
    clocks.start()
    l0 = G.gm_ctx_launches(ctx)
    zb_ms = timed(lambda: G.gm_accumulate_zbuffer(sc, sm, *fix, prm, zbp, d_fwd, d_up, stream))
    launches = (G.gm_ctx_launches(ctx) - l0) // max(1, args.steps + args.warmup)
    clk = clocks.stop()
    ray_ms = timed(lambda: G.gm_accumulate_fixations(sc, sm, *fix, prm, stream))
    cmp = G.zbuffer_params(args.zb_res, 0.05, 100.0, args.zb_eps, compare=True)
    m = G.gm_accumulate_zbuffer(sc, sm, *fix, prm, cmp, d_fwd, d_up, stream)
    _, _, st, _ = G.gm_map_info(m)
    zs = G.gm_zbuffer_stats(m)
    G.gm_map_free(m)
    line = {"metric": METRIC, "value": pairs / (zb_ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": zb_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name + "_zbuffer", "form": "z-buffer (Sections 3.2.2, 3.3.2)",
                       "zbuffer_res": args.zb_res, "eps_m": args.zb_eps, "near_m": 0.05, "far_m": 100.0,
                       "head_pose": "forward within 15 deg of the gaze, up +y", "samples": int(ns),
                       "fixations": w.fixations.n, "pairs_per_step": int(pairs),
                       "l2": "flushed between steps (256 MiB write)", "inputs": "device-resident"},
            "ray_form": {"value": pairs / (ray_ms * 1e-3), "ms_per_step": ray_ms},
            "zbuffer_over_ray_speed": ray_ms / zb_ms,
            "flips": {"in_cone_pairs": st["in_cone"], "zbuffer_visible_ray_hidden": zs["flips_to_visible"],
                      "zbuffer_hidden_ray_visible": zs["flips_to_hidden"],
                      "rate": (zs["flips_to_visible"] + zs["flips_to_hidden"]) / max(1, st["in_cone"])},
            "raster_pairs": zs["raster_pairs"], "gpu_launches": int(launches), "clocks": clk}
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)
    G.gm_destroy(ctx)
    print(json.dumps(line), flush=True)


def dynamic_arm(args):
    """Dynamic scene: the paper-shaped scene over ten windows of 600 fixations each, one mesh (the
    torus knot) turning 3 degrees per window about the vertical axis. The timed call is
    gm_accumulate_dynamic (per window: pose + refit, samples follow, accumulation of the window's
    fixations; normalisation at the end) against gm_accumulate_fixations on the static scene with
    the same windows; the pose and follow cost is also timed on its own."""
    import torch
    import synth
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    torch.cuda.set_device(0)
    w = make_workload("paper_scene", args.fixations)
    n_win = 10
    t_end = float(w.fixations.timestamp_s.max()) + 1e-3
    w.params = synth.Params(t_begin=0.0, t_end=t_end, window_s=t_end / n_win)
    rest = np.stack([m.transform for m in w.meshes])
    xf = []
    for k in range(n_win):
        a = math.radians(3.0 * k)
        R = np.eye(4)
        R[0, 0], R[0, 2], R[2, 0], R[2, 2] = math.cos(a), math.sin(a), -math.sin(a), math.cos(a)
        wk = rest.copy()
        wk[1] = R @ rest[1]
        xf.append(wk)
    xf = np.stack(xf)
    ctx = G.gm_create(0)
    stream = torch.cuda.current_stream()
    sc = G.gm_build_scene(ctx, pipeline.mesh_args(w, to_device=True), stream, dynamic=True)
    sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session, stream)
    fix = pipeline.fixation_args(w.fixations, to_device=True)
    prm = pipeline.params_of(w, normalize=True)
    ns = G.gm_samples_info(sm)
    pairs = ns * w.fixations.n
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn, free=True):
        for _ in range(args.warmup):
            r = fn()
            if free and r is not None:
                G.gm_map_free(r)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            if free and r is not None:
                G.gm_map_free(r)
        return sum(ts) / len(ts)

    clocks = ClockSampler()
    clocks.start()
    l0 = G.gm_ctx_launches(ctx)
    dyn_ms = timed(lambda: G.gm_accumulate_dynamic(sc, sm, *fix, prm, xf, stream))
    launches = (G.gm_ctx_launches(ctx) - l0) // max(1, args.steps + args.warmup)
    clk = clocks.stop()

    def pose_all():
        for k in range(n_win):
            G.gm_scene_pose(sc, xf[k], stream)
            G.gm_samples_follow(sm, stream)
        return None

    pose_ms = timed(pose_all, free=False)
    G.gm_scene_pose(sc, rest, stream)
    G.gm_samples_follow(sm, stream)
    static_ms = timed(lambda: G.gm_accumulate_fixations(sc, sm, *fix, prm, stream))
    line = {"metric": METRIC, "value": pairs / (dyn_ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dyn_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name + "_dynamic_10win", "windows": n_win, "moving_mesh": "torus knot, 3 deg per window",
                       "samples": int(ns), "fixations": w.fixations.n, "pairs_per_step": int(pairs),
                       "l2": "flushed between steps (256 MiB write)", "inputs": "device-resident"},
            "static_same_windows_ms": static_ms, "pose_and_follow_10_windows_ms": pose_ms,
            "dynamic_over_static": dyn_ms / static_ms, "gpu_launches": int(launches), "clocks": clk}
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)
    G.gm_destroy(ctx)
    print(json.dumps(line), flush=True)


def normalize_roofline(ns: int, nonempty_windows: int, ms: float):
    """HBM roofline of the map normalisation (Section 3.2.3): every value of a non-empty window
    read and written once, 8 B per sample and window, over the kernel's CUDA-event time."""
    peak, basis = measured_hbm_peak()
    if ms <= 0:
        return None
    nbytes = 8.0 * ns * nonempty_windows
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "kernel": "k_normalize", "bytes": nbytes, "kernel_ms": ms, "peak_basis": basis,
            "work_basis": f"8 B (read + write) per sample of each of {nonempty_windows} non-empty window(s)"}


def measured_hbm_peak():
    """HBM copy rate (GB/s) from MEASURED_PEAKS.json, else a fallback of 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def sampler_arm(args):
    """Surface sampling and the export record on the paper-shaped scene: the area-weighted sampler
    (FP64 areas, fixed-point counts, int64 prefix, Philox expansion, Morton work order), the
    paper's grid sampler (Section 3.1: adaptive integer resolution, (r+1)(r+2)/2 samples per
    triangle) at the same density, and the per-sample export record (Section 3.3.3) of the Philox
    samples. Each call is timed with CUDA events (L2 flushed between steps) and its algorithmic
    bytes are set against the measured HBM copy rate."""
    import torch
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    torch.cuda.set_device(0)
    w = make_workload("paper_scene", args.fixations)
    ctx = G.gm_create(0)
    stream = torch.cuda.current_stream()
    sc = G.gm_build_scene(ctx, pipeline.mesh_args(w, to_device=True), stream)
    dens = [m.density for m in w.meshes]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn, release):
        for _ in range(args.warmup):
            release(fn())
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            release(r)
        return sum(ts) / len(ts)

    clocks = ClockSampler()
    clocks.start()
    philox_ms = timed(lambda: G.gm_sample_surface(sc, dens, w.seed, w.session, stream), G.gm_samples_free)
    grid_ms = timed(lambda: G.gm_sample_surface_grid(sc, dens, stream), G.gm_samples_free)
    sm = G.gm_sample_surface(sc, dens, w.seed, w.session, stream)
    ns = G.gm_samples_info(sm)
    gs = G.gm_sample_surface_grid(sc, dens, stream)
    ng = G.gm_samples_info(gs)
    G.gm_samples_free(gs)
    fix = pipeline.fixation_args(w.fixations, to_device=True)
    m = G.gm_accumulate_fixations(sc, sm, *fix, pipeline.params_of(w, normalize=True), stream)
    outs = dict(value=torch.empty(ns, dtype=torch.float32, device="cuda"),
                object_id=torch.empty(ns, dtype=torch.int32, device="cuda"),
                triangle=torch.empty(ns, dtype=torch.int32, device="cuda"),
                bary3=torch.empty((ns, 3), dtype=torch.float32, device="cuda"),
                local_xyz=torch.empty((ns, 3), dtype=torch.float32, device="cuda"),
                world_xyz=torch.empty((ns, 3), dtype=torch.float32, device="cuda"))
    export_ms = timed(lambda: G.gm_samples_export(sm, m, 0, stream=stream, **outs), lambda r: None)
    clk = clocks.stop()
    ntri = int(G.gm_scene_info(sc)[0])
    peak, basis = measured_hbm_peak()
    # algorithmic bytes: world triangles read (3 x float4), offsets written (int64), per sample the
    # stored record (float4 position + float2 barycentrics) and the work order (float4 + uint32)
    b_philox = 48 * ntri + 8 * (ntri + 1) + (24 + 20) * ns
    b_grid = 48 * ntri + 8 * (ntri + 1) + 4 * ntri + (24 + 20) * ng
    # export: position, barycentrics and map value read; value, object, triangle, 3 barycentrics,
    # local and world position written
    b_export = (16 + 8 + 4) * ns + (4 + 4 + 4 + 12 + 12 + 12) * ns

    def roof(bytes_, ms, kernel):
        ach = bytes_ / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "kernel": kernel, "peak_basis": basis, "algorithmic_bytes": int(bytes_)}

    line = {"metric": "surface samples/s", "value": ns / (philox_ms * 1e-3), "unit": "samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": philox_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+u32", "data": "synthetic",
            "config": {"workload": w.name + "_sampling", "triangles": ntri, "samples": int(ns),
                       "grid_samples": int(ng), "l2": "flushed between steps (256 MiB write)",
                       "inputs": "device-resident"},
            "roofline": roof(b_philox, philox_ms, "gm_sample_surface (k_tri_counts, scan, k_offsets, k_expand, work order)"),
            "grid": {"ms": grid_ms, "samples_per_s": ng / (grid_ms * 1e-3),
                     "roofline": roof(b_grid, grid_ms, "gm_sample_surface_grid")},
            "export": {"ms": export_ms, "records_per_s": ns / (export_ms * 1e-3),
                       "roofline": roof(b_export, export_ms, "gm_samples_export (k_export_record)")},
            "clocks": clk}
    G.gm_map_free(m)
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)
    G.gm_destroy(ctx)
    print(json.dumps(line), flush=True)


def field_measure(G, pipeline, ctx, stream, w, h, steps, lr, lr_min, queries, n_timed, n_warm, kernels=False,
                  batch=65536):
    """Config 3 on the map `h` of workload `w` (already accumulated and normalised): train the
    neural density field on its samples (MSE, Adam, batch 65 536, lr cosine from `lr` to `lr_min`
    over `steps` steps), then answer `queries` fresh surface points (the sampler again, seed 33, the
    density scaled up) with the field and with the plain accumulation at the same points (the
    judge). Returns the field's measurement: queries/s of both forms, the field's relative L2 error
    against the plain values, the query kernel's roofline, the training step time and the clocks
    sampled while the field kernels ran."""
    import torch
    import synth
    W, ns, st, _ = G.gm_map_info(h.map)
    xyz = torch.empty((ns, 3), dtype=torch.float32, device="cuda")
    G.gm_samples_copy(h.samples, xyz, None, None, None, stream)
    lo, hi = xyz.min(0).values.cpu().numpy(), xyz.max(0).values.cpu().numpy()
    scale = queries / ns
    qs = G.gm_sample_surface(h.scene, [m.density * scale for m in w.meshes], 33, 0, stream)
    nq = G.gm_samples_info(qs)
    qxyz = torch.empty((nq, 3), dtype=torch.float32, device="cuda")
    G.gm_samples_copy(qs, qxyz, None, None, None, stream)
    f = G.gm_field_create(ctx, lo, hi, synth.field_init(3), stream)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    t0 = time.perf_counter()
    loss = G.gm_field_train(f, h.samples, h.map, 0, steps=steps, batch=batch, lr=lr, lr_min=lr_min, seed=33,
                            stream=stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    out = torch.empty(nq, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def time_queries(kernel):
        G.gm_field_query_kernel(f, kernel)
        for _ in range(n_warm):
            G.gm_field_query(f, qxyz, nq, out, stream)
        q_t = []
        for _ in range(n_timed):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.gm_field_query(f, qxyz, nq, out, stream)
            e1.record(stream)
            e1.synchronize()
            q_t.append(e0.elapsed_time(e1))
        G.gm_sync(ctx, stream)
        return sum(q_t) / len(q_t)

    def train_step_ms(kernel, n=2000):
        # a fresh field trained by one kernel: device milliseconds per Adam step
        ft = G.gm_field_create(ctx, lo, hi, synth.field_init(3), stream)
        G.gm_field_train_kernel(ft, kernel)
        G.gm_field_train(ft, h.samples, h.map, 0, steps=n, batch=65536, lr=lr, lr_min=lr_min, seed=34,
                         stream=stream)
        ms = G.gm_field_info(ft)["train_ms"] / n
        G.gm_field_free(ft)
        return ms

    train_tc_ms = G.gm_field_info(f)["train_ms"] / steps
    extra = {}
    if kernels:
        extra["train_step_ms_mma_sync"] = train_step_ms(G.GM_FIELD_QUERY_MMA_SYNC)
        extra["query_ms_mma_sync"] = time_queries(G.GM_FIELD_QUERY_MMA_SYNC)
    field_ms = time_queries(G.GM_FIELD_QUERY_TCGEN05)   # the default kernel; `out` keeps its values
    clk = clocks.stop()
    # the reference values: plain accumulation at the query points, normalised by the training map's raw
    # maximum (a normalised map keeps it: gm_map_copy returns it)
    raw_max = G.gm_map_copy(h.map, 0, torch.empty(ns, dtype=torch.float32, device="cuda"), stream)
    prm = pipeline.params_of(w, flags=G.GM_F_TIMING, normalize=False)
    fix = pipeline.fixation_args(w.fixations, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mq = G.gm_accumulate_fixations(h.scene, qs, *fix, prm, stream)
    e1.record(stream)
    _, _, qst, _ = G.gm_map_info(mq)
    plain_ms = e0.elapsed_time(e1)
    ref = torch.empty(nq, dtype=torch.float32, device="cuda")
    G.gm_map_copy(mq, 0, ref, stream)
    ref = ref / raw_max
    err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
    # the same error on the training points themselves (the map the field was fitted to)
    tgt = torch.empty(ns, dtype=torch.float32, device="cuda")
    G.gm_map_copy(h.map, 0, tgt, stream)
    fit = torch.empty(ns, dtype=torch.float32, device="cuda")
    G.gm_field_query(f, xyz, ns, fit, stream)
    err_train = float(torch.linalg.vector_norm(fit - tgt) / torch.linalg.vector_norm(tgt))
    info = G.gm_field_info(f)
    flop_q = 2 * (4 * 64 * 64 + 64)            # hidden-layer MACs per query on the tensor cores (x2)
    train_flop = 65536 * (flop_q + 2 * 3 * 64 * 64 + 2 * 4 * 64 * 64)   # per Adam step
    peak, basis = measured_bf16_peak()
    ach = flop_q * nq / (field_ms * 1e-3) / 1e12
    roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": "k_field_query_tc", "peak_basis": basis,
            "work_basis": f"{flop_q} FLOP per query (four 64x64 BF16 layers + output)"}
    res = {"metric": "neural-field queries/s vs plain", "value": nq / (field_ms * 1e-3), "unit": "queries/s",
           "ms_per_query_batch": field_ms, "dtype": "bf16",
           "config": {"workload": f"field_on_{w.name}", "train_samples": int(ns), "queries": int(nq),
                      "fixations": w.fixations.n, "field": "64 Fourier features (10 octaves), 4x64 ReLU, softplus",
                      "train": {"steps": steps, "batch": batch, "lr": f"{lr:g} cosine to {lr_min:g}",
                                "optimizer": "Adam (0.9, 0.999)", "loss": "MSE on the max-normalised map"},
                      "l2": "flushed between query batches (256 MiB write)"},
           "rel_l2_vs_plain": err, "rel_l2_target": 1e-2, "rel_l2_on_training_points": err_train, "train_s": train_s, "train_ms_device": info["train_ms"],
           "final_batch_mse": loss,
           "plain_form": {"value": nq / (plain_ms * 1e-3), "ms": plain_ms, "pairs": int(qst["pairs"]),
                          "form": "gm_accumulate_fixations at the query points"},
           "field_over_plain": plain_ms / field_ms, "roofline": roof,
           "train_step_ms": train_tc_ms,
           "train_tflops": train_flop / (train_tc_ms * 1e-3) / 1e12,
           "train_work_basis": "65536 points x 90240 FLOP (forward 32896, dH 24576, dW 32768)",
           "clocks": clk, **extra}
    G.gm_field_free(f)
    G.gm_map_free(mq)
    G.gm_samples_free(qs)
    return res


def field_arm(args):
    """Neural density field on the paper-shaped scene as its own line (config 3 with the step
    budget and learning rate of the command line), plus the warp-level mma.sync kernels timed
    beside the tensor-core ones."""
    import torch
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    torch.cuda.set_device(0)
    w = make_workload("paper_scene", args.fixations)
    ctx = G.gm_create(0)
    stream = torch.cuda.current_stream()
    h = pipeline.run(ctx, w, stream=stream, normalize=True)
    r = field_measure(G, pipeline, ctx, stream, w, h, args.field_steps, args.field_lr,
                      args.field_lr_min if args.field_lr_min is not None else args.field_lr / 100,
                      args.queries, args.steps, args.warmup, kernels=True, batch=args.field_batch)
    line = {"metric": r.pop("metric"), "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.pop("ms_per_query_batch"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r.pop("dtype"),
            "data": "synthetic", "config": r.pop("config"), **r}
    h.free()
    G.gm_destroy(ctx)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "field":
        field_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batched":
        batched_arm(args)
        return
    if args.workload == "zbuffer":
        zbuffer_arm(args)
        return
    if args.workload == "dynamic":
        dynamic_arm(args)
        return
    if args.workload == "sampler":
        sampler_arm(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2601_07571_gb300 import build as B
    B.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline

    w = make_workload(args.workload, args.fixations)
    if args.eps_rel is not None:
        w.params.eps_rel = args.eps_rel
    ctx = G.gm_create(local)
    stream = torch.cuda.current_stream()
    dev_meshes = pipeline.mesh_args(w, to_device=True)
    dev_fix = pipeline.fixation_args(w.fixations, to_device=True)
    dens = [m.density for m in w.meshes]
    prm = pipeline.params_of(w, flags=G.GM_F_TIMING | args.flags, normalize=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    builder = {"default": None, "lbvh": G.GM_BUILD_LBVH, "ploc": G.GM_BUILD_PLOC}[args.builder]

    # one GPU: the whole path; several: the sample-sharded path (each rank its slice of the samples,
    # one all-reduce of the per-window maxima before the normalisation)
    sharded = world > 1
    from paper_2601_07571_gb300 import shard

    def step(meshes, fix):
        if sharded:
            sc, sm, mp, _, _ = shard.run_sharded(ctx, w, rank, world, dist, stream, flags=G.GM_F_TIMING | args.flags,
                                                 device="cuda", meshes=meshes, fixations=fix)
            return sc, sm, mp
        sc = G.gm_build_scene(ctx, meshes, stream, builder=builder, ploc_radius=args.ploc_radius)
        sm = G.gm_sample_surface(sc, dens, w.seed, w.session, stream)
        mp = G.gm_accumulate_fixations(sc, sm, *fix, prm, stream)
        return sc, sm, mp

    def release(h):
        sc, sm, mp = h
        G.gm_map_free(mp)
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)

    for _ in range(args.warmup):
        h = step(dev_meshes, dev_fix)
        G.gm_map_info(h[2])
        release(h)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    times, acc_ms, prep_ms, norm_ms, grid_ms, launches = [], [], [], [], [], 0
    stats = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    nonempty = 0
    for it in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = G.gm_ctx_launches(ctx)
        e0.record(stream)
        h = step(dev_meshes, dev_fix)
        e1.record(stream)
        launches += G.gm_ctx_launches(ctx) - l0
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        _, ns, stats, _ = G.gm_map_info(h[2])
        acc_ms.append(stats["accumulate_ms"])
        prep_ms.append(stats["prep_ms"])
        norm_ms.append(stats["normalize_ms"])
        grid_ms.append(stats["grid_ms"])
        if it == args.steps - 1:
            # windows the normalisation reads and writes (an empty window is skipped)
            maxima = np.empty(max(1, stats["n_windows"]), np.float32)
            G.gm_map_max(h[2], maxima)
            nonempty = int((maxima > 0).sum())
        release(h)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = reduce_max(sum(times) / len(times), dist, "cuda")
    pairs = stats["pairs"]
    # every rank's pairs (its slice of the samples x all fixations)
    total_pairs = int(reduce_sum(pairs, dist, "cuda")) if sharded else world * pairs
    value = total_pairs / (step_ms * 1e-3)

    # ---- end to end from pinned host buffers -------------------------------------------------
    host_meshes = [(torch.from_numpy(np.ascontiguousarray(v)).pin_memory(),
                    torch.from_numpy(np.ascontiguousarray(f).view(np.int32)).pin_memory(), xf, o)
                   for v, f, xf, o in pipeline.mesh_args(w)]
    host_fix = [torch.from_numpy(a).pin_memory() for a in pipeline.fixation_args(w.fixations)]
    out = torch.empty(int(stats["pairs"] // max(1, stats["n_fixations_used"])) if stats["n_fixations_used"] else 1,
                      dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * v.element_size() + f.numel() * f.element_size() for v, f, _, _ in host_meshes)
    h2d += sum(a.numel() * a.element_size() for a in host_fix)
    e2e_t = []
    for i in range(min(args.warmup, 2) + max(1, min(3, args.steps))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = step(host_meshes, host_fix)
        G.gm_map_copy(h[2], 0, out, stream)
        t1 = time.perf_counter()
        if i >= min(args.warmup, 2):
            e2e_t.append(t1 - t0)
        release(h)
    e2e_s = reduce_max(statistics.mean(e2e_t), dist, "cuda")

    # ---- roofline of the dominant kernel (the fused accumulate) ------------------------------
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    acc = sum(acc_ms) / len(acc_ms)
    gms = sum(grid_ms) / len(grid_ms)
    peak = n_sm * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    grid_on = stats["grid_chunks"] > 0
    # executed FP32 work, from the kernel's own counters: the cone tests it evaluated (pairs of warp
    # tiles whose sphere the cone misses are skipped), the Gaussian and compensated sum of every
    # in-cone pair, and the occlusion tests (BVH: two slab tests per node visit; eye grid: one
    # depth compare per list entry) plus one watertight test per triangle tested
    per_visit = FP32_INSTR_PER_ENTRY if grid_on else FP32_INSTR_PER_NODE
    executed = (FP32_INSTR_PER_PAIR * stats["pairs_tested"] + FP32_INSTR_PER_INCONE * stats["in_cone"]
                + per_visit * stats["nodes_visited"] + FP32_INSTR_PER_TRI * stats["tris_tested"])
    achieved = executed / (acc * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s (FP32)", "frac": achieved / peak,
            "traffic": recorded_traffic(w.name, args.flags, args.builder,
                                        args.ploc_radius in (0, 8) and args.eps_rel is None),
            "kernel": "k_accumulate" + ("<eye grid>" if grid_on else "<BVH>"),
            "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ_NOMINAL:.0f} MHz (nominal)",
            "work_basis": (f"executed FP32 instructions from the kernel's counters: {FP32_INSTR_PER_PAIR} per cone test "
                           f"evaluated ({stats['pairs_tested']:.4g} of {stats['pairs']:.4g} nominal pairs), "
                           f"{FP32_INSTR_PER_INCONE} per in-cone pair (Gaussian + compensated sum), {per_visit} per "
                           + ("eye-grid entry read" if grid_on else "BVH node visit")
                           + f", {FP32_INSTR_PER_TRI} per triangle test"),
            "kernel_ms": acc}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (n_sm * FP32_LANES_PER_SM * clk["sm_mhz"] * 1e6 / 1e12)
    # the nominal-pair figure of earlier lines: 18 instructions for every sample x fixation pair
    nominal = FP32_INSTR_PER_PAIR * pairs / (acc * 1e-3) / 1e12
    roof["nominal_pairs"] = {"achieved": nominal, "frac": nominal / peak,
                             "work_basis": f"{FP32_INSTR_PER_PAIR} FP32 instructions per nominal pair"}

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "triangles": w.n_tris, "samples": int(ns if not sharded else
                                                                                   reduce_sum(ns, dist, "cuda")),
                       "fixations": w.fixations.n, "pairs_per_step": int(pairs),
                       "l2": "flushed between steps (256 MiB write)", "inputs": "device-resident",
                       "parallelism": (f"samples{world}: each rank a contiguous slice of the samples, "
                                       "all-reduce MAX of the per-window maxima") if sharded else "single",
                       "accumulate_flags": args.flags, "builder": args.builder, "eps_rel": w.params.eps_rel,
                       "ploc_radius": args.ploc_radius or 8},
            "stages_ms": {"accumulate": acc, "eye_grid": gms, "fixation_prep": sum(prep_ms) / len(prep_ms),
                          "normalize": sum(norm_ms) / len(norm_ms),
                          "build_and_sample": step_ms - acc - gms - sum(prep_ms) / len(prep_ms)
                          - sum(norm_ms) / len(norm_ms)},
            "occlusion": (f"eye grid {64 if args.flags & G.GM_F_GRID64 else 128}^2 cells per fixation, "
                          f"{stats['grid_chunks']} chunk(s), {stats['grid_launches']} launch(es)") if grid_on else "BVH",
            "in_cone_pairs": int(stats["in_cone"]), "visible_pairs": int(stats["visible"]),
            "cone_tests_evaluated": int(stats["pairs_tested"]),
            "rays_per_s": stats["in_cone"] / (acc * 1e-3),
            ("grid_entries_per_ray" if grid_on else "nodes_per_ray"): stats["nodes_visited"] / max(1, stats["in_cone"]),
            "tris_per_ray": stats["tris_tested"] / max(1, stats["in_cone"]),
            "roofline": roof,
            "normalize_roofline": normalize_roofline(ns, nonempty, sum(norm_ms) / len(norm_ms)),
            "e2e": {"value": total_pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(out.numel() * 4), "ms_per_step": e2e_s * 1e3},
            "gpu_launches": int(launches), "clocks": clk}
    if rank == 0 and world == 1 and not args.no_field and args.workload == "paper_scene" and not args.fixations:
        # the metric's second half: config 3 on this workload's map, with its own clock record
        hf = pipeline.run(ctx, w, stream=stream, normalize=True)
        line["field"] = field_measure(G, pipeline, ctx, stream, w, hf, args.field_steps, args.field_lr,
                                      args.field_lr_min if args.field_lr_min is not None else args.field_lr / 100,
                                      args.queries, args.steps, args.warmup)
        hf.free()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        dt, p, n = calibrated_oracle(w, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": p / dt, "unit": "pairs/s", "cores": min(cores, n), "kind": "oracle",
                                "sample": f"{n} evenly strided samples x all {w.fixations.n} fixations, "
                                          f"whole-scene transform/areas/counts included ({dt:.1f} s)"}
    G.gm_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
