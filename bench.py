#!/usr/bin/env python
"""Frame-throughput benchmark of the HashPoint hot path on B300.

One step = one frame of the whole hot path (table build + window search +
primary-surface sampling + IDW aggregation + MLP decode + compositing) for
every pixel of an 800x800 view of the 1M-point object scene (6 nested or
overlapping ellipsoids, boxes and tori, 32-d features, r = 0.005, K = 8,
n = 8, MLP 32-128-128-128-4), cycling through 8 cameras on a radius-4
sphere.  Inputs are seeded synthetic data; L2 is flushed (256 MB write)
before every step, outside the per-step CUDA-event timing.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (same workload, bounded ray samples per step).
Multi-GPU (torchrun): independent replicas, one view stream per rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2404_14044_b300 import scenes  # noqa: E402

METRIC = "rays/s (build+search+sample+render) at 800x800, 1M pts"
N_VIEWS = 8
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hashpoint", choices=["hashpoint", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-proposal", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--points", type=int, default=1_000_000)
    ap.add_argument("--res", type=int, default=800)
    return ap.parse_args()


def workload(n_points, res):
    pts = scenes.object_points(n_points, 0)
    feats = scenes.random_features(n_points, 32, 1)
    params = scenes.Params(radius_mode=scenes.RADIUS_FIXED, r=0.005, K=8, n_max=8)
    dims = [32, 128, 128, 128, 4]
    mlp = scenes.random_mlp(dims, 0, sigma_bias=1.5 / params.r)
    cams = scenes.random_sphere_cameras(N_VIEWS, 4.0, 0, width=res, height=res)
    return pts, feats, params, dims, mlp, cams


def config_dict(n_points, res, extra=None):
    d = {"workload": f"objects_{res}: {n_points} points on 6 closed shapes, {res}x{res} rays per frame, "
                     f"8 views on a radius-4 sphere, r=0.005, K=8, n=8, MLP 32-128-128-128-4, FP32",
         "rays_per_step": res * res, "points": n_points, "views": N_VIEWS,
         "l2": "flushed before every step (256 MB write), flush outside the per-step event timing",
         "neighbour_lists": "left in the search workspace, read there by the decode (hp_samples.nbr NULL)"}
    if extra:
        d.update(extra)
    return d


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------- algorithmic traffic/flops

def algorithmic(kernel, N, Nv, P, R, S, K, F, dims, U, tensor_decode=True, packed_lists=False):
    """Algorithmic bytes (or FLOPs for the decode) of one launch of each kernel.
    The search's bytes are charged to its walk (k_search_select); the pick
    and the warp-per-ray kernel work on what the walk left.  packed_lists:
    the pack also copies the neighbour lists (the frame leaves them in the
    search's slots and writes each sample's slot index instead)."""
    mlp_flops = 2 * S * sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1))
    table = {
        "k_project_count": ("hbm", 12 * N + 8 * N + 8 * P),
        "k_scan": ("hbm", 8 * (P + 1)),
        "k_scatter": ("hbm", 12 * N + 8 * N + 4 * Nv + 16 * Nv + 4 * Nv),
        "k_bucket_sort": ("hbm", 8 * P + 32 * Nv),
        "k_search_select": ("hbm", 4 * P + 16 * Nv + 12 * R + (12 + 8 * K) * S),
        "k_search_pick": ("hbm", 0),
        "k_search_select_wide": ("hbm", 0),
        "k_pack_samples": ("hbm", 4 * R + 8 * (R + 1) + (12 + 8 * K) * S + (16 + 8 * K) * S if packed_lists
                           else 4 * R + 8 * (R + 1) + 16 * S + 20 * S),
        "k_aggregate_decode": ("tensor" if tensor_decode else "alu", mlp_flops),
        "k_composite": ("hbm", 28 * R + 20 * S),
        # the pass-start clears (table counts, then the search's per-pixel
        # counts), averaged over the frame's two launches
        "k_clear": ("hbm", (4 * (P + 1) + 4 * R) // 2),
        "k_ray_table": ("hbm", 16 * R),
    }
    return table.get(kernel, ("hbm", 0))


# DRAM bytes (read + write) of one launch, from one ncu capture of
# `bench.py --steps 1 --warmup 1` at 800x800 (first view), keyed by the
# profiler's kernel name.  Each entry carries the SHA-256 of the sources the
# kernel is compiled from when it was captured; once those change the figure
# no longer describes the kernel and the roofline reports traffic = null; so
# does a run of another workload (points, resolution).
NCU_TRAFFIC_WORKLOAD = (1_000_000, 800)
NCU_TRAFFIC = {
    # the search stage's time (k_search_select) covers the point-major pass
    # (k_search_splat) and the selection launch: their bytes are summed
    "k_search_select": {"bytes": 52944640 + 38285568 + 116661248 + 33304576,
                        "sources": ('hp_search.cu', 'hp_common.cuh', 'hp_kernels.cuh'),
                        "sha256": "6a84c8f727c389c5b3ab049c6bf856b9dd57ffbb256b3ca96722245deab79ddd"},
    "k_pack_samples": {"bytes": 17950208 + 2560,
                       "sources": ('hp_search.cu', 'hp_common.cuh', 'hp_kernels.cuh'),
                       "sha256": "6a84c8f727c389c5b3ab049c6bf856b9dd57ffbb256b3ca96722245deab79ddd"},
    "k_aggregate_decode": {"bytes": 88080896 + 4325120,
                           "sources": ('hp_decode_tc.cu', 'hp_tc.cuh', 'hp_common.cuh', 'hp_kernels.cuh'),
                           "sha256": "0a123ecbffd333950c33ce5a5e6e1308eedac9dc0835800c41604c2dcbbcddc2"},
}


def sources_sha256(names):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2404_14044_b300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(kernel, workload=NCU_TRAFFIC_WORKLOAD):
    e = NCU_TRAFFIC.get(kernel)
    if tuple(workload) != NCU_TRAFFIC_WORKLOAD or e is None or e["sha256"] is None or sources_sha256(e["sources"]) != e["sha256"]:
        return None
    return e["bytes"]


def agg_gather_bytes(S, K, F, U):
    return 8 * K * S + 4 * F * U + 16 * S


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak_tflops(sm_count=148, clock_mhz=2032.0):
    # 128 FP32 FMA lanes per SM, 2 FLOP per FMA
    return sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ CPU side

def oracle_frame_seconds(pts, feats, params, dims, mlp, cam, nthreads=None):
    """Seconds the oracle takes for one whole frame (its own table build and
    every ray of the view, OpenMP over rays on ``nthreads`` host threads)."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.render(pts, feats, cam, params, dims, mlp, nthreads=nthreads)
    return time.perf_counter() - t0, nthreads


def oracle_views_rate(pts, feats, params, dims, mlp, cams):
    """Oracle rays/s over whole frames of the given views (one frame each)."""
    secs = []
    cores = 1
    for cam in cams:
        t, cores = oracle_frame_seconds(pts, feats, params, dims, mlp, cam)
        secs.append(t)
    R = cams[0].width * cams[0].height
    return R * len(cams) / sum(secs), secs, cores


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores,
    rendering the same whole frames (views cycled in the same order) that the
    GPU arm times; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pts, feats, params, dims, mlp, cams = workload(args.points, args.res)
    R = args.res * args.res
    for w in range(args.warmup):
        oracle_frame_seconds(pts, feats, params, dims, mlp, cams[w % N_VIEWS])
    frames = []
    cores = 1
    t_run = time.perf_counter()
    for k in range(args.steps):
        t, cores = oracle_frame_seconds(pts, feats, params, dims, mlp, cams[k % N_VIEWS])
        frames.append(t)
    t_run = time.perf_counter() - t_run
    t_frame = float(np.mean(frames))
    value = R / t_frame
    sample = (f"per step: one whole frame -- the oracle builds the table of {args.points} points and renders all "
              f"{R} rays (OpenMP over rays); views cycled as in the GPU arm")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_frame, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.points, args.res, {"parallelism": "cpu oracle, rank 0 only"}),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s_timed_region": t_run}
    print(json.dumps(line), flush=True)


# ------------------------------------------------- learned proposal + BF16

def psnr(a, b):
    import torch
    mse = torch.mean((a.double() - b.double()) ** 2).item()
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def proposal_section(hp, H, pts_np, feats_np, params, dims, mlp_np, cam, train_cams, steps, dev, flush):
    """Learned depth-interval proposal + BF16 decode against the plain FP32
    path: train the proposal on the plain search's intervals of 64 views;
    fit features for 200 steps to a target image (plain FP32 render of view 0
    with a second feature draw; that path matches the FP64 oracle to 1e-4)
    with the library's render + backward; then compare speed and PSNR against
    that target, and judge the proposal's misses with the plain search."""
    import torch
    R = cam.width * cam.height
    t = lambda a: torch.from_numpy(a).to(dev)
    pts, mlp = t(pts_np), t(mlp_np)
    # 1) proposal training on the training views (8 passes)
    n_train = len(train_cams)
    state = H.ProposalState(dev, seed=0)
    t0 = time.perf_counter()
    for it in range(8 * n_train):
        tc = train_cams[it % n_train]
        hp.build_table(pts, tc, params.r)
        plain = hp.search_sample(None, params.K, params.n_max)
        hp.proposal_train_step(None, plain, state, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    l = state.loss.cpu().numpy()
    # 2) target and fitted features (the evaluation view)
    tgt, _, _ = hp.render(pts, t(scenes.random_features(len(pts_np), 32, 7)), cam, dims, mlp)
    tgt = tgt.clone()
    feats = t(feats_np).clone()
    opt = torch.optim.Adam([feats], lr=2e-2)
    rng = np.random.default_rng(0)
    for it in range(200):
        rays = t(np.sort(rng.choice(R, 8192, replace=False)).astype(np.int32))
        rgb, wsum, smp = hp.render(pts, feats, cam, dims, mlp, rays=rays)
        g = (2.0 / rgb.numel()) * (rgb - tgt[rays.long()])
        gf, _ = hp.aggregate_render_backward(smp, pts, feats, dims, mlp, g, want_points=False)
        feats.grad = gf
        opt.step()
    # 3) full frames: plain FP32 vs proposal + BF16 (and each change alone)
    def run(mode, decode, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n + 2):
            flush.zero_()
            if k >= 2:
                ev[k - 2][0].record()
            hp.build_table(pts, cam, params.r)
            if mode == "plain":
                smp = hp.search_sample(None, params.K, params.n_max)
            else:
                iv = hp.proposal_infer(None, state.bf16)
                smp = hp.search_sample_proposal(None, params.K, params.n_max, iv, fallback_count=fb)
            rgb, wsum = hp.aggregate_render(smp, feats, dims, mlp, decode=decode)
            if k >= 2:
                ev[k - 2][1].record()
        torch.cuda.synchronize()
        # the median frame: these auxiliary comparisons launch from Python
        # frame by frame, and one host-side stall inside a frame would
        # otherwise move a 20-frame mean by a third
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        return ms, rgb.clone(), smp
    n = max(5, min(steps, 20))
    fb = torch.zeros(1, dtype=torch.int32, device=dev)
    kernels = {}
    for mode, dec in (("plain", H.DECODE_FP32), ("proposal", H.DECODE_BF16)):
        hp.profile_start(256)
        run(mode, dec, 1)
        kernels[mode] = {k: round(v[0] / max(v[1], 1), 5) for k, v in hp.profile_stop().items() if v[1]}
    ms_plain, rgb_plain, smp_plain = run("plain", H.DECODE_FP32, n)
    ms_bf16, rgb_bf16, _ = run("plain", H.DECODE_BF16, n)
    ms_prop, rgb_prop32, _ = run("proposal", H.DECODE_FP32, n)
    ms_both, rgb_both, smp_prop = run("proposal", H.DECODE_BF16, n)
    code, detail = hp.status()
    if code != 0:
        raise SystemExit(f"device status after proposal pass: {H.status_string(code)} ({detail})")
    # misses judged by the plain search: rays whose samples differ
    a, b = smp_plain.packed(R), smp_prop.packed(R)
    oa, ob = a["sample_offset"].numpy(), b["sample_offset"].numpy()
    sa, sb = a["src"].numpy(), b["src"].numpy()
    hit = np.nonzero(a["n_s"].numpy() > 0)[0]
    miss = float(np.mean([not np.array_equal(sa[oa[i]:oa[i + 1]], sb[ob[i]:ob[i + 1]]) for i in hit]))
    p_plain, p_both = psnr(rgb_plain, tgt), psnr(rgb_both, tgt)
    return {"value": R / (ms_both / 1e3), "unit": "rays/s", "ms_per_step": ms_both,
            "speedup_vs_plain_fp32": ms_plain / ms_both,
            "ms_plain_fp32": ms_plain, "ms_plain_bf16": ms_bf16, "ms_proposal_fp32": ms_prop,
            "psnr_plain_fp32_db": p_plain, "psnr_proposal_bf16_db": p_both, "psnr_drop_db": p_plain - p_both,
            "psnr_bf16_vs_plain_db": psnr(rgb_bf16, rgb_plain), "psnr_proposal_vs_plain_db": psnr(rgb_prop32, rgb_plain),
            "miss_rate": miss, "fallback_rays": int(fb.item()), "per_kernel_ms": kernels, "train": {"views": n_train, "steps": 8 * n_train, "seconds": t_train,
                                         "final_loss": float(l[0] / max(l[1], 1))},
            "protocol": "target = plain FP32 render of view 0 with a second feature draw (matches the FP64 "
                        "oracle to 1e-4); features fitted 200 Adam steps (8192 rays/step) with "
                        "hp_aggregate_render_backward; proposal frames: hp_proposal_infer then "
                        "hp_search_sample_proposal; misses = hit rays whose sample sources differ from the "
                        "plain search; ms = median of the frames' device times (L2 flushed before each)"}


# ------------------------------------------------------ training step (f2)

def train_section(hp, H, pts_np, feats_np, params, dims, mlp_np, cams, steps, dev, flush):
    """Training step with differentiation: 4 views of the object scene x 4096
    random pixels per view; per view the forward (table build, search on the
    listed rays, aggregate + render) and hp_aggregate_render_backward with
    respect to the point features and positions, for the MSE loss against a
    target image (the forward with a second feature draw).  The views are
    independent until the gradient sums (the backward accumulates them with
    atomics), so each runs on its own stream with its own library context;
    a step forks from and joins the current stream.  Rays/s = 16,384 rays per
    step over the step's device time."""
    import torch
    t = lambda a: torch.from_numpy(a).to(dev)
    pts, feats, mlp = t(pts_np), t(feats_np), t(mlp_np)
    W, Hh = cams[0].width, cams[0].height
    n_rays = 4096
    views = cams[:4]
    rays = [t(np.sort(scenes.random_rays(W, Hh, n_rays, v)).astype(np.int32)) for v in range(len(views))]
    feats2 = t(scenes.random_features(len(pts_np), 32, 7))
    tgt = []
    for v, cam in enumerate(views):
        rgb, _, _ = hp.render(pts, feats2, cam, dims, mlp, rays=rays[v])
        tgt.append(rgb.clone())
    gf = torch.zeros_like(feats)
    gp = torch.zeros_like(pts)
    smp = H.SampleBuffers.allocate(n_rays, params.K, params.n_max, dev)
    ctxs = [hp] + [H.HashPoint(params, dev) for _ in range(len(views) - 1)]
    smps = [smp] + [H.SampleBuffers.allocate(n_rays, params.K, params.n_max, dev) for _ in range(len(views) - 1)]
    streams = [torch.cuda.Stream() for _ in views]

    def view_pass(c, v, cam, sm):
        c.build_table(pts, cam, params.r)
        c.search_sample(rays[v], params.K, params.n_max, out=sm)
        rgb, wsum = c.aggregate_render(sm, feats, dims, mlp)
        d = rgb - tgt[v]
        c.aggregate_render_backward(sm, pts, feats, dims, mlp, (2.0 / d.numel()) * d, grad_feats=gf,
                                    grad_points=gp)
        return (d * d).mean()

    def step():
        # the views on their own streams and contexts, forked from and joined
        # to the current stream
        main = torch.cuda.current_stream()
        gf.zero_()
        gp.zero_()
        fork = torch.cuda.Event()
        fork.record(main)
        loss, joins = [], []
        for v, cam in enumerate(views):
            streams[v].wait_event(fork)
            with torch.cuda.stream(streams[v]):
                loss.append(view_pass(ctxs[v], v, cam, smps[v]))
                e = torch.cuda.Event()
                e.record(streams[v])
                joins.append(e)
        for e in joins:
            main.wait_event(e)
        return loss

    def step_serial():
        # one context, one stream: the per-kernel profile of a step
        gf.zero_()
        gp.zero_()
        return [view_pass(hp, v, cam, smp) for v, cam in enumerate(views)]

    for _ in range(3):
        step()
    n = max(5, min(steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush.zero_()
        ev[k][0].record()
        loss = step()
        ev[k][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / n
    hp.profile_start(256)
    step_serial()
    prof = hp.profile_stop()
    for c in ctxs:
        code, detail = c.status()
        if code != 0:
            raise SystemExit(f"device status after training pass: {H.status_string(code)} ({detail})")
    for c in ctxs[1:]:
        c.close()
    per_kernel = {k: round(v[0] / max(v[1], 1), 5) for k, v in prof.items() if v[1]}
    launches = {k: v[1] for k, v in prof.items() if v[1]}
    # the last view's samples: the backward's work per launch
    S = int(smp.sample_offset[n_rays].item())
    sigma_io = sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1))
    flops = 4 * S * sigma_io              # forward recompute + back-propagation through the MLP (FP32 SIMT)
    ms_dec = prof["k_decode_bwd"][0] / max(prof["k_decode_bwd"][1], 1)
    peak = fp32_peak_tflops(148, 2032.0)
    achieved = flops / (ms_dec / 1e3) / 1e12
    return {"value": len(views) * n_rays / (ms / 1e3), "unit": "rays/s", "ms_per_step": ms,
            "rays_per_step": len(views) * n_rays, "views": len(views), "loss": float(sum(x.item() for x in loss)),
            "per_kernel_ms": per_kernel, "launches_per_step": launches,
            "roofline_decode_bwd": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                    "frac": achieved / peak, "flops_per_launch": flops, "samples_per_launch": S,
                                    "peak_source": "derived: 148 SMs x 128 FP32 FMA lanes x 2 FLOP x 2032 MHz"},
            "protocol": "per view: hp_build_table, hp_search_sample on 4096 random pixels, hp_aggregate_render, "
                        "MSE loss against the forward with a second feature draw, "
                        "hp_aggregate_render_backward (features and positions); the 4 views on 4 streams with "
                        "one library context each, the gradients summed by the backward's atomics; L2 flushed "
                        "before each step; per_kernel_ms from a serial step on one context"}


# ------------------------------------------------------------------ GPU side

def rank_views(n_views, rank, world):
    """View indices a rank renders, in order: rank r takes views r, r + N,
    r + 2N, ... (mod the view count), so every rank does the same per-step
    work (weak scaling) and no data crosses ranks."""
    return [(rank + i * world) % n_views for i in range(n_views)]


def job_rate(local_ms, rays_per_step, steps, world, device):
    """Whole-job throughput: the slowest rank's time (max over ranks) against
    the rays all ranks processed.  Returns (rays/s, max ms)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * rays_per_step * steps / (ms / 1e3), ms


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2404_14044_b300 import hashpoint as H

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    pts_np, feats_np, params, dims, mlp_np, cams = workload(args.points, args.res)
    R = args.res * args.res
    N = len(pts_np)
    pts = torch.from_numpy(pts_np).to(dev)
    feats = torch.from_numpy(feats_np).to(dev)
    mlp = torch.from_numpy(mlp_np).to(dev)
    hp = H.HashPoint(params, dev)
    hp.reserve(cams[0], params.r, N, R, params.n_max)
    # the frame's samples without packed neighbour lists: the search leaves
    # them in its workspace and the decode reads them there (hp_samples.nbr NULL)
    smp = H.SampleBuffers.allocate(R, params.K, params.n_max, dev, lists=False)
    rgb = torch.empty(R, 3, dtype=torch.float32, device=dev)
    wsum = torch.empty(R, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    views = [cams[i] for i in rank_views(N_VIEWS, rank, world)]

    def frame(cam, p=pts):
        hp.build_table(p, cam, params.r)
        hp.search_sample(None, params.K, params.n_max, out=smp)
        hp.aggregate_render(smp, feats, dims, mlp, rgb, wsum)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(args.warmup):
        flush.zero_()
        frame(views[w % N_VIEWS])
    code, detail = hp.status()
    if code != 0:
        raise SystemExit(f"device status after warm-up: {H.status_string(code)} ({detail})")

    # ---- timed pass: K frames, per-step CUDA events (flush outside)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        frame(views[k % N_VIEWS])
        ev[k][1].record()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    code, detail = hp.status()
    if code != 0:
        raise SystemExit(f"device status after timed pass: {H.status_string(code)} ({detail})")
    value, dev_ms_max = job_rate(dev_ms, R, args.steps, world, dev)

    # per-frame sizes (last view) for the algorithmic traffic
    S = int(smp.sample_offset[R].item())
    tb = hp.table_info()
    P = int(tb.n_buckets)
    nv_t = torch.empty(1, dtype=torch.int32, device=dev)
    Nv = int(hp.table()["start"][-1].item())
    # distinct points gathered (U): the last view searched once more into
    # buffers that keep the packed lists (outside the timed region)
    smp_l = H.SampleBuffers.allocate(R, params.K, params.n_max, dev)
    hp.search_sample(None, params.K, params.n_max, out=smp_l)
    U = int(torch.unique(smp_l.nbr[:S][smp_l.nbr[:S] >= 0]).numel())
    del smp_l

    # ---- profiled pass: per-kernel device time on the launching stream
    hp.profile_start(64 * args.steps)
    Ss, Nvs = [], []
    for k in range(args.steps):
        flush.zero_()
        frame(views[k % N_VIEWS])
    prof = hp.profile_stop()
    launches = sum(nk for _, _, nk in prof.values())      # CUDA kernels, not timed brackets
    per_kernel = {name: {"ms_total": ms, "launches": n, "kernels": nk, "ms_avg": ms / n if n else 0.0}
                  for name, (ms, n, nk) in prof.items()}
    # the dominant kernel: the largest measured time among those with an
    # algorithmic count
    dom = max((kv for kv in prof.items() if algorithmic(kv[0], 1, 1, 1, 1, 1, 1, 32, dims, 1)[1] > 0),
              key=lambda kv: kv[1][0])[0]
    pk = peaks()

    def roofline_of(kernel):
        bound, units = algorithmic(kernel, N, Nv, P, R, S, params.K, 32, dims, U)
        ms = per_kernel[kernel]["ms_avg"]
        if bound == "tensor":
            # FP32-accurate decode: each product costs three FP16 MMAs (split
            # operands); the achieved figure counts the FP32 MLP's FLOPs once
            peak = pk.get("bf16_tflops", 1800.0)
            achieved = units / (ms / 1e3) / 1e12
            return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ncu_traffic(kernel, (args.points, args.res)),
                    "peak_source": ("MEASURED_PEAKS.json bf16_tflops (burst; FP16 dense rate equals BF16)"
                                    if "bf16_tflops" in pk else "fallback 1800 TFLOP/s"),
                    "tensor_flops_executed_per_launch": 3 * units,
                    "gather_bytes_per_launch": agg_gather_bytes(S, params.K, 32, U)}
        if bound == "alu":
            peak = fp32_peak_tflops(148, 2032.0)
            achieved = units / (ms / 1e3) / 1e12
            return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ncu_traffic(kernel, (args.points, args.res)),
                    "peak_source": "derived: 148 SMs x 128 FP32 FMA lanes x 2 FLOP x 2032 MHz",
                    "gather_bytes_per_launch": agg_gather_bytes(S, params.K, 32, U)}
        peak = pk.get("hbm_gbs", 6400.0)
        achieved = units / (ms / 1e3) / 1e9
        return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(kernel, (args.points, args.res)),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in pk else "fallback 6400 GB/s"}

    roof = roofline_of(dom)
    roof["others"] = {k: {x: roofline_of(k)[x] for x in ("bound", "achieved", "unit", "frac", "traffic")}
                      for k in ("k_search_select", "k_aggregate_decode", "k_pack_samples", "k_bucket_sort")
                      if k != dom and per_kernel.get(k, {}).get("launches")}

    # ---- end to end: per-frame point positions H2D from pinned memory, image
    # D2H, through the C-ABI.  The copies run on a second stream, double
    # buffered, so frame k+1's upload and frame k-1's download overlap frame
    # k's compute (the ordering is kept with events).
    e2e = None
    if not args.no_e2e:
        host_pts = torch.from_numpy(pts_np).pin_memory()
        host_rgb = [torch.empty(R, 3, dtype=torch.float32).pin_memory() for _ in range(2)]
        host_ws = [torch.empty(R, dtype=torch.float32).pin_memory() for _ in range(2)]
        dev_pts = [torch.empty_like(pts) for _ in range(2)]
        dev_rgb = [torch.empty(R, 3, dtype=torch.float32, device=dev) for _ in range(2)]
        dev_ws = [torch.empty(R, dtype=torch.float32, device=dev) for _ in range(2)]
        comp = torch.cuda.Stream()          # compute (the library's calls)
        cps = torch.cuda.Stream()           # uploads (host -> device)
        dps = torch.cuda.Stream()           # downloads (device -> host): the other PCIe direction
        ev = lambda: torch.cuda.Event()
        up_done = [ev(), ev()]        # H2D of buffer b finished
        frame_done = [ev(), ev()]     # compute of the frame in buffer b finished
        down_done = [ev(), ev()]      # D2H of buffer b finished

        def run(n):
            with torch.cuda.stream(cps):
                dev_pts[0].copy_(host_pts, non_blocking=True)
                up_done[0].record(cps)
            for k in range(n):
                b = k & 1
                comp.wait_event(up_done[b])
                if k >= 2:
                    comp.wait_event(down_done[b])          # rgb[b] read back before it is rewritten
                with torch.cuda.stream(comp):
                    hp.build_table(dev_pts[b], views[k % N_VIEWS], params.r)
                    smp_k = hp.search_sample(None, params.K, params.n_max, out=smp)
                    hp.aggregate_render(smp_k, feats, dims, mlp, dev_rgb[b], dev_ws[b])
                frame_done[b].record(comp)
                if k + 1 < n:
                    with torch.cuda.stream(cps):
                        if k >= 1:
                            cps.wait_event(frame_done[b ^ 1])  # frame k-1 done with dev_pts[b^1]
                        dev_pts[b ^ 1].copy_(host_pts, non_blocking=True)
                        up_done[b ^ 1].record(cps)
                with torch.cuda.stream(dps):
                    dps.wait_event(frame_done[b])
                    host_rgb[b].copy_(dev_rgb[b], non_blocking=True)
                    host_ws[b].copy_(dev_ws[b], non_blocking=True)
                    down_done[b].record(dps)
            comp.wait_stream(cps)
            comp.wait_stream(dps)

        run(max(2, args.warmup))
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        cps.wait_event(e0)
        dps.wait_event(e0)
        run(args.steps)
        e1.record(comp)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        e2e = {"value": job_rate(e2e_ms, R, args.steps, world, dev)[0], "unit": "rays/s",
               "h2d_bytes_per_step": int(host_pts.numel() * 4), "d2h_bytes_per_step": int(R * 16),
               "what": "per step: point positions H2D (pinned), table+search+render through the C-ABI, "
                       "rgb+weight-sum D2H (pinned); uploads and downloads on their own streams (both PCIe "
                       "directions at once), double buffered and overlapped with the neighbouring frames' "
                       "compute; features and MLP weights resident"}
    code, detail = hp.status()
    if code != 0:
        raise SystemExit(f"device status after e2e pass: {H.status_string(code)} ({detail})")

    # per-frame statistics of the last timed view (outside the timed region)
    ns_last = smp.n_s[:R]
    cc_last = smp.cand_count[:R]
    stats = {"n_s_histogram": [int(x) for x in torch.bincount(ns_last.long(), minlength=params.n_max + 1).tolist()],
             "rays_over_candidate_cap": int((cc_last > params.cand_cap).sum().item()),
             "rays_over_lane_column_40": int((cc_last > 40).sum().item()),
             "sample_capacity_overflow": bool(S > smp.capacity),
             "candidates_per_ray_mean": float(cc_last.float().mean().item())}

    train = None
    if rank == 0 and world == 1 and not args.no_train:
        train = train_section(hp, H, pts_np, feats_np, params, dims, mlp_np, views, args.steps, dev, flush)

    prop = None
    if rank == 0 and world == 1 and not args.no_proposal:
        train_cams = scenes.random_sphere_cameras(64, 4.0, 100, width=args.res, height=args.res)
        prop = proposal_section(hp, H, pts_np, feats_np, params, dims, mlp_np, views[0], train_cams, args.steps,
                                dev, flush)
        prop["workload"] = f"objects_{args.res} (view 0, held out of the 64 training views)"
        # the forward-facing scene at 1008 x 756 (cone radius, K = 16): trained on
        # 64 jittered forward views, evaluated on the reference view
        fw = scenes.forward_1008()
        hpf = H.HashPoint(fw.params, dev)
        fcams = scenes.forward_cameras(65, 4)
        prop_fw = proposal_section(hpf, H, fw.points, fw.feats, fw.params, fw.mlp_dims, fw.mlp_params, fcams[0],
                                   fcams[1:], args.steps, dev, flush)
        prop_fw["workload"] = ("forward_1008: 1.5M points, 1008x756, cone radius (rho 2), K=16, n=8, reference view "
                               "held out of 64 jittered forward views")
        hpf.close()
        prop = {"objects": prop, "forward_1008": prop_fw}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, cores = oracle_views_rate(pts_np, feats_np, params, dims, mlp_np, cams)
        cpu = {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle",
               "sample": f"one whole frame of each of the {len(cams)} views (table of {N} points + all {R} rays, "
                         f"OpenMP over rays), {sum(secs):.2f} s in total"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(args.points, args.res,
                                      {"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                       "samples_last_frame": S, "visible_points_last_frame": Nv,
                                       "buckets": P, "unique_points_gathered": U}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "proposal_bf16": prop, "train_step": train, "frame_stats": stats,
                "clocks": clk, "per_kernel_ms": {k: round(v["ms_avg"], 5) for k, v in per_kernel.items()},
                "wall_s_timed_region": t_wall}
        print(json.dumps(line), flush=True)
    hp.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
