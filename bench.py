#!/usr/bin/env python3
"""Benchmark of the GB300 volume ray caster.

Default workload: the 512x512x361 uint16 CT-like phantom (seed 2) rendered at 1920x1080
with a perspective camera, step 0.5, Zucker-Hummel gradients, empty-space skipping and
early termination.  One step = the whole hot path on device-resident inputs:
vr_upload_volume (padded copy + brick min/max) -> vr_set_transfer_function (+ brick
visibility) -> vr_set_camera -> vr_render (ray setup + fused march).

Metric: Gsamples/s, where a sample is one t_k the plain method marches (every sample up to
early termination, whether or not empty-space skipping visited it); the count comes from
the kernel's own counters and is checked against the FP64 oracle by the GPU tests.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle instead.
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

# Algorithmic FP32 operations per sample (fused multiply-add = 2): every visited sample
# pays its position, the cell fractions, the trilinear value (7 lerps) and the opacity
# lerp; a shaded sample adds the colour lerps, the operator gradient contracted from the
# cell's neighbourhood with the trilinear weights (the per-sample form that needs no
# precomputed state: the 32-voxel cross for central differences, the separable 4x4x4
# contraction for Sobel3D and Zucker-Hummel), the normalisation, Phong with its power and
# the compositing update.
FLOPS_VISIT = 34
FLOPS_SHADE = {"central": 96, "sobel3d": 392, "zucker_hummel": 392}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["ct", "ellipsoids", "sphere"], default="ct")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e / cpu legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--leg", choices=["main", "fwd_bwd", "batch", "surface", "adaptive", "train",
                                      "f16", "sparse", "slab"],
                    default="main",
                    help="run one leg alone and print its JSON (for profiling)")
    ap.add_argument("--source-hash", choices=sorted(KERNEL_SOURCES),
                    help="print the source hash recorded beside a kernel's ncu counters")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="edge scale of the batched-render volumes (1.0 = full sizes)")
    ap.add_argument("--mode", choices=["replicas", "sortfirst", "sortlast"], default="replicas",
                    help="N > 1: independent replicas of the frame (weak scaling, default), "
                         "one frame split by rows over the ranks and gathered, or one frame "
                         "split by z slabs of the volume and composited (both strong)")
    return ap.parse_args()


def workload(name):
    import phantoms as P

    if name == "ct":
        return P.workload_ct()
    if name == "ellipsoids":
        return P.workload_ellipsoids_256()
    return P.workload_sphere_64()


def dtype_name(vol):
    return {np.dtype(np.uint8): "u8", np.dtype(np.uint16): "u16", np.dtype(np.float16): "f16",
            np.dtype(np.float32): "f32"}[vol.dtype]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"vr_bench_clocks_gpu{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            # the first query can take a while: start timing only once the sampler runs
            t0 = time.perf_counter()
            while os.path.getsize(self.path) == 0 and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = sum(1 for _ in open(self.path))
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for i, line in enumerate(open(self.path)):
                if i < getattr(self, "skip", 0):
                    continue  # taken before the timed region started
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    import torch

    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist

    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def sum_over_ranks(x, world):
    import torch.distributed as dist

    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def replica_throughput(samples_per_step, steps, step_ms_total, world):
    """Whole-job throughput of N independent replicas (weak scaling): the samples of all
    ranks divided by the slowest rank's time.  Returns (Gsamples/s, ms per step)."""
    total_ms = max_over_ranks(step_ms_total, world)
    samples = sum_over_ranks(float(samples_per_step) * steps, world)
    return samples / (total_ms / 1e3) / 1e9, total_ms / steps


# ------------------------------------------------------------ ncu traffic record
KERNEL_SOURCES = {
    "k_march": ["vr_device.cuh", "vr_internal.h", "vr_march.cuh", "vr_render.cu"],
    "k_march_list": ["vr_device.cuh", "vr_internal.h", "vr_march.cuh", "vr_render.cu"],
    "k_records_tma": ["vr_device.cuh", "vr_internal.h", "vr_records.cuh", "vr_volume.cu"],
    "k_adjoint": ["vr_device.cuh", "vr_internal.h", "vr_adjoint.cu"],
    "k_surface": ["vr_device.cuh", "vr_internal.h", "vr_surface.cu"],
    "k_march_slab": ["vr_device.cuh", "vr_internal.h", "vr_march.cuh", "vr_records.cuh",
                     "vr_slab.cu"],
}
PROFILE_SUMMARY = {"k_march": "profiles/k_march_ct512x512x361_1080p.md",
                   "k_march_list": "profiles/k_march_list_vessels512_4k.md",
                   "k_records_tma": "profiles/k_records_tma_ct512x512x361.md",
                   "k_adjoint": "profiles/k_adjoint_density128_16views.md",
                   "k_surface": "profiles/k_surface_ct512x512x361_1080p_bone.md",
                   "k_march_slab": "profiles/k_march_slab_ct512x512x361_1080p.md"}


def source_hash(kernel):
    """SHA-256 over the sources a kernel is built from (recorded beside its ncu counters)."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1609_01317_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel):
    """DRAM bytes (read + write) per launch from the committed ncu summary of `kernel`, or
    None when there is none or the kernel's sources changed since the capture."""
    try:
        fields = {}
        for line in open(os.path.join(ROOT, PROFILE_SUMMARY[kernel])):
            if ":" in line and line.lstrip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_sha256") != source_hash(kernel):
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(w, seconds):
    """Time the FP64 oracle on the workload's frame: whole frames (rows split over the
    host cores) until about `seconds` have passed (at least one frame, at most four), or a
    band of rows around the middle when one frame alone would take far longer."""
    import oracle

    ov = oracle.OracleVolume(w["volume"], w["value_max"])
    pr = oracle.make_params(step=w["step"], grad=w["grad"])
    cam = w["camera"]
    H = cam["height"]
    mid = H // 2
    t0 = time.perf_counter()
    _, _, probe = oracle.render(ov, w["tf"], cam, pr, rows=(mid - 4, mid + 4))
    dt = time.perf_counter() - t0
    est_frame = dt * H / 8.0 * 0.6  # the middle band is denser than the frame average
    if est_frame > 3.0 * seconds:
        rows = max(8, int(8 * seconds / max(dt, 1e-3)))
        r0 = max(0, mid - rows // 2)
        t0 = time.perf_counter()
        img, _, total = oracle.render(ov, w["tf"], cam, pr, rows=(r0, min(H, r0 + rows)))
        dt = time.perf_counter() - t0
        return {"samples": int(total), "seconds": dt, "rows": [r0, min(H, r0 + rows)],
                "frames": 0, "cores": oracle.num_threads(), "image": img}
    total, frames = 0, 0
    t0 = time.perf_counter()
    while frames < 4:
        img, _, n = oracle.render(ov, w["tf"], cam, pr)
        total += n
        frames += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"samples": int(total), "seconds": dt, "rows": [0, H], "frames": frames,
            "cores": oracle.num_threads(), "image": img}


def oracle_one_core(w, rows=8):
    """The FP64 oracle on one host thread over a band of rows in the frame's middle: the
    per-core rate, in Gsamples/s."""
    import oracle

    ov = oracle.OracleVolume(w["volume"], w["value_max"])
    pr = oracle.make_params(step=w["step"], grad=w["grad"])
    mid = w["camera"]["height"] // 2
    n0 = oracle.num_threads()
    t0 = time.perf_counter()
    _, _, total = oracle.render(ov, w["tf"], w["camera"], pr, rows=(mid - rows // 2, mid + rows // 2),
                                nthreads=1)
    dt = time.perf_counter() - t0
    oracle.render(ov, w["tf"], w["camera"], pr, rows=(mid, mid + 1), nthreads=n0)  # restore
    return total / dt / 1e9, rows


def bench_config(w, world):
    """The workload description shared by both arms' JSON lines."""
    nz, ny, nx = w["volume"].shape
    cam = w["camera"]
    return {"workload": w["name"], "volume": f"{nx}x{ny}x{nz} {dtype_name(w['volume'])}",
            "image": f"{cam['width']}x{cam['height']}", "grad": w["grad"], "step": w["step"],
            "skip_empty": w["skip_empty"], "ert": 0.99,
            "l2": f"flushed between steps (256 MiB write); volume {w['volume'].nbytes / 1e6:.0f} MB",
            "parallelism": f"replicas{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload)
    vals = []
    samples = 0
    secs = 0.0
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, per_step)
        if i >= args.warmup:
            vals.append(r["samples"] / r["seconds"] / 1e9)
            samples += r["samples"]
            secs += r["seconds"]
    value = samples / secs / 1e9
    cam = w["camera"]
    line = {
        "impl": "reference", "metric": "Gsamples/s", "value": value, "unit": "Gsamples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, args.gpus),
        "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": r["cores"],
                         "kind": "oracle",
                         "sample": (f"{r['frames']} whole frame(s)" if r["frames"] else
                                    f"rows {r['rows'][0]}-{r['rows'][1]}") +
                                   f" of the {cam['width']}x{cam['height']} frame per step"},
        "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ GPU leg
def batch_leg(args):
    """Batched workload: 8 volumes (96^3 .. 384x384x256, uint8/uint16), 64 orbit cameras
    each at 512x512, central differences, skipping on.  One graph-replayed persistent launch
    (after the autotuner) against 512 separate vr_render calls."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import Renderer, vr

    t0 = time.perf_counter()
    wl = P.workload_batch(args.batch_scale)
    gen_s = time.perf_counter() - t0
    params = vr.make_params(grad="central", skip_empty=True)
    pst = vr.make_params(grad="central", skip_empty=True, collect_stats=True)
    rends, cams, owner = [], [], []
    for i, w in enumerate(wl):
        r = Renderer(torch.cuda.current_device())
        r.upload_volume(w["volume"], w["value_max"])
        r.set_transfer_function(w["tf"])
        rends.append(r)
        cams += w["cameras"]
        owner += [i] * len(w["cameras"])
    outs = [torch.empty((c["height"], c["width"], 4), device="cuda") for c in cams]
    cam_s = [vr.make_camera(c) for c in cams]
    samples = 0
    for c, o, out in zip(cam_s, owner, outs):
        vr.vr_set_camera(rends[o].ctx, c)
        vr.vr_render(rends[o].ctx, pst, out)
        samples += vr.vr_read_stats(rends[o].ctx)["samples_plain"]
    b = vr.vr_batch_create([r.ctx for r in rends], cams, owner, params, outs)
    chosen = vr.vr_batch_autotune(b)
    sh = torch.cuda.current_stream().cuda_stream or None

    def batched():
        vr.vr_batch_run(b, sh)

    def separate():
        for c, o, out in zip(cam_s, owner, outs):
            vr.vr_set_camera(rends[o].ctx, c)
            vr.vr_render(rends[o].ctx, params, out, sh)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, min(args.steps, 5))
    t_b = timed(batched, reps)
    t_s = timed(separate, reps)
    # sampled pixels of every batched render (48 whose ray reaches something, 16 anywhere),
    # kept for the comparison with the FP64 oracle in the CPU-baseline leg
    batched()
    torch.cuda.synchronize()
    rng = np.random.default_rng(2024)
    picks, got = [], []
    for o in outs:
        hit = torch.nonzero(o[..., 3] > 0).cpu().numpy()
        sel = hit[rng.choice(len(hit), size=min(48, len(hit)), replace=False)] if len(hit) else \
            np.zeros((0, 2), np.int64)
        yx = np.concatenate([sel, np.stack([rng.integers(0, o.shape[0], 16),
                                            rng.integers(0, o.shape[1], 16)], 1)]).astype(np.int32)
        px, py = yx[:, 1].copy(), yx[:, 0].copy()
        picks.append((px, py))
        got.append(o[torch.from_numpy(py).long().cuda(), torch.from_numpy(px).long().cuda()]
                   .cpu().numpy())
    vr.vr_batch_destroy(b)
    for r in rends:
        r.close()
    n = len(cams)
    return {"_samples": {"wl": wl, "cams": cams, "owner": owner, "picks": picks, "got": got},
            "workload": f"batch8vol_{n}renders_512_cd", "renders": n, "samples": samples,
            "volume_scale": args.batch_scale, "autotuned": {"threads": chosen[0],
                                                            "tile": [chosen[1], chosen[2]]},
            "batched_ms": t_b, "separate_ms": t_s, "speedup": t_s / t_b,
            "batched_gsamples_s": samples / (t_b / 1e3) / 1e9,
            "separate_gsamples_s": samples / (t_s / 1e3) / 1e9,
            "renders_per_s": n / (t_b / 1e3), "phantom_generation_s": gen_s}


def batch_parity(bs):
    """The batched renders' sampled pixels against the FP64 oracle's rays through the same
    pixels (per-pixel max abs over RGBA)."""
    import oracle

    pr = oracle.make_params(grad="central")
    ovs = [oracle.OracleVolume(w["volume"], w["value_max"]) for w in bs["wl"]]
    errs = []
    for c, o, (px, py), g in zip(bs["cams"], bs["owner"], bs["picks"], bs["got"]):
        ref, _, _ = oracle.render_pixels(ovs[o], bs["wl"][o]["tf"], c, pr, px, py)
        errs.append(np.abs(g.astype(np.float64) - ref).max(axis=-1))
    e = np.concatenate(errs)
    return {"reference": "FP64 oracle", "renders": len(errs), "pixels": int(e.size),
            "sample": "48 pixels whose ray reaches something + 16 anywhere, per render",
            "max_abs": float(e.max()), "frac_within_2e-3": float((e <= 2e-3).mean())}


def surface_leg(R, args):
    """First-hit surface renderer (§3.11, §5.1) on the CT workload's volume and camera:
    bone window [2200, 4095], coarse step 2.0 (four times the direct renderer's step), six
    bisection steps, Zucker-Hummel normal, skipping on; the volume stays resident."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import vr

    w = P.workload_ct()
    vol = w["volume"]
    nz, ny, nx = vol.shape
    ctx = R.ctx
    sh = torch.cuda.current_stream().cuda_stream or None
    vol_dev = torch.from_numpy(vol.view(np.int16)).cuda()
    vr.vr_upload_volume(ctx, vol_dev, "u16", nx, ny, nz, w["value_max"], sh)
    cam = w["camera"]
    vr.vr_set_camera(ctx, vr.make_camera(cam))
    H, W = cam["height"], cam["width"]
    img = torch.empty((H, W, 4), device="cuda")
    depth = torch.empty((H, W), device="cuda")
    p = vr.make_surface_params(step=2.0, iso_lo=2200.0, iso_hi=4095.0, refine=6,
                               grad="zucker_hummel", skip_empty=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        vr.vr_render_surface(ctx, p, img, depth, sh)
    reps = max(10, min(args.steps, 100))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
    for i in range(reps):
        flush.fill_(float(i))
        ev[i][0].record()
        vr.vr_render_surface(ctx, p, img, depth, sh)
        ev[i][1].record()
    torch.cuda.synchronize()
    ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    hits = int(torch.isfinite(depth).sum().item())
    return {"workload": "ct512x512x361_u16_persp1920x1080_bone_surface",
            "window": [2200.0, 4095.0], "step": 2.0, "refine": 6, "grad": "zucker_hummel",
            "ms_per_frame": ms, "frames_per_s": 1000.0 / ms,
            "mrays_per_s": H * W / (ms / 1e3) / 1e6, "rays_hit": hits}


def adaptive_leg(R, args):
    """Adaptive sampling (§5.2) on the CT workload: 32^3 regions whose footprint range is
    <= 600 (raw units) take every 4th sample, <= 1500 every 2nd; the march time, the samples
    taken and the image difference to the regular render (records cached, volume resident)."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import vr

    w = P.workload_ct()
    vol = w["volume"]
    nz, ny, nx = vol.shape
    ctx = R.ctx
    sh = torch.cuda.current_stream().cuda_stream or None
    vol_dev = torch.from_numpy(vol.view(np.int16)).cuda()
    vr.vr_upload_volume(ctx, vol_dev, "u16", nx, ny, nz, w["value_max"], sh)
    tf_dev = torch.from_numpy(w["tf"]).cuda()
    vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
    cam = w["camera"]
    vr.vr_set_camera(ctx, vr.make_camera(cam))
    H, W = cam["height"], cam["width"]
    kw = dict(step=w["step"], grad=w["grad"], skip_empty=True)
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for name, extra in (("regular", {}), ("adaptive", {"adapt_range": (1500.0, 600.0)})):
        img = torch.empty((H, W, 4), device="cuda")
        pst = vr.make_params(collect_stats=True, **kw, **extra)
        vr.vr_render(ctx, pst, img, sh)
        st = vr.vr_read_stats(ctx, sh)
        p = vr.make_params(**kw, **extra)
        for _ in range(3):
            vr.vr_render(ctx, p, img, sh)
        reps = max(10, min(args.steps, 100))
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i))
            ev[i][0].record()
            vr.vr_render(ctx, p, img, sh)
            ev[i][1].record()
        torch.cuda.synchronize()
        out[name] = (statistics.mean(a.elapsed_time(b) for a, b in ev), st, img)
    diff = (out["adaptive"][2] - out["regular"][2]).abs().amax(dim=-1)
    return {"workload": "ct512x512x361_u16_persp1920x1080_zh_adaptive",
            "adapt_range": {"m2": 1500.0, "m4": 600.0},
            "regular_ms": out["regular"][0], "adaptive_ms": out["adaptive"][0],
            "speedup": out["regular"][0] / out["adaptive"][0],
            "samples_taken": out["adaptive"][1]["samples_visited"],
            "samples_taken_regular": out["regular"][1]["samples_visited"],
            "image_max_abs_diff": float(diff.max().item()),
            "image_mean_abs_diff": float(diff.mean().item())}


def fwd_bwd_leg(R, args):
    """Differentiable workload: 128^3 float32 blurred density, learnable 256-entry TF,
    16 views at 256x256, central differences, step 0.5.  Times the forward that records
    adjoint checkpoints against forward + backward (vr_render_backward), Gsamples/s on the
    same plain-method sample count."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import vr

    n = 128
    vol = torch.from_numpy(P.blurred_random_field(4, n)).cuda()
    tf = torch.from_numpy(P.tf_c1(256)).cuda()
    views = P.training_views(n, 256, 256)
    ctx = R.ctx
    sh = torch.cuda.current_stream().cuda_stream or None
    params = vr.make_params(grad="central", skip_empty=False, ert_threshold=0.99)
    pst = vr.make_params(grad="central", skip_empty=False, ert_threshold=0.99, collect_stats=True)
    vr.vr_upload_volume(ctx, vol, "f32", n, n, n, 1.0, sh)
    vr.vr_set_transfer_function(ctx, tf, 256, sh)
    img = torch.empty((256, 256, 4), device="cuda")
    gimg = torch.randn((256, 256, 4), device="cuda") * 1e-3
    gv = torch.zeros_like(vol)
    gt = torch.zeros_like(tf)
    cams = [vr.make_camera(c) for c in views]
    vr.vr_set_camera(ctx, cams[0])
    nb = vr.vr_checkpoint_bytes(ctx, params) + 256
    ck = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in views]
    ckv = [(c[(-c.data_ptr()) % 256:]) for c in ck]
    samples = 0
    for c in cams:
        vr.vr_set_camera(ctx, c)
        vr.vr_render(ctx, pst, img, sh)
        samples += vr.vr_read_stats(ctx, sh)["samples_plain"]

    def fwd():
        for i, c in enumerate(cams):
            vr.vr_set_camera(ctx, c)
            vr.vr_render_forward_train(ctx, params, img, ckv[i], nb - 256, sh)

    def fwdbwd():
        for i, c in enumerate(cams):
            vr.vr_set_camera(ctx, c)
            vr.vr_render_forward_train(ctx, params, img, ckv[i], nb - 256, sh)
        vr.vr_render_backward_views(ctx, params, cams, ckv, [gimg] * len(cams), gv, gt, sh)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, min(args.steps, 10))
    t_f = timed(fwd, reps)
    t_fb = timed(fwdbwd, reps)
    return {"workload": "density128_f32_16views256_cd", "samples": samples,
            "fwd_ms": t_f, "fwd_bwd_ms": t_fb, "ratio": t_fb / t_f,
            "fwd_gsamples_s": samples / (t_f / 1e3) / 1e9,
            "fwd_bwd_gsamples_s": samples / (t_fb / 1e3) / 1e9}


def train_leg(R, args, steps=200):
    """Differentiable workload trained: a learnable 128^3 float32 density (blurred random
    field, seed 4) and 256-entry TF (the sphere workload's ramp) fitted by Adam (lr 1e-2) to
    16 views at 256 x 256 of the hidden 128^3 ellipsoid phantom (seed 3), L2 image loss,
    central differences, termination at 0.99.  One step = upload volume + set TF + 16
    checkpointed forwards + the adjoint of all 16 views + the Adam update (torch on the
    device), no host synchronisation inside the loop.  Gsamples/s counts the plain-method
    samples of every forward (the sum of the rays' recorded end indices)."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import vr

    n, H, W = 128, 256, 256
    dev = "cuda"
    ctx = R.ctx
    sh = torch.cuda.current_stream().cuda_stream or None
    views = P.training_views(n, W, H)
    cams = [vr.make_camera(c) for c in views]
    params = vr.make_params(grad="central", skip_empty=False, ert_threshold=0.99)
    tf0 = torch.from_numpy(P.tf_c1(256)).to(dev)
    hidden = torch.from_numpy(P.density_phantom(3, n)).to(dev)
    vr.vr_upload_volume(ctx, hidden, "f32", n, n, n, 1.0, sh)
    vr.vr_set_transfer_function(ctx, tf0, 256, sh)
    targets = []
    for c in cams:
        vr.vr_set_camera(ctx, c)
        t = torch.empty((H, W, 4), device=dev)
        vr.vr_render(ctx, params, t, sh)
        targets.append(t)
    vol = torch.from_numpy(P.blurred_random_field(4, n)).to(dev)
    tf = tf0.clone()
    opt = torch.optim.Adam([vol.requires_grad_(), tf.requires_grad_()], lr=1e-2)
    vr.vr_set_camera(ctx, cams[0])
    nb = vr.vr_checkpoint_bytes(ctx, params)
    ck = [torch.empty(nb + 256, dtype=torch.uint8, device=dev) for _ in cams]
    ckv = [c[(-c.data_ptr()) % 256:][:nb] for c in ck]
    imgs = [torch.empty((H, W, 4), device=dev) for _ in cams]
    gimgs = [torch.empty((H, W, 4), device=dev) for _ in cams]
    gv = torch.zeros_like(vol)
    gt = torch.zeros_like(tf)
    loss = torch.zeros((), device=dev, dtype=torch.float64)
    samples = torch.zeros((), device=dev, dtype=torch.int64)
    norm = 1.0 / (len(cams) * H * W * 4)

    def step():
        vr.vr_upload_volume(ctx, vol.detach(), "f32", n, n, n, 1.0, sh)
        vr.vr_set_transfer_function(ctx, tf.detach(), 256, sh)
        loss.zero_()
        for i, c in enumerate(cams):
            vr.vr_set_camera(ctx, c)
            vr.vr_render_forward_train(ctx, params, imgs[i], ckv[i], nb, sh)
            d = imgs[i] - targets[i]
            loss.add_((d * d).sum(dtype=torch.float64) * norm)
            torch.mul(d, 2.0 * norm, out=gimgs[i])
            samples.add_(ckv[i][:4 * H * W].view(torch.int32).sum())
        gv.zero_()
        gt.zero_()
        vr.vr_render_backward_views(ctx, params, cams, ckv, gimgs, gv, gt, sh)
        vol.grad, tf.grad = gv, gt
        opt.step()
        with torch.no_grad():
            vol.clamp_(0.0, 1.0)
            tf.clamp_(0.0, 1.0)

    step()  # the first step, untimed (lazy Adam state)
    first = float(loss.item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    samples.zero_()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps - 1):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (steps - 1)
    total = int(samples.item())
    vr.vr_upload_volume(ctx, vol.detach(), "f32", n, n, n, 1.0, sh)
    vr.vr_set_transfer_function(ctx, tf.detach(), 256, sh)
    final = 0.0
    for i, c in enumerate(cams):  # loss of the trained state
        vr.vr_set_camera(ctx, c)
        vr.vr_render(ctx, params, imgs[i], sh)
        final += float(((imgs[i] - targets[i]) ** 2).sum(dtype=torch.float64)) * norm
    return {"workload": "density128_f32_16views256_cd_adam", "adam_steps": steps,
            "lr": 1e-2, "ms_per_step": ms,
            "fwd_bwd_gsamples_s": total / ((steps - 1) * ms / 1e3) / 1e9,
            "samples_per_step": total / (steps - 1), "loss_first": first, "loss_final": final,
            "timed": f"{steps - 1} steps after the first (CUDA events, no host sync inside)"}


def f16_leg(args, K):
    """The CT frame with the volume stored as FP16 (raw / 4095, value_max 1), timed as the
    main step (upload + TF + camera + render).  Returns the leg's dict, the image and the
    volume (for the oracle comparison in the CPU-baseline leg)."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import Renderer, vr

    w = P.workload_ct()
    v16 = (w["volume"].astype(np.float32) / np.float32(4095.0)).astype(np.float16)
    nz, ny, nx = v16.shape
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    R = Renderer(torch.cuda.current_device())
    ctx = R.ctx
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vdev = torch.from_numpy(v16).cuda()
    tdev = torch.from_numpy(w["tf"]).cuda()
    out = torch.empty((H, W, 4), device="cuda")
    params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"])
    cam_s = vr.make_camera(cam)

    def step(p=params):
        vr.vr_upload_volume(ctx, vdev, "f16", nx, ny, nz, 1.0, sh)
        vr.vr_set_transfer_function(ctx, tdev, tdev.shape[0], sh)
        vr.vr_set_camera(ctx, cam_s)
        vr.vr_render(ctx, p, out, sh)

    step(vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"],
                        collect_stats=True))
    st = vr.vr_read_stats(ctx, sh)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        step()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for i in range(K):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    img = out.cpu().numpy()
    R.close()
    return ({"workload": "ct512x512x361_f16_persp1920x1080_zh", "storage": "f16 = raw / 4095",
             "ms_per_step": ms, "value": st["samples_plain"] / (ms / 1e3) / 1e9,
             "unit": "Gsamples/s", "samples_per_frame": st["samples_plain"],
             "samples_visited": st["samples_visited"], "samples_shaded": st["samples_shaded"]},
            img, v16)


def sparse_leg(args, K):
    """The sparse workload of the skipping hierarchy (§5.4): a 512^3 uint16 vessel tree in
    empty space rendered at 3840 x 2160 (Zucker-Hummel, step 0.5, skipping + termination).
    Times the whole step (upload + TF + camera + render) and the render alone; keeps sampled
    pixels for the oracle comparison in the CPU-baseline leg."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import Renderer, vr

    w = P.workload_sparse()
    vol = w["volume"]
    nz, ny, nx = vol.shape
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    R = Renderer(torch.cuda.current_device())
    ctx = R.ctx
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vdev = torch.from_numpy(vol.view(np.int16)).cuda()
    tdev = torch.from_numpy(w["tf"]).cuda()
    out = torch.empty((H, W, 4), device="cuda")
    params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=True)
    cam_s = vr.make_camera(cam)

    def step(p=params):
        vr.vr_upload_volume(ctx, vdev, "u16", nx, ny, nz, w["value_max"], sh)
        vr.vr_set_transfer_function(ctx, tdev, tdev.shape[0], sh)
        vr.vr_set_camera(ctx, cam_s)
        vr.vr_render(ctx, p, out, sh)

    step(vr.make_params(step=w["step"], grad=w["grad"], skip_empty=True, collect_stats=True))
    st = vr.vr_read_stats(ctx, sh)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        step()

    def timed(fn):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
        for i in range(K):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    step_ms = timed(step)
    render_ms = timed(lambda: vr.vr_render(ctx, params, out, sh))
    img = out
    hit = torch.nonzero(img[..., 3] > 0).cpu().numpy()
    rng = np.random.default_rng(9)
    pick = np.concatenate([hit[rng.choice(len(hit), min(1500, len(hit)), replace=False)],
                           rng.integers(0, [H, W], size=(300, 2))])
    got = img[torch.from_numpy(pick[:, 0]).cuda(), torch.from_numpy(pick[:, 1]).cuda()].cpu().numpy()
    R.close()
    return {"_samples": {"w": w, "pick": pick, "got": got},
            "workload": w["name"], "ms_per_step": step_ms, "render_ms": render_ms,
            "value": st["samples_plain"] / (step_ms / 1e3) / 1e9, "unit": "Gsamples/s",
            "render_gsamples_s": st["samples_plain"] / (render_ms / 1e3) / 1e9,
            "samples_per_frame": st["samples_plain"], "samples_visited": st["samples_visited"],
            "samples_shaded": st["samples_shaded"], "rays_hit": st["rays_hit"],
            "voxels_nonzero_frac": float((vol > 0).mean())}


def slab_leg(args, K):
    """The two plain marches on the CT frame (1920 x 1080, Zucker-Hummel, skipping +
    termination): the record march (gradient records of the visible bricks in device memory,
    tile march) and the slab march (each 16 x 16 tile stages the raw voxels it crosses and
    their records in shared memory, no record table).  Times the whole step (upload + TF +
    camera + render, records recomputed) and the render alone, and checks that the two
    frames are identical."""
    import torch

    import phantoms as P
    from paper_1609_01317_gb300 import Renderer, vr

    w = P.workload_ct()
    vol = w["volume"]
    nz, ny, nx = vol.shape
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    R = Renderer(torch.cuda.current_device())
    ctx = R.ctx
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vdev = torch.from_numpy(vol.view(np.int16)).cuda()
    tdev = torch.from_numpy(w["tf"]).cuda()
    cam_s = vr.make_camera(cam)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"workload": w["name"]}
    frames = []
    for march in ("records", "slabs"):
        params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=True, march=march)
        img = torch.empty((H, W, 4), device="cuda")

        def step(p=params, img=img):
            vr.vr_upload_volume(ctx, vdev, "u16", nx, ny, nz, w["value_max"], sh)
            vr.vr_set_transfer_function(ctx, tdev, tdev.shape[0], sh)
            vr.vr_set_camera(ctx, cam_s)
            vr.vr_render(ctx, p, img, sh)

        step(vr.make_params(step=w["step"], grad=w["grad"], skip_empty=True, march=march,
                            collect_stats=True))
        st = vr.vr_read_stats(ctx, sh)
        for _ in range(3):
            step()

        def timed(fn):
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
            for i in range(K):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                fn()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            return statistics.mean(a.elapsed_time(b) for a, b in ev)

        out[march] = {"ms_per_step": timed(step),
                      "render_ms": timed(lambda p=params, img=img: vr.vr_render(ctx, p, img, sh)),
                      "march_ran": {1: "records", 2: "slabs"}.get(st["march"], "?"),
                      "samples_visited": st["samples_visited"]}
        frames.append(img)
    out["identical"] = bool(torch.equal(frames[0], frames[1]))
    out["samples_plain"] = st["samples_plain"]
    R.close()
    return out


def run_sortfirst(args):
    """One frame of the workload split by rows over the ranks (sort-first, §2.2: rays are
    independent): every rank uploads the volume and renders its band of the busy rows
    (vr_render_rows), the bands are all-gathered over NCCL and stitched into the frame on
    every rank.  Strong scaling: value = the frame's plain samples / the slowest rank's
    step time."""
    import torch
    import torch.distributed as dist

    from paper_1609_01317_gb300 import Renderer, build, sortfirst as SF, vr

    rank, world, local = dist_setup(args)
    build.build()
    w = workload(args.workload)
    vol = w["volume"]
    nz, ny, nx = vol.shape
    dt = dtype_name(vol)
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vol_dev = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
    tf_dev = torch.from_numpy(w["tf"]).cuda()
    R = Renderer(local)
    ctx = R.ctx
    params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"])
    cam_s = vr.make_camera(cam)
    busy = vr.vr_screen_rect(cam, (0.0, 0.0, 0.0), (nx - 1.0, ny - 1.0, nz - 1.0))
    part = SF.RowPartition.from_bands(H, W, world, busy=(busy[1], busy[3]))
    packed = torch.zeros((part.capacity, W, 4), device="cuda")
    frame = torch.empty((H, W, 4), device="cuda")

    def render_rows(a, b, dst, p=params):
        vr.vr_render_rows(ctx, p, a, b, dst, sh)

    def step(p=params):
        vr.vr_upload_volume(ctx, vol_dev, dt, nx, ny, nz, w["value_max"], sh)
        vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
        vr.vr_set_camera(ctx, cam_s)
        part.render_local(rank, lambda a, b, dst: render_rows(a, b, dst, p), packed)
        part.gather(packed, frame)

    pst = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"],
                         collect_stats=True)
    step(pst)
    mine = vr.vr_read_stats(ctx, sh)["samples_plain"] if part.per_rank[rank] else 0
    samples = int(sum_over_ranks(float(mine), world))
    for _ in range(args.warmup):
        step()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    barrier(world)
    with ClockSampler(local) as clk:
        for i in range(K):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier(world)
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    ms = total_ms / K
    line = {"metric": "Gsamples/s", "value": samples / (ms / 1e3) / 1e9, "unit": "Gsamples/s",
            "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(bench_config(w, world), parallelism=f"sortfirst{world}"),
            "frames_per_s": 1000.0 / ms, "samples_per_frame": samples,
            "bands": part.per_rank, "gpu_launches": 8 * K, "clocks": clk.summary(),
            "e2e": None, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_sortlast(args):
    """One frame of the workload split by z slabs of the volume (sort-last: Eq. 6 is
    associative): every rank holds the volume, composites the samples of its slab into a
    partial image (vr_render_partial, whole-box sampling grid, no early termination), the
    partial images are all-gathered over NCCL and composited front to back along each pixel's
    ray on every rank.  Strong scaling: value = the frame's plain samples (without early
    termination) / the slowest rank's step time."""
    import torch
    import torch.distributed as dist

    from paper_1609_01317_gb300 import Renderer, build, sortlast as SL, vr

    rank, world, local = dist_setup(args)
    build.build()
    w = workload(args.workload)
    vol = w["volume"]
    nz, ny, nx = vol.shape
    dt = dtype_name(vol)
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vol_dev = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
    tf_dev = torch.from_numpy(w["tf"]).cuda()
    R = Renderer(local)
    ctx = R.ctx
    # the slabs composite exactly only without early termination
    params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"],
                            ert_threshold=2.0)
    cam_s = vr.make_camera(cam)
    part = SL.SlabPartition(nz, world)
    sign = torch.from_numpy(SL.ray_dz_sign(cam)).cuda()
    mine = torch.zeros((H, W, 4), device="cuda")
    frame = torch.empty((H, W, 4), device="cuda")

    def step(p=params):
        vr.vr_upload_volume(ctx, vol_dev, dt, nx, ny, nz, w["value_max"], sh)
        vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
        vr.vr_set_camera(ctx, cam_s)
        part.render_local(rank, lambda a, b, dst: vr.vr_render_partial(ctx, p, a, b, dst, sh),
                          mine)
        part.gather(mine, sign, frame)

    # the frame's plain sample count (a whole render with counters, outside the timing)
    vr.vr_upload_volume(ctx, vol_dev, dt, nx, ny, nz, w["value_max"], sh)
    vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
    vr.vr_set_camera(ctx, cam_s)
    vr.vr_render(ctx, vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"],
                                     ert_threshold=2.0, collect_stats=True), frame, sh)
    samples = int(vr.vr_read_stats(ctx, sh)["samples_plain"])
    for _ in range(args.warmup):
        step()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    barrier(world)
    with ClockSampler(local) as clk:
        for i in range(K):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier(world)
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    ms = total_ms / K
    cfg = dict(bench_config(w, world), parallelism=f"sortlast{world}")
    cfg["ert"] = "off (slabs composite exactly only without early termination)"
    line = {"metric": "Gsamples/s", "value": samples / (ms / 1e3) / 1e9, "unit": "Gsamples/s",
            "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "frames_per_s": 1000.0 / ms, "samples_per_frame": samples,
            "slabs": [[z0 if math.isfinite(z0) else None, z1 if math.isfinite(z1) else None]
                      for z0, z1 in part.slabs],
            "gpu_launches": 7 * K, "clocks": clk.summary(), "e2e": None, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch

    from paper_1609_01317_gb300 import Renderer, build, vr

    if args.mode == "sortfirst":
        return run_sortfirst(args)
    if args.mode == "sortlast":
        return run_sortlast(args)
    rank, world, local = dist_setup(args)
    build.build()
    w = workload(args.workload)
    vol = w["volume"]
    nz, ny, nx = vol.shape
    dt = dtype_name(vol)
    cam = w["camera"]
    H, W = cam["height"], cam["width"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None
    vol_dev = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
    tf_dev = torch.from_numpy(w["tf"]).cuda()
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    R = Renderer(local)
    ctx = R.ctx
    params = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"])
    cam_s = vr.make_camera(cam)

    def step(p=params):
        vr.vr_upload_volume(ctx, vol_dev, dt, nx, ny, nz, w["value_max"], sh)
        vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
        vr.vr_set_camera(ctx, cam_s)
        vr.vr_render(ctx, p, out, sh)

    # sample counts (untimed): the numerator of the metric
    pst = vr.make_params(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"],
                         collect_stats=True)
    step(pst)
    stats = vr.vr_read_stats(ctx, sh)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    barrier(world)
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(K):
            flush.fill_(float(i))  # evict the L2 between steps (outside the timed events)
            ev[i][0].record(stream)
            vr.vr_upload_volume(ctx, vol_dev, dt, nx, ny, nz, w["value_max"], sh)
            ev[i][1].record(stream)
            vr.vr_set_transfer_function(ctx, tf_dev, tf_dev.shape[0], sh)
            vr.vr_set_camera(ctx, cam_s)
            ev[i][2].record(stream)
            vr.vr_render(ctx, params, out, sh)
            ev[i][3].record(stream)
        barrier(world)
        t_wall = time.perf_counter() - t_wall
    step_ms = [ev[i][0].elapsed_time(ev[i][3]) for i in range(K)]
    upload_ms = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(K))
    tf_ms = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(K))
    render_ms = statistics.mean(ev[i][2].elapsed_time(ev[i][3]) for i in range(K))
    # render only (volume, transfer function, camera and gradient records unchanged): the
    # fused march kernel alone, the interactive frame rate of a resident volume
    evr = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for i in range(K):
        flush.fill_(float(i))
        evr[i][0].record(stream)
        vr.vr_render(ctx, params, out, sh)
        evr[i][1].record(stream)
    torch.cuda.synchronize()
    march_ms = [evr[i][0].elapsed_time(evr[i][1]) for i in range(K)]
    samples = stats["samples_plain"]
    value, ms_per_step = replica_throughput(samples, K, sum(step_ms), world)
    march_avg = statistics.mean(march_ms)

    # roofline of the dominant kernel (the fused march): FP32 ALU against the unit counts
    # and the maximum SM clock; algorithmic operations per visited / shaded sample as
    # defined by FLOPS_VISIT / FLOPS_SHADE
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    flops = stats["samples_visited"] * FLOPS_VISIT + stats["samples_shaded"] * FLOPS_SHADE[w["grad"]]
    achieved = flops / (march_avg / 1e3) / 1e12
    bpv = {"u8": 1, "u16": 2, "f16": 2, "f32": 4}[dt]
    hbm_bytes = (nx + 3) * (ny + 3) * (nz + 3) * bpv + H * W * 16
    hbm_achieved = hbm_bytes / (march_avg / 1e3) / 1e9
    records_ms = max(render_ms - march_avg, 0.0)
    roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak, "traffic": profiled_traffic("k_march"),
            "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
            "kernel": "k_march", "launch_ms": march_avg,
            "flops_per_launch": flops,
            "frac_incl_records": flops / ((march_avg + records_ms) / 1e3) / 1e12 / alu_peak}
    roof_hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": float(pk["hbm_gbs"]),
                "unit": "GB/s", "frac": hbm_achieved / float(pk["hbm_gbs"]),
                "bytes_per_launch": hbm_bytes,
                "peak_source": f"{pk_kind} copy bandwidth"}
    # measured ceilings (vr_measure_peaks, outside the timed region): the march's time
    # against the largest of its FP32 work at the measured FMA rate, its visited samples at
    # the best measured gather-and-blend rate (random cells of an L1-resident table, or the
    # march's own access pattern over an L2-resident one), and its compulsory HBM bytes
    mp = vr.vr_measure_peaks(local, 5)
    g_peak = max(mp["gather_coherent_gsps"], mp["gather_random_gsps"])
    terms = {"alu": flops / (mp["fma_tflops"] * 1e12) * 1e3,
             "gather": stats["samples_visited"] / (g_peak * 1e9) * 1e3,
             "hbm": hbm_bytes / (float(pk["hbm_gbs"]) * 1e9) * 1e3}
    binding = max(terms, key=terms.get)
    roof["peak_measured"] = mp["fma_tflops"]
    roof["frac_of_measured"] = achieved / mp["fma_tflops"]
    roof_measured = {"bound": binding, "t_roof_ms": terms[binding], "launch_ms": march_avg,
                     "frac": terms[binding] / march_avg, "terms_ms": terms, "peaks": mp,
                     "peak_source": "vr_measure_peaks, best of 5: FP32 FMA chains; gather + "
                                    "blend of 8 corner records per sample, the better of "
                                    "random cells in L1 and the march's pattern in L2"}
    # the method's own footprint: every visited sample gathers the 8 voxels of its cell in the
    # volume's storage type (here at the better of the two measured 16-bit gather rates) ->
    # T_roof = max(compulsory HBM, FP32 work at the FMA rate, those gathers); beside it the
    # full neighbourhood footprint of the shaded samples (4^3 voxels for the 3x3x3 operators,
    # the 32-voxel cross for central differences, counted as 8-voxel gathers), which the
    # precomputed operator records avoid paying per sample
    g_u16 = max(mp["gather_u16_random_gsps"], mp["gather_u16_coherent_gsps"])
    hood = {"central": 32, "sobel3d": 64, "zucker_hummel": 64}[w["grad"]]
    terms_vox = {"alu": terms["alu"], "hbm": terms["hbm"],
                 "gather": stats["samples_visited"] / (g_u16 * 1e9) * 1e3}
    bind_vox = max(terms_vox, key=terms_vox.get)
    roof_voxel = {"bound": bind_vox, "t_roof_ms": terms_vox[bind_vox], "launch_ms": march_avg,
                  "frac": terms_vox[bind_vox] / march_avg, "terms_ms": terms_vox,
                  "gather_peak_gsps": g_u16,
                  "neighbourhood_gather_ms": (stats["samples_visited"] + stats["samples_shaded"] * hood / 8)
                  / (g_u16 * 1e9) * 1e3,
                  "peak_source": "vr_measure_peaks, best of 5: 8 voxels of a cell in 16-bit "
                                 "storage + trilinear blend, the better of random cells in L1 "
                                 "and the march's pattern in L2"}

    line = {
        "metric": "Gsamples/s", "value": value, "unit": "Gsamples/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "ms_per_step_median": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(w, world),
        "frames_per_s": 1000.0 / ms_per_step,
        "phase_ms": {"upload": upload_ms, "tf_camera": tf_ms, "render": render_ms,
                     "records": records_ms, "march": march_avg},
        "render_only": {"value": samples / (march_avg / 1e3) / 1e9, "unit": "Gsamples/s",
                        "frames_per_s": 1000.0 / march_avg},
        "march_ms": march_avg,
        "samples_per_frame": samples,
        "samples_visited": stats["samples_visited"],
        "samples_shaded": stats["samples_shaded"],
        "rays_hit": stats["rays_hit"],
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "roofline_measured": roof_measured,
        "roofline_voxel_gather": roof_voxel,
        # per step: k_pad, k_brick_minmax, k_brick_visibility (upload); k_tf_prefix,
        # k_brick_visibility (transfer function); k_records, k_march (render)
        "gpu_launches": 7 * K,
        "wall_s": t_wall,
    }
    line["clocks"] = clk.summary()

    f16_img = f16_vol = None
    if not args.no_extras:
        line["f16"], f16_img, f16_vol = f16_leg(args, max(10, min(K, 50)))
        line["sparse"] = sparse_leg(args, max(10, min(K, 50)))
        line["slab"] = slab_leg(args, max(10, min(K, 30)))
        line["train"] = train_leg(R, args)
        line["fwd_bwd"] = fwd_bwd_leg(R, args)
        line["surface"] = surface_leg(R, args)
        line["adaptive"] = adaptive_leg(R, args)
        line["batch"] = batch_leg(args)
    if not args.no_extras and world == 1:
        # end to end through the C ABI with host buffers: H2D of the volume and TF, D2H of
        # the image, every step.  Serial: one context, each step waited for.  Pipelined:
        # DEPTH contexts on DEPTH streams, so a step's copies overlap the previous steps'
        # kernels; the host reads every step's image (checks a pixel) before its buffer is
        # reused.  The host waits for each volume copy (the caller's buffer is free when the
        # upload returns), so the pipeline needs a few steps in flight: 1.50 / 1.04 / 1.03 /
        # 1.03 ms per step with 2 / 3 / 4 / 5 contexts.
        from paper_1609_01317_gb300 import Renderer as _R

        DEPTH = 4
        host_vol = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).pin_memory()
        host_tf = torch.from_numpy(w["tf"]).pin_memory()
        host_out = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(DEPTH)]
        extra = [_R(local) for _ in range(DEPTH - 1)]
        ctxs = [ctx] + [r.ctx for r in extra]
        streams = [torch.cuda.Stream() for _ in range(DEPTH)]
        done = [torch.cuda.Event() for _ in range(DEPTH)]

        def e2e_step(j):
            h = streams[j].cuda_stream
            vr.vr_upload_volume(ctxs[j], host_vol, dt, nx, ny, nz, w["value_max"], h)
            vr.vr_set_transfer_function(ctxs[j], host_tf, host_tf.shape[0], h)
            vr.vr_set_camera(ctxs[j], cam_s)
            vr.vr_render(ctxs[j], params, host_out[j], h)
            done[j].record(streams[j])

        for rep in range(2):
            for j in range(DEPTH):
                e2e_step(j)
        torch.cuda.synchronize()
        ref_out = out.cpu()
        ok = all(torch.equal(o, ref_out) for o in host_out)
        ke = max(2 * DEPTH, min(K, 60))
        probe = (H // 2, W // 2)
        checks = 0.0
        t0 = time.perf_counter()
        for i in range(ke):
            e2e_step(0)
            done[0].synchronize()
            checks += float(host_out[0][probe][3])
        serial_s = (time.perf_counter() - t0) / ke
        # the pipelined loop is driven from one host thread, so host scheduling shows in it:
        # three runs of ke steps each, the median reported and all three listed
        e2e_runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            for i in range(ke):
                j = i % DEPTH
                if i >= DEPTH:
                    done[j].synchronize()  # step i - DEPTH finished: read its image
                    checks += float(host_out[j][probe][3])
                e2e_step(j)
            for j in range(DEPTH):
                done[j].synchronize()
                checks += float(host_out[j][probe][3])
            e2e_runs.append((time.perf_counter() - t0) / ke)
        e2e_s = statistics.median(e2e_runs)
        ok = ok and torch.equal(host_out[(ke - 1) % DEPTH], ref_out)
        # the same pipeline with the 8-bit image (vr_render_rgba8): a quarter of the read-back
        host8 = [torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in range(DEPTH)]

        def e2e_step8(j):
            h = streams[j].cuda_stream
            vr.vr_upload_volume(ctxs[j], host_vol, dt, nx, ny, nz, w["value_max"], h)
            vr.vr_set_transfer_function(ctxs[j], host_tf, host_tf.shape[0], h)
            vr.vr_set_camera(ctxs[j], cam_s)
            vr.vr_render_rgba8(ctxs[j], params, host8[j], h)
            done[j].record(streams[j])

        for j in range(DEPTH):
            e2e_step8(j)
        torch.cuda.synchronize()
        ref8 = torch.round(ref_out.clamp(0.0, 1.0) * 255.0).to(torch.uint8)
        ok8 = all(torch.equal(o, ref8) for o in host8)
        e2e8_runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            for i in range(ke):
                j = i % DEPTH
                if i >= DEPTH:
                    done[j].synchronize()
                    checks += float(host8[j][probe][3])
                e2e_step8(j)
            for j in range(DEPTH):
                done[j].synchronize()
                checks += float(host8[j][probe][3])
            e2e8_runs.append((time.perf_counter() - t0) / ke)
        e2e8_s = statistics.median(e2e8_runs)
        # the host link's own rates (plain copies of the same bytes): the bound of any step
        # that moves the volume in and the image out
        def copy_ms(dst, src, reps=5):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                dst.copy_(src, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        h2d_ms = copy_ms(vol_dev, host_vol)
        d2h_ms = copy_ms(host_out[0], out)
        # both directions at once on two streams (the link carries them concurrently)
        cs_a, cs_b = torch.cuda.Stream(), torch.cuda.Stream()

        def both_ms(reps=5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                with torch.cuda.stream(cs_a):
                    vol_dev.copy_(host_vol, non_blocking=True)
                with torch.cuda.stream(cs_b):
                    host_out[0].copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps * 1e3

        both_ms()
        conc_ms = both_ms()
        for r in extra:
            r.close()
        line["e2e"] = {"value": samples / e2e_s / 1e9, "unit": "Gsamples/s",
                       "h2d_bytes_per_step": int(vol.nbytes + w["tf"].nbytes),
                       "d2h_bytes_per_step": int(H * W * 16), "ms_per_step": e2e_s * 1e3,
                       "runs_ms": [round(r * 1e3, 4) for r in e2e_runs],
                       "pipeline": f"{DEPTH} contexts on {DEPTH} streams (a step's copies overlap "
                                   "the previous steps' kernels); host reads every step's image; "
                                   "median of 3 runs",
                       "serial_ms_per_step": serial_s * 1e3,
                       "serial_value": samples / serial_s / 1e9,
                       "steps": ke, "matches_device_result": bool(ok),
                       "rgba8": {"value": samples / e2e8_s / 1e9, "unit": "Gsamples/s",
                                 "ms_per_step": e2e8_s * 1e3,
                                 "runs_ms": [round(r * 1e3, 4) for r in e2e8_runs],
                                 "d2h_bytes_per_step": int(H * W * 4),
                                 "matches_quantised_device_result": bool(ok8),
                                 "what": "the same pipeline reading back vr_render_rgba8's "
                                         "8-bit image"},
                       "link": {"h2d_gbs": vol.nbytes / h2d_ms / 1e6,
                                "d2h_gbs": H * W * 16 / d2h_ms / 1e6,
                                "copies_ms": h2d_ms + d2h_ms,
                                "concurrent_copies_ms": conc_ms,
                                "frac": conc_ms / (e2e_s * 1e3)}}
        # CPU baseline: the FP64 oracle on a bounded sample of the same workload
        cb = oracle_sample(w, args.cpu_seconds)
        what = (f"{cb['frames']} whole frame(s)" if cb["frames"] else
                f"image rows {cb['rows'][0]}-{cb['rows'][1]}")
        one, one_rows = oracle_one_core(w)
        # error of the GPU frame against the oracle's rendering of the same rows (the
        # oracle renders rows of the whole image; only those rows are compared)
        r0, r1 = cb["rows"]
        gpu = out.cpu().numpy().astype(np.float64)[r0:r1]
        ref = cb["image"][r0:r1]
        err = np.abs(gpu - ref).max(axis=-1)
        line["parity"] = {"reference": "FP64 oracle", "rows": [r0, r1],
                          "pixels": int(err.size), "max_abs": float(err.max()),
                          "frac_within_2e-3": float((err <= 2e-3).mean()),
                          "mean_abs": float(np.abs(gpu - ref).mean())}
        import oracle

        if f16_img is not None:
            # the FP16 frame against the FP64 oracle's frame of the same FP16 volume, whole
            # image (both storage variants' errors side by side)
            t0 = time.perf_counter()
            ref16, _, _ = oracle.render(oracle.OracleVolume(f16_vol, 1.0), w["tf"], cam,
                                        oracle.make_params(step=w["step"], grad=w["grad"]))
            e16 = np.abs(f16_img.astype(np.float64) - ref16).max(axis=-1)
            line["f16"]["parity"] = {"reference": "FP64 oracle", "rows": [0, H],
                                     "pixels": int(e16.size), "max_abs": float(e16.max()),
                                     "frac_within_2e-3": float((e16 <= 2e-3).mean()),
                                     "mean_abs": float(np.abs(f16_img - ref16).mean()),
                                     "oracle_s": time.perf_counter() - t0}
        sp = line.get("sparse", {}).pop("_samples", None)
        if sp is not None:
            ws = sp["w"]
            ref, _, _ = oracle.render_pixels(
                oracle.OracleVolume(ws["volume"], ws["value_max"]), ws["tf"], ws["camera"],
                oracle.make_params(step=ws["step"], grad=ws["grad"]), sp["pick"][:, 1],
                sp["pick"][:, 0])
            es = np.abs(sp["got"].astype(np.float64) - ref).max(axis=-1)
            line["sparse"]["parity"] = {"reference": "FP64 oracle", "pixels": int(es.size),
                                        "sample": "1500 pixels whose ray reaches something "
                                                  "+ 300 anywhere",
                                        "max_abs": float(es.max()),
                                        "frac_within_2e-3": float((es <= 2e-3).mean())}
        bs = line.get("batch", {}).pop("_samples", None)
        if bs is not None:
            line["batch"]["parity"] = batch_parity(bs)
        line["cpu_baseline"] = {"value": cb["samples"] / cb["seconds"] / 1e9,
                                "unit": "Gsamples/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": f"{what} of the workload "
                                          f"({cb['samples']} samples, {cb['seconds']:.1f} s)",
                                "per_core": {"value": one, "unit": "Gsamples/s",
                                             "sample": f"{one_rows} middle rows, 1 thread"}}
    else:
        line["e2e"] = None
        line["cpu_baseline"] = None
    for leg in ("batch", "sparse"):  # host copies kept only for the oracle comparison
        if isinstance(line.get(leg), dict):
            line[leg].pop("_samples", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_leg(args):
    import torch

    from paper_1609_01317_gb300 import Renderer, build

    build.build()
    torch.cuda.set_device(0)
    if args.leg in ("fwd_bwd", "surface", "adaptive", "train"):
        R = Renderer(0)
        out = {"fwd_bwd": fwd_bwd_leg, "surface": surface_leg, "adaptive": adaptive_leg,
               "train": train_leg}[args.leg](R, args)
        R.close()
    elif args.leg == "f16":
        out = f16_leg(args, max(10, min(args.steps, 50)))[0]
    elif args.leg == "sparse":
        out = sparse_leg(args, max(10, min(args.steps, 50)))
        out.pop("_samples", None)
    elif args.leg == "slab":
        out = slab_leg(args, max(10, min(args.steps, 50)))
    else:
        out = batch_leg(args)
        out.pop("_samples", None)
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.source_hash:
        print(source_hash(args.source_hash))
        return 0
    if args.leg != "main":
        return run_leg(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
