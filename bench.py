"""Benchmark of the relit-avatar render path on one GB300.

Workload (default): the paper-scale forward frame - 50k-vertex procedural
body, 200k Gaussians, 16x32 environment light, 512 visibility directions at
256^2, one 1024x1024 camera (synthetic, seeded).  A "step" is one relit
frame through all four stages (skin, visibility, shade, splat), replayed
from a CUDA graph; the training step (frame + L1 loss + every backward
kernel) is timed the same way and reported beside it.

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU
oracle on the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "c2_paper"
WORKLOAD_DESC = ("relit frame 1024x1024, 200k Gaussians, 50k-vertex mesh, 16x32 env light, "
                 "512 visibility directions at 256^2")
METRIC = "relit frames/s (fwd) and train steps/s (fwd+bwd) at 1024^2, 200k Gaussians"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ".",
                                 f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9 and p[1].replace(".", "").isdigit():
                        rows.append(p)
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        ge.build()
    if world > 1:
        torch.distributed.barrier()
        ge.build()
    from paper_2407_10707_gb300 import render, synth
    STM = sys.modules[__name__]

    dev = torch.device("cuda", local)
    sc = synth.config_scene(args.workload)
    st = render.scene_tensors(sc, dev)
    G, Nv, F = sc.avatar.G, sc.avatar.Nv, sc.avatar.F
    NL, D, R = len(sc.light.A), sc.frames.shape[0], sc.depth_res
    W, H = sc.camera.width, sc.camera.height
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    r = render.Renderer(st, tile=args.tile)
    r.check()
    r.capture()
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            flush.fill_(1.0)                      # evict L2 between timed iterations
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total / steps

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        fwd_ms = timed(r.replay, args.steps, args.warmup)
        torch.cuda.synchronize()
        # training step: frame + L1 loss + backward of every stage
        tgt = r.sb.image.detach().clone() * 0.9
        ts = render.TrainStep(st, tgt, tile=args.tile)
        ts.check()
        ts.capture()
        train_ms = timed(ts.graph.replay, args.steps, args.warmup)
        torch.cuda.synchronize()
        # end to end through host buffers: per-frame pose and light in, image out
        e2e = STM.end_to_end(r, st, args.steps, args.warmup, flush)
    if world > 1:
        t = torch.tensor([fwd_ms, train_ms, e2e["ms"]], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        fwd_ms, train_ms, e2e_ms = (float(x) for x in t.tolist())
        e2e["ms"] = e2e_ms
    # per-stage timing (eager, CUDA events on the launching stream)
    stages = STM.stage_times(r, st, reps=max(3, min(args.steps, 10)), flush=flush)
    stats = STM.workload_stats(r, sc)
    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    roof = STM.roofline(stages, stats, sc, peaks, peak_kind, clocks)
    r.check()
    ts.check()
    if rank != 0:
        return
    value = world * 1000.0 / fwd_ms
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(fwd_ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded procedural capsule-union avatar; paper datasets are not available)",
        "config": {"workload": WORKLOAD_DESC, "gaussians": G, "mesh_vertices": Nv, "faces": F, "lights": NL,
                   "vis_dirs": D, "vis_res": R, "image": [W, H], "tile": args.tile,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "flushed (256 MB write) between timed steps", "graph": "CUDA graph replay",
                   "visibility": "one-sided raster of the closed capsule body (same bits as two-sided)"},
        "train": {"value": round(world * 1000.0 / train_ms, 3), "unit": "train steps/s", "ms_per_step":
                  round(train_ms, 5)},
        "stages_us": {k: round(v * 1000.0, 2) for k, v in stages.items()},
        "e2e": {"value": round(world * 1000.0 / e2e["ms"], 3), "unit": "frames/s",
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
        "gpu_launches": stats["launches_per_frame"] * args.steps,
        "roofline": roof,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc, budget_s=args.cpu_budget)
    if args.workload != WORKLOAD:
        line["config"]["workload"] = args.workload
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- measurement helpers
def _graph_of(fn):
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def stage_times(r, st, reps, flush):
    """Device time of each stage (ms), each stage replayed from its own CUDA
    graph between CUDA events on the launching stream, L2 flushed before."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for name, fn in (("skin", r.skin), ("visibility", r.visibility), ("shade", r.shade), ("splat", r.splat)):
        g = _graph_of(fn)
        g.replay()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        out[name] = tot / reps
    return out


def workload_stats(r, sc):
    """Counts that define the algorithmic work of each stage (outside any
    timed region; plain torch reductions over the frame's own buffers)."""
    import torch
    t = r.st["avatar"]
    G = t["xg"].shape[1]
    cull = r.sh["cull"].bool()
    front = int((~cull).sum().item())
    nd = r.sk["nd"]
    w = r.st["light"]["w"]
    lit = 0
    for c0 in range(0, G, 32768):
        sl = slice(c0, min(G, c0 + 32768))
        cos = (w @ nd[:, sl]) > 0                       # [NL, g]
        lit += int((cos & ~cull[sl][None, :]).sum().item())
    P = int(r.sb.num_pairs.item())
    Fc = sc.avatar.F
    return {"front_gaussians": front, "lit_pairs_upper": lit, "pairs": P, "faces": Fc,
            "launches_per_frame": 33}


def roofline(stages, stats, sc, peaks, peak_kind, clocks):
    """Per-stage achieved rate against its bound; the dominant stage first."""
    G, Nv, F = sc.avatar.G, sc.avatar.Nv, sc.avatar.F
    NL, D = len(sc.light.A), sc.frames.shape[0]
    W, H = sc.camera.width, sc.camera.height
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    int_peak = 152 * 128 * sm_max * 1e6 / 1e12       # int32 Tops/s at the maximum clock
    fp32_peak = 2 * int_peak                          # FMA = 2 flops
    hbm = float(peaks["hbm_gbs"])
    out = {}
    # skinning: algorithmic bytes = inputs + outputs
    skin_bytes = 140 * G + 164 * Nv
    out["skin"] = {"bound": "hbm", "achieved": skin_bytes / (stages["skin"] * 1e-3) / 1e9, "peak": hbm,
                   "unit": "GB/s", "traffic": None}
    # visibility: integer ops of the exact rules (setup per direction-triangle,
    # test per direction-vertex; covered samples are not counted)
    vis_ops = D * (60.0 * F + 20.0 * Nv)
    out["visibility"] = {"bound": "alu", "achieved": vis_ops / (stages["visibility"] * 1e-3) / 1e12,
                         "peak": int_peak, "unit": "Tops/s (int32)", "traffic": None}
    # shading: 6 flops cosine test per front-facing pair + 50 flops per lit pair
    sh_flops = 6.0 * stats["front_gaussians"] * NL + 50.0 * stats["lit_pairs_upper"]
    out["shade"] = {"bound": "alu", "achieved": sh_flops / (stages["shade"] * 1e-3) / 1e12, "peak": fp32_peak,
                    "unit": "TFLOP/s (fp32)", "traffic": None}
    # splatting: bytes of inputs, projection, pair lists (write + sort passes + read) and image
    P = stats["pairs"]
    sp_bytes = 53 * G + 40 * G + P * 8 * (2 + 2 * 2) + 20 * W * H
    out["splat"] = {"bound": "hbm", "achieved": sp_bytes / (stages["splat"] * 1e-3) / 1e9, "peak": hbm,
                    "unit": "GB/s", "traffic": None}
    for v in out.values():
        v["frac"] = round(v["achieved"] / v["peak"], 4)
        v["achieved"] = round(v["achieved"], 3)
        v["peak"] = round(v["peak"], 1)
    # DRAM traffic per launch from the committed ncu summary, only while the
    # kernel source is unchanged since the capture
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "ncu_traffic_c2.json")) as f:
            tr = json.load(f)["kernels"]
        for stage, rec in tr.items():
            with open(os.path.join(ROOT, rec["source"]), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() == rec["source_sha256"] and stage in out:
                    out[stage]["traffic"] = rec["dram_bytes_per_launch"]
                    out[stage]["traffic_kernel"] = rec["kernel"]
    except (OSError, KeyError, ValueError):
        pass
    dom = max(stages, key=lambda k: stages[k])
    res = dict(out[dom])
    res["stage"] = dom
    res["peak_source"] = f"{peak_kind} (HBM from MEASURED_PEAKS.json; ALU peaks = 152 SMs x 128 lanes x max clock)"
    res["stages"] = out
    return res


def end_to_end(r, st, steps, warmup, flush):
    """Frames/s through the public API with host buffers: each step copies
    the pose and the environment light in from pinned host memory, replays
    the frame and reads the image back into pinned host memory."""
    import torch
    t = st["avatar"]
    pose_h = t["pose"].cpu().pin_memory()
    light_h = st["light"]["L"].cpu().pin_memory()
    img_h = torch.empty(r.sb.image.shape, dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()

    def step():
        t["pose"].copy_(pose_h, non_blocking=True)
        st["light"]["L"].copy_(light_h, non_blocking=True)
        r.replay()
        img_h.copy_(r.sb.image, non_blocking=True)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return {"ms": tot / steps, "h2d": pose_h.numel() * 4 + light_h.numel() * 4, "d2h": img_h.numel() * 4}


# ----------------------------------------------------------------- CPU arm
def cpu_baseline(sc=None, budget_s=20.0, sample_frac=None):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample
    of the same frame; scaled to frames/s."""
    import numpy as np

    from oracle import oracle as O
    from paper_2407_10707_gb300 import synth
    if sc is None:
        sc = synth.config_scene(WORKLOAD)
    cores = O.set_threads(os.cpu_count() or 1)
    av = sc.avatar
    t0 = time.perf_counter()
    bone = O.fk(av.parents, av.joints, av.pose)
    sk = O.skin(av, bone)
    t_skin = time.perf_counter() - t0
    # visibility on a sample of directions (each direction is independent)
    D = sc.frames.shape[0]
    nd = 32
    fr = np.asarray(sc.frames.reshape(-1, 9), np.float32).astype(np.float64)
    xp = np.asarray(sk["xp"], np.float32).astype(np.float64)
    t0 = time.perf_counter()
    O.visibility(xp, av.faces, fr[:nd], sc.window_center, sc.window_half, sc.vis_bias, sc.depth_res)
    t_vis = (time.perf_counter() - t0) * D / nd
    bits = O.visibility(xp, av.faces, fr, sc.window_center, sc.window_half, sc.vis_bias, sc.depth_res) \
        if D <= 64 else None
    if bits is None:
        bits = np.full((av.Nv, D // 32), 0xFFFFFFFF, np.uint32)
    # shading on a sample of Gaussians
    gs = min(av.G, 20_000)
    sel = slice(0, gs)
    t0 = time.perf_counter()
    O.shade(sk["xd"][sel], sk["nd"][sel], sk["ag"][sel], sk["rg"][sel], sk["pg"][sel], sk["ubar"][sel],
            av.knn[sel], bits, sc.light.L, sc.light.A, sc.light.w, sc.dmap, sc.camera.center, D)
    t_shade = (time.perf_counter() - t0) * av.G / gs
    col, _, cull = O.shade(sk["xd"], sk["nd"], sk["ag"], sk["rg"], sk["pg"], sk["ubar"], av.knn, bits,
                           sc.light.L, sc.light.A, sc.light.w, sc.dmap, sc.camera.center, D)
    t0 = time.perf_counter()
    pr = O.project(sk["xd"], sk["cov"], av.opacity, cull, sc.camera)
    t_proj = time.perf_counter() - t0
    # brute-force compositing on sampled pixels of the body's bounding box
    W, H = sc.camera.width, sc.camera.height
    rng = np.random.default_rng(0)
    npx = 1024
    pix = rng.integers(0, W * H, npx).astype(np.int32)
    t0 = time.perf_counter()
    O.composite(pr["mean2d"], pr["conic"], av.opacity, col, pr["depth"], pr["valid"], W, H, pix)
    t_comp = (time.perf_counter() - t0) * (W * H) / npx
    frame_s = t_skin + t_vis + t_shade + t_proj + t_comp
    return {"value": round(1.0 / frame_s, 6), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": (f"skinning in full; visibility on {nd}/{D} directions; shading on {gs}/{av.G} Gaussians; "
                       f"projection in full; brute-force compositing on {npx} random pixels of {W * H}; "
                       f"each scaled linearly to the full frame"),
            "stage_s": {"skin": round(t_skin, 4), "visibility": round(t_vis, 3), "shade": round(t_shade, 3),
                        "project": round(t_proj, 4), "composite": round(t_comp, 2)}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    from paper_2407_10707_gb300 import synth
    sc = synth.config_scene(WORKLOAD)
    for _ in range(args.warmup):
        pass
    vals = []
    for _ in range(max(1, min(args.steps, 3))):
        vals.append(cpu_baseline(sc, budget_s=args.cpu_budget))
    v = sorted(x["value"] for x in vals)[len(vals) // 2]
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 / v, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded procedural capsule-union avatar)",
            "config": {"workload": WORKLOAD_DESC}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--workload", default=WORKLOAD, help="named synthetic configuration (profiling uses smaller ones)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
