#!/usr/bin/env python
"""Benchmark: synchronized tracing of a seeded 1,024-primitive blobtree at 1920x1080.

One step = the whole hot path on one frame: st_build_tiles (per-tile culling
into the A-buffer) + st_trace (synchronized sphere tracing with sparse
pruning), inputs resident in HBM.  The headline mode is the learned
relaxation step; the plain step, fixed omega = 1.7 and the paper's own ray
processing (Sec. 10: omega = 1.7, minimum step, crossing test, no step cap) are
timed in the same run with identical Lipschitz bound and subfrustum sizes.
--workload table1 times the synchronized pipeline against the paper's
per-pixel comparison variants (Table 1).
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 1080p|small|clustered|clustered1080p|families1080p|batch64|table1|blend] [--modes learned,plain,overrelax,crossing]

Multi-GPU: one independent replica per rank (the path has no exchange step);
value = all ranks' rays / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import re
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "rays/s and prim-evals/s at 1080p (1k–10k prims), learned vs plain step, same tol"
FP32_LANES_PER_SM = 128


def workload(name: str):
    from paper_2304_09673_b300 import scenegen as sg
    if name == "1080p":
        return sg.workload_1080p(100), sg.default_camera(1920, 1080), dict(
            workload="1,024-primitive seeded blobtree (depth<=14, seed 100), 1920x1080, tile 16, "
                     "synchronized sphere tracing, eps 1e-4, max 256 steps", prims=1024,
            resolution="1920x1080", tile=16)
    if name == "small":
        return sg.workload_small(0), sg.default_camera(256, 256), dict(
            workload="64-primitive seeded blobtree (complete depth 6, seed 0), 256x256, tile 16", prims=64,
            resolution="256x256", tile=16)
    if name == "clustered":
        return sg.workload_clustered(200), sg.default_camera(3840, 2160), dict(
            workload="10,000 primitives in 50 Gaussian clusters (sigma 0.05, depth<=20, seed 200), 3840x2160, "
                     "tile 16", prims=10000, resolution="3840x2160", tile=16)
    if name == "clustered1080p":
        return sg.workload_clustered(200), sg.default_camera(1920, 1080), dict(
            workload="10,000 primitives in 50 Gaussian clusters (sigma 0.05, depth<=20, seed 200), 1920x1080, "
                     "tile 16", prims=10000, resolution="1920x1080", tile=16)
    if name == "families1080p":
        return sg.workload_families(100, n_prims=1024, max_depth=14), sg.default_camera(1920, 1080), dict(
            workload="1,024 primitives of six families (sphere, rounded box, capsule, torus, sphere-cone, "
                     "ellipsoid; depth<=14, seed 100), 1920x1080, tile 16", prims=1024, resolution="1920x1080",
            tile=16)
    raise SystemExit(f"unknown workload {name}")


def workload_of(args):
    """The single-scene workload of the command line, at --res if given (a
    smaller frame of the same scene, for profiling captures of small cases)."""
    scene, cam, cfg = workload(args.workload)
    if getattr(args, "res", None):
        from paper_2304_09673_b300 import scenegen as sg
        w, h = (int(v) for v in args.res.lower().split("x"))
        cam = sg.default_camera(w, h)
        cfg = dict(cfg, resolution=f"{w}x{h}", workload=cfg["workload"] + f", rendered at {w}x{h}")
    return scene, cam, cfg


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The slowest rank's time (replicas: every rank runs the same work)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units processed by all ranks / the max-over-ranks time."""
    return units_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.tmp.flush()
        rows = list(csv.reader(io.StringIO(Path(self.tmp.name).read_text())))
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return json.loads(p.read_text())
        except Exception:
            pass
    return {}


def kernel_hash() -> str:
    """Hash of the traced kernel's sources with comments and blank space
    removed: a recorded ncu traffic figure stays valid across comment edits
    and goes stale on any change to the code."""
    h = hashlib.sha256()
    for f in ("st_trace.cu", "st_field.cuh", "st_geom.cuh", "st_internal.h", "st_mlp.cuh", "st_kernels.h"):
        src = (ROOT / "paper_2304_09673_b300" / "csrc" / f).read_text()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str, mode: str):
    """DRAM bytes per trace launch from a committed ncu summary, valid only
    while the traced kernel's sources are unchanged."""
    p = ROOT / "profiles" / f"trace_{mode}_{workload_name}_traffic.json"
    if not p.exists():
        return None
    try:
        d = json.loads(p.read_text())
    except Exception:
        return None
    if d.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    return d.get("dram_bytes_per_launch")


def cpu_baseline(scene, cam, seconds: float, seed: int = 7) -> dict:
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)

    def run(n):
        pi = rng.integers(0, cam.width, n).astype(np.int32)
        pj = rng.integers(0, cam.height, n).astype(np.int32)
        t0 = time.perf_counter()
        oracle.trace(scene, cam, pi, pj, max_steps=100000)
        return time.perf_counter() - t0

    n = 64
    t = run(n)
    while t < 0.5 and n < 1 << 20:
        n *= 4
        t = run(n)
    n_final = max(n, int(n * seconds / max(t, 1e-6)))
    t = run(n_final)
    return {"value": n_final / t, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_final} random pixel rays of the {cam.width}x{cam.height} frame, dense FP64 "
                      f"full-tree sphere tracing (no A-buffer), {t:.1f} s"}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    import numpy as np
    import oracle
    scene, cam, cfg = workload_of(args)
    oracle.build()
    rng = np.random.default_rng(11)
    n = args.ref_pixels
    times = []
    for it in range(args.warmup + args.steps):
        pi = rng.integers(0, cam.width, n).astype(np.int32)
        pj = rng.integers(0, cam.height, n).astype(np.int32)
        t0 = time.perf_counter()
        oracle.trace(scene, cam, pi, pj, max_steps=100000)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = n / mean
    cfg = dict(cfg, parallelism="host cores", sample=f"{n} random pixel rays per step")
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n} random pixel rays of the {cam.width}x{cam.height} frame per step, "
                                       "dense FP64 full-tree sphere tracing"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ray_dirs(cam, torch):
    """Unit view-ray directions of every pixel centre (float64, device), the
    pinhole model of the library (d = F + u R + v U)."""
    import numpy as np
    eye = np.array(cam.eye, np.float64)
    F = np.array(cam.target, np.float64) - eye
    F /= np.linalg.norm(F)
    R = np.cross(F, np.array(cam.up, np.float64))
    R /= np.linalg.norm(R)
    U = np.cross(R, F)
    th = math.tan(math.radians(cam.vfov_deg) / 2)
    R *= th * cam.width / cam.height
    U *= th
    dev = torch.device("cuda")
    u = (2 * torch.arange(cam.width, device=dev, dtype=torch.float64) + 1) / cam.width - 1
    v = 1 - (2 * torch.arange(cam.height, device=dev, dtype=torch.float64) + 1) / cam.height
    d = (torch.tensor(F, device=dev)[None, None, :] + u[None, :, None] * torch.tensor(R, device=dev)[None, None, :]
         + v[:, None, None] * torch.tensor(U, device=dev)[None, None, :])
    return (d / d.norm(dim=-1, keepdim=True)).reshape(-1, 3)


def agreement(cam, diam, ref, got, torch):
    """Agreement of a mode with the plain tracer at the same eps.  The
    silhouette band (plain mask differs from a 4-neighbour, or a grazing
    plain hit with |n.d| < 0.05) is where the stopping rule f <= eps decides
    hit or miss for rays that pass within eps of the surface; outside it the
    modes must agree.  Depth in scene units (Euclidean)."""
    fp, dp, npl = ref
    fm, dm = got
    H, W = cam.height, cam.width
    hp, hm = (fp & 1).bool(), (fm & 1).bool()
    m2 = hp.reshape(H, W)
    edge = torch.zeros_like(m2)
    edge[1:, :] |= m2[1:, :] != m2[:-1, :]
    edge[:-1, :] |= m2[:-1, :] != m2[1:, :]
    edge[:, 1:] |= m2[:, 1:] != m2[:, :-1]
    edge[:, :-1] |= m2[:, :-1] != m2[:, 1:]
    cosn = (npl.reshape(-1, 3).double() * ray_dirs(cam, torch)).sum(-1).abs()
    band = edge.reshape(-1) | (hp & (cosn < 0.05))
    both = hp & hm
    dd = (dm - dp).abs()
    far = both & (dd > 1e-4 * diam)
    out = {"mask_mismatch_frac": float((hp != hm).float().mean().item()),
           "depth_diff_p99": float(torch.quantile(dd[both][:1 << 24].float(), 0.99).item()) if both.any() else 0.0,
           "depth_diff_max": float(dd[both].max().item()) if both.any() else 0.0,
           "silhouette_band_frac": float(band.float().mean().item()),
           "mask_mismatch_outside_band_frac": float(((hp != hm) & ~band).float().mean().item()),
           "depth_beyond_tol_outside_band_frac": float((far & ~band).float().mean().item()),
           "depth_tol": 1e-4 * diam}
    return out


# Launch options shared by every mode (set from the command line).
TRACE_EXTRA: dict = {}


def mode_opts(st, name: str, mlp, max_new: int):
    """Trace options of one step mode; eps, L, step cap and subfrustum sizes are identical across modes."""
    x = TRACE_EXTRA
    if name == "learned":
        return st.make_opts(step_mode=st.ST_STEP_LEARNED, mlp=mlp.data_ptr(), max_new_per_turn=max_new, **x)
    if name == "overrelax":
        return st.make_opts(step_mode=st.ST_STEP_OVERRELAX, omega=1.7, max_new_per_turn=max_new, **x)
    if name == "plain":
        return st.make_opts(step_mode=st.ST_STEP_PLAIN, max_new_per_turn=max_new, **x)
    if name == "crossing":
        # Sec. 10's own ray processing: omega = 1.7 with sphere reuse, minimum
        # step instead of eps and step cap (hits are crossings, f <= 0)
        return st.make_opts(step_mode=st.ST_STEP_CROSSING, omega=1.7, max_new_per_turn=max_new, **x)
    raise SystemExit(f"unknown step mode {name}")


def timed_loop(st, r, cam, opts, steps: int, warmup: int, flush, stream):
    """warmup untimed steps, then `steps` timed steps (tiles + trace), L2
    flushed before each; returns per-step and per-trace ms, counters, launches."""
    import numpy as np
    import torch
    for _ in range(warmup):
        r.build_tiles()
        r.trace(opts)
    torch.cuda.synchronize()
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(steps)]
    cnts = [torch.zeros_like(r.counters) for _ in range(steps)]
    launches0 = st.st_kernel_launches()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()                     # L2 flush between timed steps (outside the events)
        e0, e1, e2 = ev[k]
        e0.record(stream)
        r.build_tiles()
        e1.record(stream)
        st.st_trace(r.h, cam, r.tiles, opts, r.depth, r.normal, r.evals, r.flags, cnts[k], stream)
        e2.record(stream)
    torch.cuda.synchronize()
    launches = st.st_kernel_launches() - launches0
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    trace_ms = [m.elapsed_time(c) for _, m, c in ev]
    tiles_ms = [a.elapsed_time(m) for a, m, _ in ev]
    cnt = torch.stack(cnts).cpu().numpy().astype(np.float64)
    return dict(step_ms=step_ms, trace_ms=trace_ms, tiles_ms=tiles_ms, cnt=cnt, launches=launches)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2304_09673_b300 import build as b
    b.build()
    from paper_2304_09673_b300 import learn
    from paper_2304_09673_b300 import st

    scene, cam, cfg = workload_of(args)
    modes = [m.strip() for m in args.modes.split(",") if m.strip()]
    head = modes[0]
    stream = torch.cuda.current_stream()
    r = st.Renderer(scene, cam, tile=cfg["tile"], stream=stream)
    mlp = learn.packed_device(learn.load())
    W, H = cam.width, cam.height
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    props = torch.cuda.get_device_properties(0)
    try:
        gpu_id = str(props.uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None

    def measure(rr, cam_, steps):
        """Every mode timed on one renderer; clocks sampled in the head mode's
        timed region; agreement of each mode with the plain tracer."""
        res_all, imgs, clk = {}, {}, None
        for name in modes:
            opts = mode_opts(st, name, mlp, args.max_new)
            if world > 1:
                dist.barrier()
            sampler = ClockSampler(gpu_id) if (rank == 0 and name == head) else None
            res = timed_loop(st, rr, cam_, opts, steps, args.warmup, flush, stream)
            if sampler:
                clk = sampler.stop()
            res["ms_per_step"] = max_over_ranks(sum(res["step_ms"]), world) / steps
            res_all[name] = res
            imgs[name] = (rr.flags.clone(), rr.depth.clone(), rr.normal.clone())
        agr = {}
        if "plain" in imgs:
            d = st.st_scene_info(rr.h)["diameter"]
            for name, (f, dep, _) in imgs.items():
                if name != "plain":
                    agr[name] = agreement(cam_, d, imgs["plain"], (f, dep), torch)
        return res_all, agr, clk

    results, agreement_all, clocks = measure(r, cam, args.steps)

    # The other end of the metric's primitive range: 10,000 clustered
    # primitives at the same 1920x1080 (tile lists of thousands of entries),
    # every mode, fewer timed steps (each takes tens of milliseconds).
    secondary = None
    if args.workload == "1080p" and not args.no_secondary:
        s_scene, s_cam, s_cfg = workload("clustered1080p")
        r2 = st.Renderer(s_scene, s_cam, tile=s_cfg["tile"], stream=stream)
        s_steps = max(1, min(args.steps, 3))
        s_res, s_agr, s_clk = measure(r2, s_cam, s_steps)
        secondary = dict(cfg=s_cfg, cam=s_cam, res=s_res, agreement=s_agr, clocks=s_clk, steps=s_steps)
        r2.close()

    # ---- end to end through the public API with host buffers (headline mode) ----
    opts = mode_opts(st, head, mlp, args.max_new)
    ids = np.flatnonzero(scene.kind < 16).astype(np.int32)
    params = np.ascontiguousarray(scene.params[ids])
    words = {0: 1, 1: 4, 2: 3, 11: 5, 12: 2, 13: 4, 14: 5, 15: 7}   # record words per primitive kind
    h2d = int(sum(words[int(k)] for k in scene.kind[ids]) * 20)
    host = dict(depth=torch.empty(H * W, dtype=torch.float32, pin_memory=True),
                normal=torch.empty(H * W * 3, dtype=torch.float32, pin_memory=True),
                evals=torch.empty(H * W, dtype=torch.int32, pin_memory=True),
                flags=torch.empty(H * W, dtype=torch.uint8, pin_memory=True))
    d2h = sum(t.numel() * t.element_size() for t in host.values())

    def e2e_step():
        st.st_scene_update_prims(r.h, ids, params, stream)
        r.build_tiles()
        st.st_trace(r.h, cam, r.tiles, opts, r.depth, r.normal, r.evals, r.flags, None, stream)
        host["depth"].copy_(r.depth, non_blocking=True)
        host["normal"].copy_(r.normal, non_blocking=True)
        host["evals"].copy_(r.evals, non_blocking=True)
        host["flags"].copy_(r.flags, non_blocking=True)
        stream.synchronize()

    for _ in range(2):
        e2e_step()
    n_e2e = max(3, min(args.steps, 10))
    e2e_times = []
    for _ in range(n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_serial_s = max_over_ranks(statistics.mean(e2e_times), world)

    # Frames pipelined as a renderer would run them: the read-back of frame i
    # (copy stream, into its own pinned buffers) overlaps the upload, culling
    # and tracing of frame i + 1 (second set of device outputs); each frame
    # still uploads its primitives and reads its full result back, and L2 is
    # flushed before every frame inside the timed region.
    outs = [dict(depth=r.depth, normal=r.normal, evals=r.evals, flags=r.flags),
            {k: torch.empty_like(v) for k, v in (("depth", r.depth), ("normal", r.normal), ("evals", r.evals),
                                                 ("flags", r.flags))}]
    hosts = [host, {k: torch.empty(v.numel(), dtype=v.dtype, pin_memory=True) for k, v in host.items()}]
    copy_stream = torch.cuda.Stream()
    traced = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_frames(n):
        for i in range(n):
            b = i & 1
            stream.wait_event(copied[b])   # buffer b's previous read-back is done
            flush.zero_()
            st.st_scene_update_prims(r.h, ids, params, stream)
            r.build_tiles()
            o = outs[b]
            st.st_trace(r.h, cam, r.tiles, opts, o["depth"], o["normal"], o["evals"], o["flags"], None, stream)
            traced[b].record(stream)
            copy_stream.wait_event(traced[b])
            with torch.cuda.stream(copy_stream):
                for k in ("depth", "normal", "evals", "flags"):
                    hosts[b][k].copy_(o[k], non_blocking=True)
            copied[b].record(copy_stream)
        copy_stream.synchronize()
        stream.synchronize()

    e2e_frames(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_frames(n_e2e)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, world)

    if rank == 0:
        rays = W * H * world   # whole job: every rank traces the same frame
        peaks = measured_peaks()
        sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
        peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12

        def summary(res, W=W, H=H):
            cnt = res["cnt"]
            ms = res["ms_per_step"]
            trace_s = statistics.mean(res["trace_ms"]) / 1e3
            return {"rays_per_s": whole_job_rate(W * H, world, ms / 1e3), "ms_per_step": ms,
                    "prim_evals_per_s": cnt[:, 1].mean() * world / (ms / 1e3),
                    "trace_ms": trace_s * 1e3, "build_tiles_ms": statistics.mean(res["tiles_ms"]),
                    "steps_per_ray": cnt[:, 0].mean() / (W * H),
                    "rejected_steps_per_ray": cnt[:, 5].mean() / (W * H),
                    "fp32_tflops": cnt[:, 3].mean() / trace_s / 1e12,
                    "evaluated_fp32_tflops": cnt[:, 9].mean() / trace_s / 1e12,
                    "evaluated_nodes_per_step": cnt[:, 8].mean() / max(cnt[:, 0].mean(), 1.0),
                    "device_error_flags": int(cnt[:, 7].max())}

        per_mode = {name: summary(res) for name, res in results.items()}
        hs = per_mode[head]
        achieved = hs["fp32_tflops"]
        traffic = recorded_traffic(args.workload, head)
        line = {
            "metric": METRIC, "value": hs["rays_per_s"], "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hs["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(cfg, step_mode=head, max_new_per_turn=args.max_new,
                           parallelism="replicas" if world > 1 else "single GPU",
                           l2="flushed between timed steps (256 MB write outside the timed events)"),
            "prim_evals_per_s": hs["prim_evals_per_s"],
            "modes": per_mode,
            "roofline": {"bound": "alu", "kernel": f"k_trace<{head}>", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                         "evaluated": {"achieved": hs["evaluated_fp32_tflops"],
                                       "frac": hs["evaluated_fp32_tflops"] / peak_tflops},
                         "peak_note": f"FP32 FMA pipe: {props.multi_processor_count} SMs x 128 lanes x 2 flops x "
                                      f"{sm_mhz:.0f} MHz (max SM clock); achieved = flops of the field "
                                      "evaluations of Algorithm 1's pruned views on live ray-steps (fixed per-node "
                                      "counts) / st_trace event time; 'evaluated' = flops of the nodes actually "
                                      "evaluated (the views without the subtrees their usage rewrite discards)"},
            "e2e": {"value": whole_job_rate(W * H, world, e2e_s), "unit": "rays/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "frames": n_e2e,
                    "pipelining": "read-back of frame i overlaps frame i+1 (copy stream, two output buffers)",
                    "serial_value": whole_job_rate(W * H, world, e2e_serial_s)},
            "gpu_launches": results[head]["launches"],
            "clocks": clocks,
        }
        if "plain" in per_mode and head != "plain":
            line["learned_vs_plain" if head == "learned" else f"{head}_vs_plain"] = (
                hs["rays_per_s"] / per_mode["plain"]["rays_per_s"])
        if agreement_all:
            line["agreement_with_plain"] = agreement_all
        if secondary:
            sw, sh = secondary["cam"].width, secondary["cam"].height
            s_modes = {name: summary(res, sw, sh) for name, res in secondary["res"].items()}
            sh_ = s_modes[head]
            sec = {"workload": secondary["cfg"]["workload"], "prims": secondary["cfg"]["prims"],
                   "resolution": secondary["cfg"]["resolution"], "steps": secondary["steps"],
                   "value": sh_["rays_per_s"], "unit": "rays/s", "prim_evals_per_s": sh_["prim_evals_per_s"],
                   "modes": s_modes,
                   "roofline": {"bound": "alu", "kernel": f"k_trace<{head}>", "achieved": sh_["fp32_tflops"],
                                "peak": peak_tflops, "unit": "TFLOP/s", "frac": sh_["fp32_tflops"] / peak_tflops,
                                "traffic": recorded_traffic("clustered1080p", head),
                                "evaluated": {"achieved": sh_["evaluated_fp32_tflops"],
                                              "frac": sh_["evaluated_fp32_tflops"] / peak_tflops}},
                   "agreement_with_plain": secondary["agreement"], "clocks": secondary["clocks"]}
            if "plain" in s_modes and head != "plain":
                sec[f"{head}_vs_plain"] = sh_["rays_per_s"] / s_modes["plain"]["rays_per_s"]
            line["secondary"] = sec
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(scene, cam, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        dist.destroy_process_group()


TUNE_CACHE = ROOT / "paper_2304_09673_b300" / "tune_b300.json"


def run_batch(args):
    """64 seeded scenes (N log-uniform in [32, 4096], resolutions from
    {256^2, 512^2, 1280x720, 1920x1080}) rendered by one CUDA-graph replay
    per step (batched culling + one persistent trace launch, autotuned tile
    and subfrustum sizes) against 64 sequential st_build_tiles + st_trace
    calls (tile 16, default subfrustum sizes), plain step, same eps."""
    import numpy as np
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local if world > 1 else 0)
    from paper_2304_09673_b300 import build as b
    b.build()
    from paper_2304_09673_b300 import scenegen as sg
    from paper_2304_09673_b300 import st
    n = args.batch_scenes
    work = [sg.workload_batch(i) for i in range(n)]
    scenes = [w[0] for w in work]
    cams = [w[1] for w in work]
    stream = torch.cuda.current_stream()
    handles = [st.st_scene_create(s) for s in scenes]
    dev = torch.device("cuda")
    outs = dict(depth=[], normal=[], evals=[], flags=[])
    for c in cams:
        px = c.width * c.height
        outs["depth"].append(torch.empty(px, device=dev))
        outs["normal"].append(torch.empty(px * 3, device=dev))
        outs["evals"].append(torch.empty(px, dtype=torch.int32, device=dev))
        outs["flags"].append(torch.empty(px, dtype=torch.uint8, device=dev))
    rays = sum(c.width * c.height for c in cams)
    opts = st.make_opts(**TRACE_EXTRA)
    t0 = time.time()
    batch = st.st_batch_create(handles, cams, opts, outs["depth"], outs["normal"], outs["evals"], outs["flags"],
                               autotune_cache=TUNE_CACHE, stream=stream)
    plan_s = time.time() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    def batched():
        st.st_batch_render(batch)

    def sequential():
        for i in range(n):
            t = st.st_build_tiles(handles[i], cams[i], 16, stream)
            st.st_trace(handles[i], cams[i], t, opts, outs["depth"][i], outs["normal"][i], outs["evals"][i],
                        outs["flags"][i], None, stream)

    sampler = ClockSampler(None) if rank == 0 else None
    l0 = st.st_kernel_launches()
    batch_ms = timed(batched)
    launches = (st.st_kernel_launches() - l0) // (args.steps + args.warmup)
    clocks = sampler.stop() if sampler else None
    seq_ms = timed(sequential)
    tiles = [st.st_batch_tiles(batch, i) for i in range(n)]
    st.st_batch_destroy(batch)
    for h in handles:
        st.st_scene_destroy(h)
    bm, sm = statistics.mean(batch_ms), statistics.mean(seq_ms)
    if rank == 0:
        line = {"metric": "aggregate rays/s, 64-scene batch in one CUDA graph vs 64 sequential plain launches",
                "value": rays / (bm / 1e3), "unit": "rays/s", "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": bm, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{n} seeded scenes (seed 1000+i), N log-uniform in [32, 4096], depth <= "
                                       "min(20, ceil(log2 N) + 4), resolution uniform in {256^2, 512^2, 1280x720, "
                                       "1920x1080}; plain step, eps 1e-4",
                           "rays_per_step": rays, "prims_total": int(sum(s.n_prims for s in scenes)),
                           "tiles_chosen": {str(t): tiles.count(t) for t in sorted(set(tiles))},
                           "l2": "flushed between timed steps (256 MB write outside the timed events)"},
                "sequential": {"value": rays / (sm / 1e3), "unit": "rays/s", "ms_per_step": sm,
                               "what": "per scene st_build_tiles(tile 16) + st_trace, host-synchronised sizing"},
                "speedup_vs_sequential": sm / bm, "plan_s": plan_s, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_table1(args):
    """The structure of the paper's Table 1 on synthetic stand-ins for its
    models: frame time (A-buffer + tracing, plain step, same eps) of the
    synchronized pipeline (st_build_tiles + st_trace) against per-pixel
    processing over a full-resolution A-buffer with f_A evaluated at every
    step by Algorithm 1 with fast ancestor pointers ("FastPtr/Full") or parent
    pointers ("ParentPtr/Full"): st_build_tiles + st_build_dexels +
    st_trace_dexels."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2304_09673_b300 import build as b
    b.build()
    from paper_2304_09673_b300 import scenegen as sg
    from paper_2304_09673_b300 import st
    cases = [("150-primitive seeded blobtree (depth <= 12, seed 150), 1720x1376", sg.make_scene(150, 12, 150),
              sg.default_camera(1720, 1376)),
             ("150-primitive left comb (left-heavy tree, depth 149, seed 150), 1720x1376", sg.make_comb(150, 150),
              sg.default_camera(1720, 1376)),
             ("1,024-primitive seeded blobtree (depth <= 14, seed 100), 1920x1080", sg.workload_1080p(100),
              sg.default_camera(1920, 1080))]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opts = st.make_opts()
    sampler = ClockSampler(None)
    launches0 = st.st_kernel_launches()
    results = []
    for what, scene, cam in cases:
        W, H = cam.width, cam.height
        r = st.Renderer(scene, cam, tile=16, stream=stream)

        def sync_step():
            r.build_tiles()
            st.st_trace(r.h, cam, r.tiles, opts, r.depth, r.normal, r.evals, r.flags, r.counters, stream)

        def dexel_step(trav):
            def fn():
                t = st.st_build_tiles(r.h, cam, 16, stream)
                dx = st.st_build_dexels(r.h, cam, t, stream)
                st.st_trace_dexels(r.h, cam, dx, opts, trav, r.depth, r.normal, r.evals, r.flags, r.counters,
                                   stream)
            return fn

        row = {"workload": what}
        masks = {}
        for name, fn in (("synchronized", sync_step), ("fastptr_full", dexel_step(st.ST_TRAVERSE_FAST)),
                         ("parentptr_full", dexel_step(st.ST_TRAVERSE_PARENT))):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ms, cnt = [], None
            for _ in range(args.steps):
                flush.zero_()
                r.counters.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                cnt = r.counters.cpu().numpy().astype(np.float64)
            masks[name] = (r.flags & 1).clone()
            row[name] = {"ms_per_frame": statistics.mean(ms), "rays_per_s": W * H / (statistics.mean(ms) / 1e3),
                         "steps_per_ray": cnt[0] / (W * H), "prim_evals_per_ray": cnt[1] / (W * H),
                         "device_error_flags": int(cnt[7])}
            if name != "synchronized":
                row[name]["operator_visits_per_ray"] = cnt[2] / (W * H)
        base = row["synchronized"]["ms_per_frame"]
        row["fastptr_over_synchronized"] = row["fastptr_full"]["ms_per_frame"] / base
        row["parentptr_over_synchronized"] = row["parentptr_full"]["ms_per_frame"] / base
        row["mask_mismatch_frac_vs_synchronized"] = {
            k: float((masks[k] != masks["synchronized"]).float().mean().item()) for k in ("fastptr_full", "parentptr_full")}
        results.append(row)
        r.close()
    clocks = sampler.stop()
    line = {"metric": "frame time of per-pixel ParentPtr/Full over the synchronized pipeline (Table 1 structure)",
            "value": results[0]["parentptr_over_synchronized"], "unit": "x", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results[0]["synchronized"]["ms_per_frame"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Table 1 variants on two seeded scenes (plain step, eps 1e-4, max 256 steps, "
                                   "tile 16 for the synchronized A-buffer)",
                       "l2": "flushed between timed steps (256 MB write outside the timed events)"},
            "cases": results, "gpu_launches": st.st_kernel_launches() - launches0, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_blend(args):
    """Blend localisation (the paper's blend experiment on 8..16 spheres):
    frame time (st_build_tiles + st_trace, plain step) at 1920x1080 as
    spheres are added, for a sharp union, the compact smooth union with two
    blend ranges and the same smooth union without compact support
    ("classical": unbounded range of interest, every sphere active
    everywhere)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2304_09673_b300 import build as b
    b.build()
    from paper_2304_09673_b300 import scenegen as sg
    from paper_2304_09673_b300 import st
    cam = sg.default_camera(1920, 1080)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opts = st.make_opts()
    settings = [("sharp union", "sharp", 0.0), ("compact blend k=0.06", "compact", 0.06),
                ("compact blend k=0.12", "compact", 0.12), ("classical blend k=0.06", "classical", 0.06)]
    ns = (8, 10, 12, 14, 16)
    sampler = ClockSampler(None)
    launches0 = st.st_kernel_launches()
    curves = {}
    for label, blend, k in settings:
        pts = []
        for n in ns:
            r = st.Renderer(sg.blend_spheres(n, blend, k), cam, tile=16, stream=stream)
            for _ in range(args.warmup):
                r.render(opts)
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                flush.zero_()
                r.counters.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.build_tiles()
                st.st_trace(r.h, cam, r.tiles, opts, r.depth, r.normal, r.evals, r.flags, r.counters, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            c = r.counters.cpu().numpy().astype(np.float64)
            pts.append({"spheres": n, "ms_per_frame": statistics.mean(ms),
                        "prim_evals_per_ray": c[1] / (cam.width * cam.height),
                        "mean_tile_list": float(r.tiles.n_entries) / (r.tiles.tiles_x * r.tiles.tiles_y),
                        "device_error_flags": int(c[7])})
            r.close()
        slope = float(np.polyfit(ns, [q["ms_per_frame"] for q in pts], 1)[0])
        curves[label] = {"points": pts, "ms_per_added_sphere": slope}
    clocks = sampler.stop()
    c16 = {lab: v["points"][-1]["ms_per_frame"] for lab, v in curves.items()}
    line = {"metric": "frame time with 16 spheres, classical smooth blend over compact blend (blend localisation)",
            "value": c16["classical blend k=0.06"] / c16["compact blend k=0.06"], "unit": "x", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": c16["compact blend k=0.06"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8..16 spheres (radius 0.12, 4x4 grid, spacing 0.2) under a balanced union tree, "
                                   "1920x1080, tile 16, plain step, eps 1e-4",
                       "l2": "flushed between timed steps (256 MB write outside the timed events)"},
            "curves": curves, "gpu_launches": st.st_kernel_launches() - launches0, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1080p")
    ap.add_argument("--modes", default="learned,plain,overrelax,crossing",
                    help="step modes to time; the first one is the headline value")
    ap.add_argument("--max-new", type=int, default=32, help="new primitives per subfrustum")
    ap.add_argument("--cta-min-view", type=int, default=0,
                    help="st_trace_opts.cta_eval_min_view (0: library default, < 0: no CTA-split evaluation)")
    ap.add_argument("--trace-opt", action="append", default=[], metavar="NAME=VALUE",
                    help="another st_trace_opts field for every mode (repeatable), e.g. heavy_split_len=2000")
    ap.add_argument("--batch-scenes", type=int, default=64, help="scenes of the batch64 workload")
    ap.add_argument("--res", default=None, help="WxH: render the single-scene workload at another resolution")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 10,000-primitive clustered 1920x1080 line of the default workload")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-pixels", type=int, default=8192,
                    help="oracle rays per step of the reference arm")
    args = ap.parse_args()
    if args.cta_min_view:
        TRACE_EXTRA["cta_eval_min_view"] = args.cta_min_view
    for kv in args.trace_opt:
        k, v = kv.split("=", 1)
        TRACE_EXTRA[k] = float(v) if "." in v else int(v)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "table1":
        run_table1(args)
    elif args.workload == "blend":
        run_blend(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
