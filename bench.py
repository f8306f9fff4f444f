#!/usr/bin/env python
"""Benchmark of differentiable Voronoi-foam ray tracing on GB300.

One step = forward render + MSE loss gradient + backward (re-walk with
gradient scatter) of one frame of the workload, all in the library's CUDA
kernels, with the scene resident in HBM.  The headline value is forward +
backward throughput in Mrays/s on the 3,000,000-site foam at 1920x1080
(plain FP32 attributes); forward-only, BF16/FP16 attribute storage, the
4,096-site and 1M-site workloads, the 8-camera batch and serving latency are
reported beside it.  The CPU-baseline leg (rank 0, one GPU) also compares the
GPU with the FP64 oracle on sampled pixels: per-dtype image and gradient
errors and the near-degenerate ray counts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own seeded view of the same scene (weak
scaling) and the site gradients are summed across ranks with one NCCL
all-reduce per step.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
import argparse
import copy
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd & fwd+bwd at 3M cells vs plain FP32; serving p50/p99 latency"
RECORD_STEPS = 384  # walk-record steps per ray kept by the training step
UNIT = "Mrays/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)  # ~1 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c1"])
    ap.add_argument("--sites", type=int, default=0, help="override the workload's site count")
    ap.add_argument("--crop", default="", metavar="WxH",
                    help="render only the centre WxH window of the workload's frame (the same rays as "
                         "those pixels of the full frame; for profiler captures of a smaller case)")
    ap.add_argument("--no-extras", action="store_true", help="skip dtype variants / serving")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjacency-only", action="store_true",
                    help="time only the GPU adjacency build of --sites uniform sites (profiling)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
WORKLOADS = {
    "c3": dict(desc="3M sites uniform in [-1,1]^3, SH deg 3, 1920x1080, camera at origin",
               sites=3_000_000),
    "c2": dict(desc="1M sites Gaussian mixture + uniform, SH deg 3, 1280x720", sites=1_000_000),
    "c1": dict(desc="4096 sites uniform, SH deg 0, 64x64", sites=4096),
}


def rank_camera(workload, rank):
    """Rank 0 uses the workload's camera; other ranks rotate it about the
    vertical axis by a seeded angle (their own views of the same scene)."""
    import numpy as np
    from paper_2502_01157_gb300 import scenes as S

    cam = S.config_cameras(workload)[0]
    if rank == 0:
        return cam
    a = np.random.default_rng(7000 + rank).uniform(0, 2 * math.pi)
    R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    c2w = cam.c2w.astype(np.float64).copy()
    c2w[:, :3] = R @ c2w[:, :3]
    return S.Camera(c2w, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.t_near, cam.t_far)


def crop_camera(cam, crop):
    """The centre ``WxH`` window of ``cam``'s image as a camera of its own:
    same pose and focal lengths, principal point shifted by the window's
    offset, so each of its rays is the full frame's ray through that pixel."""
    from paper_2502_01157_gb300 import scenes as S

    w, h = (int(v) for v in crop.lower().split("x"))
    w, h = min(w, cam.width), min(h, cam.height)
    x0, y0 = (cam.width - w) // 2, (cam.height - h) // 2
    return S.Camera(cam.c2w, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.t_near, cam.t_far)


def bytes_per_step(k_bar, deg, attr_bytes):
    """Algorithmic bytes one forward cell step reads with no reuse: CSR
    offsets 8 B, K faces x 16 B (a neighbour position and id), density and
    the SH row (deg 3 FP32: 8 + 16 x 15.5 + 4 + 192 = 452 B)."""
    return 8 + 16 * k_bar + attr_bytes + 3 * (deg + 1) ** 2 * attr_bytes


def bwd_extra_bytes_per_step(deg):
    """Backward: read-modify-write of the FP32 gradients one step touches:
    density 4 B, SH 12 (deg+1)^2 B and two site positions (one crossing)
    24 B (deg 3: 2 x 220 = 440 B)."""
    return 2 * (4 + 12 * (deg + 1) ** 2 + 24)


# ncu counters of the renderer's kernels, per cell step, from the captures
# summarised in profiles/ (valid only for the kernel sources they were taken on)
COUNTERS = os.path.join(ROOT, "profiles", "kernel_counters.txt")
L1_BYTES_PER_CLK = 128   # L1 load data path: one 128-byte wavefront per clock per SM


def kernel_source_hash():
    """Hash of the CUDA sources the renderer's kernels are built from, with
    comments removed and white space collapsed (a comment edit keeps the
    counters measured on the same code)."""
    import hashlib
    import re

    tok = re.compile(r'("(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\')|//[^\n]*|/\*.*?\*/', re.S)
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2502_01157_gb300", "csrc")
    for name in ("rf_host.h", "rf_internal.cuh", "rf_kernels.cuh", "rf_render.cu", "rf_scene.cu"):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            code = tok.sub(lambda m: m.group(1) or " ", f.read())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:12]


def kernel_counters(kernel, workload):
    """{dram, lts, l1_wavefronts}: bytes / wavefronts per cell step, and the
    L1 LSU pipe and occupancy percentages, of ``kernel`` on ``workload`` from
    profiles/kernel_counters.txt, or None when they were taken on other
    kernel sources."""
    if not os.path.exists(COUNTERS):
        return None
    src = kernel_source_hash()
    for line in open(COUNTERS):
        f = line.split()
        if line.startswith("#") or len(f) < 9:
            continue
        if f[0] == kernel and f[1] == workload and f[2] == src:
            steps = float(f[3])
            return {"dram_bytes_per_step": float(f[4]) / steps, "lts_bytes_per_step": float(f[5]) / steps,
                    "l1_wavefronts_per_step": float(f[6]) / steps, "l1_lsu_pct": float(f[7]),
                    "occupancy_pct": float(f[8]), "source": src}
    return None


def l2_read_peak(dev, mb=48, k=32, reps=20):
    """L2 read throughput: a column sum over k rows of a 48 MB buffer whose
    rows overlap (offsets 32 KB apart), so the k x 48 MB of reads are served
    from the 129 MB L2 after the first pass; bytes read over CUDA-event time,
    best of 3.  (A device copy within an L2-sized buffer pair reaches only
    ~7.5 TB/s: its writes go back to DRAM.)"""
    import torch

    base = torch.ones(mb << 18, device=dev)
    n = base.numel() - (k - 1) * 8192
    view = torch.as_strided(base, (k, n), (8192, 1))
    view.sum(0)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            view.sum(0)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, k * n * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.path = tempfile.mktemp(prefix="rf_clocks_", suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 8:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        import statistics

        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------
def oracle_step(scene, cam, pixels, target):
    """One FP64 oracle training step on ``pixels``: forward, MSE gradient,
    backward (``scene`` prepared once: FP64 arrays and nn(o) are not redone)."""
    import oracle

    o = oracle.render(scene, cam, pixels=pixels, tau=0.0)
    g = 2.0 * (o["rgb"] - target[pixels]) / (3 * len(pixels))
    oracle.render_bwd(scene, cam, g, pixels=pixels)


def cpu_baseline(scene, cam, target, budget_s=12.0):
    """Oracle fwd+bwd on a growing sample of pixels until ~budget_s of work."""
    import numpy as np
    import oracle

    R = cam.n_rays
    rng = np.random.default_rng(11)
    n = 2048
    P = oracle.prepare(scene)
    P.start_info(cam)
    while True:
        px = np.sort(rng.choice(R, size=min(n, R), replace=False)).astype(np.int64)
        t = time.perf_counter()
        oracle_step(P, cam, px, target)
        dt = time.perf_counter() - t
        if dt >= budget_s or n >= R or n >= (1 << 22):
            break
        n = int(n * min(8.0, max(2.0, budget_s / max(dt, 1e-3))))
    return {"value": len(px) / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle fwd+bwd (MSE loss) on {len(px)} random pixels of the "
                      f"{cam.width}x{cam.height} view, {dt:.1f} s (scene converted to FP64 and "
                      f"nn(o) found once, outside the timing)"}


def cpu_adjacency_baseline(pos, budget_s=6.0):
    """The FP64 adjacency oracle (face polygons, k-d tree candidates) on a
    growing random sample of sites of the same scene."""
    import numpy as np
    import oracle
    from oracle import adjacency as A

    rng = np.random.default_rng(12)
    n = 2000
    while True:
        sites = rng.choice(len(pos), size=min(n, len(pos)), replace=False)
        t = time.perf_counter()
        A.voronoi_neighbors(pos, sites=sites)
        dt = time.perf_counter() - t
        if dt >= budget_s or n >= len(pos):
            break
        n = int(n * min(8.0, max(2.0, budget_s / max(dt, 1e-3))))
    return {"value": len(sites) / dt / 1e6, "unit": "Msites/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"FP64 face-polygon adjacency of {len(sites)} random sites of the "
                                        f"{len(pos)}-site scene, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2502_01157_gb300 import scenes as S

    scene = oracle.prepare(S.config_scene(args.workload, n_sites=args.sites or None))
    cam = rank_camera(args.workload, 0)
    scene.start_info(cam)  # nn(o) once, like the FP64 conversion
    target = S.random_target(cam.n_rays, 2024)
    rng = np.random.default_rng(5)
    sample = 8192 if args.workload != "c1" else cam.n_rays
    times = []
    for k in range(args.warmup + args.steps):
        px = np.sort(rng.choice(cam.n_rays, size=sample, replace=False)).astype(np.int64)
        t = time.perf_counter()
        oracle_step(scene, cam, px, target)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    tot = sum(times)
    v = sample * len(times) / tot / 1e6
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}",
                       "rays_per_step": sample, "sampled_from_rays": cam.n_rays},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{sample} random pixels per step of the "
                                       f"{cam.width}x{cam.height} view, fwd+bwd (scene converted to "
                                       f"FP64 and nn(o) found once, before the steps)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------
SERVE_RATES = (50, 100, 200, 500, 1000, 2000)   # req/s: 2,000 requests or 10 s each
SERVE_REQUESTS = 2000
SERVE_SECONDS = 10.0


def effects_extras(S, rf, foam, cam, target, scale, loss, grads, args, dev):
    """Ray-based effects (Fig. 2) on the main workload's scene and image size:
    a 200-degree equidistant fisheye, a rolling shutter, and a clear-glass and a
    mirror sphere of radius 0.25 in front of the camera (FP32 attributes)."""
    import numpy as np
    import torch

    R = cam.n_rays
    fish = S.fisheye(cam.width, cam.height, 200.0, c2w=cam.c2w)
    roll = S.Camera(cam.c2w, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                    shutter=(0.02, 0.0, 0.01))
    centre = tuple(np.asarray(cam.c2w, np.float64) @ np.array([0.0, 0.0, 0.5, 1.0]))
    glass = S.Sphere(centre, 0.25, ior=1.5, max_bounces=4)
    mirror = S.Sphere(centre, 0.25, ior=0.0, max_bounces=4)
    out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
               depth=torch.empty(R, device=dev))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {"recipe": "c3 scene, 1920x1080: fisheye 200 deg; rolling shutter (0.02, 0, 0.01) over the "
                     "frame; glass (n = 1.5) / mirror sphere r = 0.25 at 0.5 along the view axis; the "
                     f"training step rebuilds its backward walk from a {RECORD_STEPS}-step segment record"}
    # the training step keeps the forward's walk record, as the headline step does
    tout = dict(out, walk_record=(torch.empty(rf.walk_record_bytes([cam], RECORD_STEPS), dtype=torch.uint8,
                                              device=dev), RECORD_STEPS))
    for name, c, sph in (("fisheye", fish, None), ("rolling_shutter", roll, None),
                         ("glass_sphere", cam, glass), ("mirror_sphere", cam, mirror),
                         ("fisheye_glass", fish, glass)):
        def fstep():
            foam.render([c], out=tout, effects=sph)
            d_rgb, _ = rf.mse_grad(tout["rgb"], target, scale, loss)
            foam.backward([c], tout, d_rgb, grads=grads, effects=sph)

        chk = foam.render([c], steps=True, effects=sph)
        k = float(chk["steps"].float().mean().item())
        for _ in range(2):
            fstep()
        torch.cuda.synchronize()
        a, b, e = ev(), ev(), ev()
        a.record()
        for _ in range(args.steps):
            foam.render([c], out=out, effects=sph)
        b.record()
        for _ in range(args.steps):
            fstep()
        e.record()
        torch.cuda.synchronize()
        res[name] = {"fwd_mrays_s": R / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6,
                     "fwdbwd_mrays_s": R / (b.elapsed_time(e) / args.steps * 1e-3) / 1e6,
                     "cell_steps_per_ray": k}
    return res


def adjacency_extras(rf, scene, mix_scene, args, dev):
    """GPU Voronoi adjacency (the neighbour lists the walk needs) of the main
    scene and of the 3M-site mixture: a full build, and an incremental rebuild
    after every site moved by a tenth of the mean spacing (default domain:
    the sites' box grown by 5%).  Each build includes its three waits for the
    GPU; times are the median of the repetitions."""
    import statistics

    import torch

    out = {}
    b = rf.Adjacency()
    try:
        for name, sc in (("main", scene), ("mixture_3m", mix_scene)):
            if sc is None:
                continue
            pos = torch.from_numpy(sc.pos).to(dev)
            spacing = float(torch.prod(pos.max(0).values - pos.min(0).values) / len(pos)) ** (1 / 3)
            moved = pos + (0.1 * spacing) * torch.randn(pos.shape, device=dev,
                                                        generator=torch.Generator(dev).manual_seed(3))

            def timed(fn, reps):
                ts = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    fn()
                    torch.cuda.synchronize()
                    ts.append((time.perf_counter() - t) * 1e3)
                return statistics.median(ts)

            full = timed(lambda: b.build(pos), 3)
            st = dict(b.stats)
            inc = timed(lambda: (b.build(pos), b.build(moved, incremental=True)), 2) - full
            out[name] = {"n_sites": len(pos), "full_build_ms": full, "msites_s": len(pos) / full / 1e3,
                         "incremental_ms": inc, "n_edges": st["n_edges"], "max_degree": st["max_degree"],
                         "fp64_tests": st["fp64_tests"], "wide_sites": st["wide_sites"],
                         "failed_sites": st["failed_sites"]}
    finally:
        b.close()
    return out


def mixture_extras(scene, args, dev):
    """The 3M-site mixture scene: 8 mixed-resolution cameras forward+backward
    in one launch (FP32), batched forward FP32 vs BF16 on the serving poses,
    and open-loop Poisson serving with BF16 attributes."""
    import numpy as np
    import torch
    from paper_2502_01157_gb300 import rf
    from paper_2502_01157_gb300 import scenes as S
    from paper_2502_01157_gb300.serve import Server, run_closed_loop, run_open_loop

    ev = lambda: torch.cuda.Event(enable_timing=True)
    foam = rf.Foam.from_scene(scene)
    cams = S.config_cameras("c4")
    R = rf.n_rays_of(cams)
    target = torch.rand(R, 3, device=dev)
    grads = dict(density=torch.zeros(scene.n_sites, device=dev),
                 sh=torch.zeros(scene.n_sites, 16, 3, device=dev),
                 pos=torch.zeros(scene.n_sites, 3, device=dev))
    out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
               depth=torch.empty(R, device=dev))
    tout = dict(out, walk_record=(torch.empty(rf.walk_record_bytes(cams, RECORD_STEPS), dtype=torch.uint8,
                                              device=dev), RECORD_STEPS))

    def step(shared=True):
        foam.render(cams, out=tout)
        d, _ = rf.mse_grad(tout["rgb"], target, 1.0 / (3 * R))
        foam.backward(cams, tout, d, grads=grads, shared_cells=shared)

    for _ in range(2):
        step()
        step(False)
    torch.cuda.synchronize()
    n = max(3, args.steps // 2)
    a, b, c, e = ev(), ev(), ev(), ev()
    a.record()
    for _ in range(n):
        foam.render(cams, out=out)
    b.record()
    for _ in range(n):
        step()
    c.record()
    for _ in range(n):
        step(False)
    e.record()
    torch.cuda.synchronize()
    res = {"scene": f"c4/c5 mixture, {scene.n_sites} sites, SH deg 3",
           "c4_cameras": "8 mixed (2x 640x480, 1280x720, 1600x900, 1920x1080) on a radius-12 sphere",
           "c4_rays": R,
           "c4_fwd_fp32_mrays_s": R * n / (a.elapsed_time(b) * 1e-3) / 1e6,
           "c4_fwdbwd_fp32_mrays_s": R * n / (b.elapsed_time(c) * 1e-3) / 1e6,
           "c4_fwdbwd_backward": "shared-cell backward (RF_RENDER_SHARED_CELLS)",
           "c4_fwdbwd_default_backward_fp32_mrays_s": R * n / (c.elapsed_time(e) * 1e-3) / 1e6}
    # serving poses and resolutions; batched forward of 16 of them, FP32 vs BF16
    rng = np.random.default_rng(1005)
    bposes = S.sphere_poses(16, 12.0, 1006)
    batch = [S.pinhole(*S.C5_RESOLUTIONS[k], 60.0, c2w=p) for k, p in zip(rng.integers(0, 4, 16), bposes)]
    Rb = rf.n_rays_of(batch)
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        foam.set_attributes(torch.from_numpy(scene.density).to(dev, dt),
                            torch.from_numpy(scene.sh).to(dev, dt))
        foam.render(batch)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(n):
            foam.render(batch)
        b.record()
        torch.cuda.synchronize()
        res[f"serve_poses_batched_fwd_{name}_mrays_s"] = Rb * n / (a.elapsed_time(b) * 1e-3) / 1e6
    # open-loop Poisson serving with BF16 attributes (set just above): at each
    # rate 2,000 requests or 10 s of arrivals, whichever is fewer
    n_req = SERVE_REQUESTS
    poses = S.sphere_poses(n_req, 12.0, 1005)
    sizes = [S.C5_RESOLUTIONS[k] for k in rng.integers(0, 4, n_req)]
    scams = [S.pinhole(w, h, 60.0, c2w=p) for (w, h), p in zip(sizes, poses)]
    srv = Server(foam, mem_budget_bytes=4 << 30, max_inflight=512, n_streams=4, max_batch=8)
    rates = []
    for k, rate in enumerate(SERVE_RATES):
        m = int(min(SERVE_REQUESTS, rate * SERVE_SECONDS))
        arr = S.poisson_arrivals(float(rate), m, 500 + k)
        st = run_open_loop(srv, scams[:m], arr, deadline_s=60.0)
        offered_rays = sum(c.n_rays for c in scams[:m])
        rates.append({"rate_req_s": rate, "offered": m, "offered_mrays_s": offered_rays / arr[-1] / 1e6,
                      "completed": st["completed"], "rejected": st["rejected_open_loop"],
                      "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                      "mrays_s": st["mrays_s"], "mean_batch": st["mean_batch"],
                      "max_busy_streams": st["max_busy_streams"]})
    # saturation: 64 requests kept in the server for 3 s
    sat = run_closed_loop(srv, scams, 64, 3.0)
    srv.close()
    res["serving_bf16"] = {"budget_gb": 4, "streams": 4, "max_batch": 8,
                           "resolutions": "uniform over 320x240, 640x480, 1280x720, 1920x1080",
                           "poses": "uniform on the radius-12 sphere, looking at the origin",
                           "requests_per_rate": f"min({SERVE_REQUESTS}, {SERVE_SECONDS:.0f} s x rate)",
                           "rates": rates,
                           "saturation": {"inflight": 64, "seconds": 3.0, "completed": sat["completed"],
                                          "mrays_s": sat["mrays_s"], "p50_ms": sat["p50_ms"],
                                          "p99_ms": sat["p99_ms"], "mean_batch": sat["mean_batch"]}}
    foam.close()
    return res


def workload_extras(rf, scene, cam, args, dev, name, shared_cells=False):
    """Throughput of another workload in the headline step's launch
    configuration: forward alone and the training step (forward with a walk
    record, MSE gradient, replayed backward), with cell steps and bytes.
    ``shared_cells``: the training step uses the shared-cell backward (the
    default backward is timed beside it)."""
    import torch

    R = cam.n_rays
    deg = scene.sh_degree
    foam = rf.Foam.from_scene(scene)
    target = torch.rand(R, 3, device=dev, generator=torch.Generator(dev).manual_seed(17))
    grads = dict(density=torch.zeros(scene.n_sites, device=dev),
                 sh=torch.zeros(scene.n_sites, (deg + 1) ** 2, 3, device=dev),
                 pos=torch.zeros(scene.n_sites, 3, device=dev))
    out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
               depth=torch.empty(R, device=dev))
    tout = dict(out, walk_record=(torch.empty(rf.walk_record_bytes([cam], RECORD_STEPS), dtype=torch.uint8,
                                              device=dev), RECORD_STEPS))
    steps_total = int(foam.render([cam], steps=True)["steps"].sum().item())
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(shared=shared_cells):
        foam.render([cam], out=tout)
        d, _ = rf.mse_grad(tout["rgb"], target, 1.0 / (3 * R))
        foam.backward([cam], tout, d, grads=grads, shared_cells=shared)

    # a small frame is launch-bound: time enough iterations for ~0.2 s
    n = max(args.steps, int(2e7 // max(R, 1)))
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    a, b, c = ev(), ev(), ev()
    a.record()
    for _ in range(n):
        foam.render([cam], out=out)
    b.record()
    for _ in range(n):
        step()
    c.record()
    torch.cuda.synchronize()
    fwd_ms = a.elapsed_time(b) / n
    step_ms = b.elapsed_time(c) / n
    default_step_ms = None
    if shared_cells:
        for _ in range(2):
            step(False)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(n):
            step(False)
        b.record()
        torch.cuda.synchronize()
        default_step_ms = a.elapsed_time(b) / n
    # the same calls replayed from CUDA graphs, each captured once: a small
    # frame is launch-bound, and a replay issues the calls' memsets and kernels
    # without the host's per-call work
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            foam.render([cam], out=out)
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g_fwd, g_step = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_fwd):
        foam.render([cam], out=out)
    with torch.cuda.graph(g_step):
        step()
    for _ in range(3):
        g_fwd.replay()
        g_step.replay()
    torch.cuda.synchronize()
    a, b, c = ev(), ev(), ev()
    a.record()
    for _ in range(n):
        g_fwd.replay()
    b.record()
    for _ in range(n):
        g_step.replay()
    c.record()
    torch.cuda.synchronize()
    gfwd_ms = a.elapsed_time(b) / n
    gstep_ms = b.elapsed_time(c) / n
    k_bar = scene.n_edges / scene.n_sites
    fb = bytes_per_step(k_bar, deg, 4)
    res = {"workload": f"{name}: {WORKLOADS[name]['desc']}", "rays": R, "n_sites": scene.n_sites,
           "backward": "shared-cell backward (RF_RENDER_SHARED_CELLS)" if shared_cells else "default backward",
           "fwdbwd_default_backward_mrays_s": R / default_step_ms / 1e3 if default_step_ms else None,
           "graph_fwd_ms": gfwd_ms, "graph_fwd_mrays_s": R / gfwd_ms / 1e3,
           "graph_fwdbwd_ms": gstep_ms, "graph_fwdbwd_mrays_s": R / gstep_ms / 1e3,
           "cell_steps_per_ray": steps_total / R, "iterations": n,
           "fwd_ms": fwd_ms, "fwd_mrays_s": R / fwd_ms / 1e3, "fwd_cell_steps_per_s": steps_total / fwd_ms * 1e3,
           "fwdbwd_ms": step_ms, "fwdbwd_mrays_s": R / step_ms / 1e3,
           "fwdbwd_cell_steps_per_s": steps_total / step_ms * 1e3,
           "fwd_algorithmic_gbs": fb * steps_total / fwd_ms / 1e6,
           "fwdbwd_algorithmic_gbs": (2 * fb + bwd_extra_bytes_per_step(deg)) * steps_total / step_ms / 1e6,
           "bytes_per_cell_step": {"fwd": fb, "fwd+bwd": 2 * fb + bwd_extra_bytes_per_step(deg)}}
    foam.close()
    return res


def oracle_comparisons(rf, scene, cam, c1_scene, c2_scene, args, dev):
    """The GPU against the FP64 oracle on sampled pixels (CPU-baseline leg):

    * precision: for FP32 / BF16 / FP16 attribute storage, the image RMSE
      against the oracle on the same rounded attributes (the compute error),
      against the oracle on the FP32 originals (the storage error), and the
      gradient's relative L2 error against the oracle's (loss on the sampled
      rays without a near-degenerate flag, the forward's walk record replayed);
    * the near-degenerate ray classes of the 4,096-site frame (all rays, with
      the GPU's visited cells checked against the oracle's) and of the
      sampled pixels of the other frames;
    * the oracle's own forward (4,096 sites) and fwd+bwd (1M sites) timings on
      the same rays as the GPU's."""
    import numpy as np
    import torch
    import oracle

    res = {}
    rng = np.random.default_rng(31)
    R = cam.n_rays
    px = np.sort(rng.choice(R, size=1500, replace=False)).astype(np.int64)
    pxt = torch.from_numpy(px).to(dev)
    P32 = oracle.prepare(scene)
    ref32 = oracle.render(P32, cam, pixels=px)
    flags = {"c3_sample": oracle.flag_counts(ref32["flags"])}
    keep = ~ref32["degen"]
    w = rng.normal(size=(int(keep.sum()), 3))
    prec = {}
    torch_dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
    foam = rf.Foam.from_scene(scene)
    for name, dt in torch_dt.items():
        if name == "f32":
            Pr, refr = P32, ref32
        else:
            sc_r = copy.copy(scene)
            sc_r.density = torch.from_numpy(scene.density).to(dt).float().numpy()
            sc_r.sh = torch.from_numpy(scene.sh).to(dt).float().numpy()
            Pr = oracle.prepare(sc_r)
            refr = oracle.render(Pr, cam, pixels=px)
        foam.set_attributes(torch.from_numpy(scene.density).to(dev, dt), torch.from_numpy(scene.sh).to(dev, dt))
        out = foam.render([cam], record=RECORD_STEPS)
        g = {k: out[k][pxt].double().cpu().numpy() for k in ("rgb", "trans", "depth")}
        rm = lambda a, b: float(np.sqrt(np.mean((a - b) ** 2)))
        d_rgb = torch.zeros(R, 3, device=dev)
        d_rgb[pxt[torch.from_numpy(keep).to(dev)]] = torch.from_numpy(w).float().to(dev)
        G = foam.backward([cam], out, d_rgb)
        Go = oracle.render_bwd(Pr, cam, w, pixels=px[keep])
        rel = {k: float(np.linalg.norm(G[k].double().cpu().numpy() - Go[k]) / np.linalg.norm(Go[k]))
               for k in ("density", "sh", "pos")}
        prec[name] = {"compute_rmse": {k: rm(g[k], refr[k]) for k in g},
                      "storage_rmse": {k: rm(g[k], ref32[k]) for k in g},
                      "grad_rel_l2": rel}
        del out, G
        if Pr is not P32:
            del Pr
    foam.close()
    res["precision"] = {"sample": f"{len(px)} random pixels of the {cam.width}x{cam.height} frame, "
                                  f"{scene.n_sites} sites; gradients of a random linear loss on the "
                                  f"{int(keep.sum())} unflagged ones, walk record replayed",
                        "bounds": {"compute_rmse": 1e-5, "grad_rel_l2": 1e-3}, **prec}
    # the 4,096-site frame: every ray, cells compared with the oracle's
    if c1_scene is not None:
        from paper_2502_01157_gb300 import scenes as S

        cam1 = S.config_cameras("c1")[0]
        f1 = rf.Foam.from_scene(c1_scene)
        cells, counts = f1.trace(cam1, max_per_ray=256)
        cells, counts = cells.cpu().numpy(), counts.cpu().numpy()
        t = time.perf_counter()
        o1 = oracle.render(c1_scene, cam1, trace=256)
        bad = 0
        for r in range(cam1.n_rays):
            if o1["tie"][r]:
                continue
            n_o, n_g = int(o1["steps"][r]), int(counts[r])
            if o1["stop_tie"][r] and abs(n_o - n_g) <= 1:
                m = min(n_o, n_g, 256)
            elif n_o == n_g:
                m = min(n_o, 256)
            else:
                bad += 1
                continue
            bad += int(not np.array_equal(cells[r, :m], o1["trace_cells"][r, :m]))
        flags["c1"] = dict(oracle.flag_counts(o1["flags"]), cells_mismatched_outside_ties=bad)
        t = time.perf_counter()
        oracle.render(c1_scene, cam1, tau=0.0)
        dt = time.perf_counter() - t
        res["c1_oracle"] = {"fwd_mrays_s": cam1.n_rays / dt / 1e6, "rays": cam1.n_rays,
                            "cores": oracle.num_threads()}
        f1.close()
    if c2_scene is not None:
        from paper_2502_01157_gb300 import scenes as S

        cam2 = S.config_cameras("c2")[0]
        P2 = oracle.prepare(c2_scene)
        px2 = np.sort(rng.choice(cam2.n_rays, size=4096, replace=False)).astype(np.int64)
        o2 = oracle.render(P2, cam2, pixels=px2[:1500])
        flags["c2_sample"] = oracle.flag_counts(o2["flags"])
        target = S.random_target(cam2.n_rays, 77)
        t = time.perf_counter()
        oracle_step(P2, cam2, px2, target)
        dt = time.perf_counter() - t
        res["c2_oracle"] = {"fwdbwd_mrays_s": len(px2) / dt / 1e6, "rays": int(len(px2)),
                            "cores": oracle.num_threads()}
        del P2
    res["near_degenerate"] = {
        "classes": "edge: passes within tau of a Voronoi edge or vertex (cells may differ); camera: "
                   "start within tau of a bisector; stop: T within 1e-3 of eps at a stop test (may stop "
                   "one step apart); graze / bend: gradient conditioning only (cells compared bit for bit)",
        "tau": "1e-6 x max(1, |scene box|, |camera|)", **flags}
    return res


def run_adjacency_only(args):
    """GPU adjacency of --sites (default 3M) sites uniform in [-1,1]^3 (seed 7),
    default domain: --warmup untimed and --steps timed builds, one JSON line."""
    import statistics

    import numpy as np
    import torch
    from paper_2502_01157_gb300 import rf
    from paper_2502_01157_gb300 import scenes as S

    n = args.sites or 3_000_000
    pos = torch.from_numpy(S.uniform_sites(n, -1.0, 1.0, np.random.default_rng(7))).cuda()
    b = rf.Adjacency()
    ts = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        b.build(pos)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ts.append((time.perf_counter() - t) * 1e3)
    ms = statistics.median(ts)
    print(json.dumps({"metric": "GPU Voronoi adjacency build", "value": n / ms / 1e3, "unit": "Msites/s",
                      "ms_per_build": ms, "n_sites": n, "stats": b.stats}), flush=True)
    b.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.adjacency_only:
        return run_adjacency_only(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np
    from paper_2502_01157_gb300 import scenes as S

    # scene generation uses a spawn process pool: do it before CUDA starts
    scene = S.config_scene(args.workload, n_sites=args.sites or None)
    cam = rank_camera(args.workload, rank)
    if args.crop:
        cam = crop_camera(cam, args.crop)
    target_np = S.random_target(cam.n_rays, 2024 + rank)
    mix_scene = c1_scene = c2_scene = None
    if not args.no_extras and world == 1:
        mix_scene = S.config_scene("c4")  # 3M-site mixture: batched and serving workloads
        c1_scene = S.config_scene("c1") if args.workload != "c1" else scene
        c2_scene = S.config_scene("c2") if args.workload != "c2" else scene

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2502_01157_gb300 import dist as rfdist
    from paper_2502_01157_gb300 import rf

    R = cam.n_rays
    deg = scene.sh_degree
    foam = rf.Foam.from_scene(scene)
    target = torch.from_numpy(target_np).to(dev)
    grads = dict(density=torch.zeros(scene.n_sites, device=dev),
                 sh=torch.zeros(scene.n_sites, (deg + 1) ** 2, 3, device=dev),
                 pos=torch.zeros(scene.n_sites, 3, device=dev))
    # the forward keeps a segment record (exit, t1, density, colour per step)
    # that the backward rebuilds its walk from
    out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
               depth=torch.empty(R, device=dev),
               walk_record=(torch.empty(rf.walk_record_bytes([cam], RECORD_STEPS), dtype=torch.uint8,
                                        device=dev), RECORD_STEPS))
    loss = torch.zeros(1, device=dev)
    scale = 1.0 / (3 * R)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(marks=None):
        if marks is not None:
            marks[0].record()
        foam.render([cam], out=out)
        if marks is not None:
            marks[1].record()
        d_rgb, _ = rf.mse_grad(out["rgb"], target, scale, loss)
        if marks is not None:
            marks[2].record()
        foam.backward([cam], out, d_rgb, grads=grads)
        if marks is not None:
            marks[3].record()
        if world > 1:
            rfdist.allreduce_grads(grads)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # workload facts (outside the timed region)
    chk = foam.render([cam], steps=True)
    steps_total = int(chk["steps"].sum().item())
    k_bar = scene.n_edges / scene.n_sites

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    marks = [[ev() for _ in range(4)] for _ in range(args.steps)]
    t0, t1 = ev(), ev()
    barrier()
    t0.record()
    for k in range(args.steps):
        step(marks[k])
    t1.record()
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    fwd_ms = sum(m[0].elapsed_time(m[1]) for m in marks) / args.steps
    bwd_ms = sum(m[2].elapsed_time(m[3]) for m in marks) / args.steps
    ms = rfdist.max_over_ranks(ms, device=dev)
    value = world * R / (ms * 1e-3) / 1e6

    # end to end through the public API with host buffers, right after the
    # device-timed steps (same state of the GPU)
    pin_t = torch.from_numpy(target_np).pin_memory()
    pin_rgb = torch.empty(R, 3).pin_memory()
    pin_loss = torch.empty(1).pin_memory()
    barrier()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        target.copy_(pin_t, non_blocking=True)
        loss.zero_()
        step()
        pin_rgb.copy_(out["rgb"], non_blocking=True)
        pin_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = (time.perf_counter() - w0) / args.steps
    barrier()


    # forward-only throughput (rendering alone: no walk record)
    fwd_only = None
    res = {}
    out_fwd = {k: out[k] for k in ("rgb", "trans", "depth")}
    if not args.no_extras:
        barrier()
        a, b = ev(), ev()
        a.record()
        for _ in range(args.steps):
            foam.render([cam], out=out_fwd)
        b.record()
        barrier()
        fwd_only = R / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6
        res["fwd_fp32_mrays_s"] = fwd_only
        # the same training step by pure recomputation: no segment record, the
        # backward searches every exit again and re-reads density and SH

        def rstep():
            foam.render([cam], out=out_fwd)
            d_rgb, _ = rf.mse_grad(out_fwd["rgb"], target, scale, loss)
            foam.backward([cam], out_fwd, d_rgb, grads=grads)

        for _ in range(2):
            rstep()
        barrier()
        a, b = ev(), ev()
        a.record()
        for _ in range(args.steps):
            rstep()
        b.record()
        barrier()
        res["fwdbwd_recompute_fp32_mrays_s"] = R / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6
        # attribute storage variants (same geometry, own copies of the attributes)
        for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16)):
            d2 = torch.from_numpy(scene.density).to(dev, dt)
            s2 = torch.from_numpy(scene.sh).to(dev, dt)
            foam.set_attributes(d2, s2)
            for _ in range(2):
                step()
            barrier()
            a, b, c = ev(), ev(), ev()
            a.record()
            for _ in range(args.steps):
                foam.render([cam], out=out_fwd)
            b.record()
            for _ in range(args.steps):
                step()
            c.record()
            barrier()
            res[f"fwd_{name}_mrays_s"] = R / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6
            res[f"fwdbwd_{name}_mrays_s"] = R / (b.elapsed_time(c) / args.steps * 1e-3) / 1e6
        foam.set_attributes(torch.from_numpy(scene.density).to(dev),
                            torch.from_numpy(scene.sh).to(dev))
        # training step with the quantile regulariser of Eq. 6 fused into the walks:
        # L = MSE + lambda * mean quantile loss (lambda = 0.01)
        qout = dict(out, quantile=torch.empty(R, device=dev), quantile_aux=torch.empty(R, 5, device=dev))
        d_q = torch.full((R,), 0.01 / R, device=dev)

        def qstep():
            foam.render([cam], out=qout)
            d_rgb, _ = rf.mse_grad(qout["rgb"], target, scale, loss)
            foam.backward([cam], qout, d_rgb, grads=grads, d_quantile=d_q)

        for _ in range(2):
            qstep()
        barrier()
        a, b, c = ev(), ev(), ev()
        a.record()
        for _ in range(args.steps):
            foam.render([cam], out=qout)
        b.record()
        for _ in range(args.steps):
            qstep()
        c.record()
        barrier()
        res["fwd_quantile_fp32_mrays_s"] = R / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6
        res["fwdbwd_quantile_fp32_mrays_s"] = R / (b.elapsed_time(c) / args.steps * 1e-3) / 1e6
        res["effects"] = effects_extras(S, rf, foam, cam, target, scale, loss, grads, args, dev)
        res["adjacency"] = adjacency_extras(rf, scene, mix_scene, args, dev)
        for name, sc in (("c1", c1_scene), ("c2", c2_scene)):
            if sc is not None and name != args.workload:
                res[f"{name}_gpu"] = workload_extras(rf, sc, S.config_cameras(name)[0], args, dev, name,
                                                     shared_cells=name == "c2")

    mixture = None
    if mix_scene is not None:
        mixture = mixture_extras(mix_scene, args, dev)

    # roofline of the dominant kernel.  The walk is a dependent gather whose
    # neighbouring rays read the same cells, so its algorithmic bytes (what a
    # cell step reads with no reuse) are served almost entirely by L1 and L2:
    # the binding unit is the L1 load data path (ncu: the LSU pipe's
    # wavefronts), whose ceiling is 128 bytes per clock per SM.  The DRAM and
    # L2 blocks hold ncu's bytes per cell step over the live duration.
    attr_b = 4
    fwd_step_b = bytes_per_step(k_bar, deg, attr_b)
    bwd_step_b = fwd_step_b + bwd_extra_bytes_per_step(deg)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm, hbm_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm, hbm_src = 6800.0, "fallback"
    dominant = "bwd" if bwd_ms >= fwd_ms else "fwd"
    kms = bwd_ms if dominant == "bwd" else fwd_ms
    step_b = bwd_step_b if dominant == "bwd" else fwd_step_b
    kname = f"{dominant}_kernel<float,{deg}>"
    wl = args.workload if not args.sites else f"{args.workload}@{scene.n_sites}"
    achieved = step_b * steps_total / (kms * 1e-3) / 1e9
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    l1_peak = n_sm * L1_BYTES_PER_CLK * sm_mhz * 1e6 / 1e9
    l2_peak = l2_read_peak(dev)
    cnt = kernel_counters(kname, wl)
    roof = {"kernel": f"rf::{kname}", "bound": "l1", "unit": "GB/s",
            "achieved": achieved, "peak": l1_peak, "frac": achieved / l1_peak,
            "peak_source": f"derived: {n_sm} SMs x {L1_BYTES_PER_CLK} B/clock x {sm_mhz:.0f} MHz "
                           "(median SM clock under load)",
            "traffic": cnt["dram_bytes_per_step"] * steps_total if cnt else None,
            "algorithmic_bytes_per_cell_step": step_b,
            "algorithmic_bytes_per_launch": step_b * steps_total,
            "cell_steps_per_launch": steps_total, "ms_per_launch": kms,
            "reuse_vs_hbm": achieved / hbm,
            "dram": ({"achieved": cnt["dram_bytes_per_step"] * steps_total / (kms * 1e-3) / 1e9,
                      "peak": hbm, "peak_source": hbm_src, "unit": "GB/s"} if cnt else None),
            "l2": ({"achieved": cnt["lts_bytes_per_step"] * steps_total / (kms * 1e-3) / 1e9,
                    "peak": l2_peak, "peak_source": "measured: strided re-read of a 48 MB buffer "
                                                    "(served from L2), CUDA events", "unit": "GB/s"}
                   if cnt else {"achieved": None, "peak": l2_peak}),
            "l1_lsu_pct": cnt["l1_lsu_pct"] if cnt else None,
            "occupancy_pct": cnt["occupancy_pct"] if cnt else None,
            "counters_source": (f"profiles/kernel_counters.txt (kernel sources {cnt['source']})" if cnt
                                else f"none for kernel sources {kernel_source_hash()}"),
            "note": "bound = the L1 load data path (the LSU pipe's wavefronts, ncu); achieved = "
                    "algorithmic bytes (no reuse) / live kernel time; reuse_vs_hbm = achieved / HBM copy peak"}
    for blk in ("dram", "l2"):
        if roof[blk] and roof[blk].get("achieved"):
            roof[blk]["frac"] = roof[blk]["achieved"] / roof[blk]["peak"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}"
                                   + (f" (with {scene.n_sites} sites)" if args.sites else "")
                                   + (f" (centre {cam.width}x{cam.height} window only)" if args.crop else ""),
                       "n_sites": scene.n_sites, "n_edges": scene.n_edges, "rays_per_step": R,
                       "cell_steps_per_ray": steps_total / R, "sh_degree": deg,
                       "step": f"fwd + mse grad + bwd (FP32 attributes; the backward rebuilds its walk "
                               f"from a {RECORD_STEPS}-step segment record of the forward)",
                       "l2": "inputs larger than L2 (packed foam %.2f GB)" % (foam.info()["device_bytes"] / 1e9),
                       "parallelism": f"dp{world}" if world > 1 else "single"},
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "cell_steps_per_s": steps_total / (ms * 1e-3),
            **res,
            "mixture_3m": mixture,
            "gpu_launches": args.steps * 6,
            "fwd_bytes_per_cell_step": fwd_step_b, "bwd_bytes_per_cell_step": bwd_step_b,
            "roofline": roof,
            "clocks": clk,
            "e2e": {"value": R / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(pin_t.numel() * 4),
                    "d2h_bytes_per_step": int(pin_rgb.numel() * 4 + 4)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cam, target_np)
        if not args.no_extras:
            line["cpu_baseline"]["adjacency"] = cpu_adjacency_baseline(scene.pos)
            cmp_ = oracle_comparisons(rf, scene, cam, c1_scene, c2_scene, args, dev)
            line["precision"] = cmp_.pop("precision")
            line["near_degenerate"] = cmp_.pop("near_degenerate")
            line["cpu_baseline"].update(cmp_)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
