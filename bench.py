#!/usr/bin/env python
"""Benchmark of differentiable Voronoi-foam ray tracing on GB300.

One step = forward render + MSE loss gradient + backward (re-walk with
gradient scatter) of one frame of the workload, all in the library's CUDA
kernels, with the scene resident in HBM.  The headline value is forward +
backward throughput in Mrays/s on the 3,000,000-site foam at 1920x1080
(plain FP32 attributes); forward-only, BF16/FP16 attribute storage and
serving latency are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own seeded view of the same scene (weak
scaling) and the site gradients are summed across ranks with one NCCL
all-reduce per step.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
import argparse
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


def bytes_per_step(k_bar, deg, attr_bytes):
    """Algorithmic bytes one cell step reads (no reuse): cell header 16 B,
    K faces x 12 B, the exit face's neighbour id 4 B, density and SH
    coefficients."""
    return 16 + 12 * k_bar + 4 + attr_bytes + 3 * (deg + 1) ** 2 * attr_bytes


def replay_bytes_per_step(deg, attr_bytes):
    """Algorithmic bytes one replayed backward step reads (no reuse): the
    walk-record byte, cell header 16 B, the exit face 12 B, its neighbour id
    4 B, density and SH coefficients."""
    return 1 + 16 + 12 + 4 + attr_bytes + 3 * (deg + 1) ** 2 * attr_bytes


def bwd_extra_bytes_per_step(deg):
    """Backward: read-modify-write of the FP32 gradients touched per step:
    density 4 B, SH 12 (deg+1)^2 B, and two site positions (one crossing) 24 B."""
    return 2 * (4 + 12 * (deg + 1) ** 2 + 24)


def kernel_source_hash():
    """Hash of the CUDA sources the renderer's kernels are built from."""
    import hashlib

    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2502_01157_gb300", "csrc")
    for name in ("rf_host.h", "rf_internal.cuh", "rf_kernels.cuh", "rf_render.cu", "rf_scene.cu"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel, workload):
    """DRAM bytes per launch of ``kernel`` on ``workload`` from the ncu
    capture recorded in profiles/dram_traffic.txt, or None if that capture
    was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload and f[2] == src:
            return float(f[3])
    return None


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
    import numpy as np
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
    while True:
        px = np.sort(rng.choice(R, size=min(n, R), replace=False)).astype(np.int64)
        t = time.perf_counter()
        oracle_step(scene, cam, px, target)
        dt = time.perf_counter() - t
        if dt >= budget_s or n >= R or n >= (1 << 22):
            break
        n = int(n * min(8.0, max(2.0, budget_s / max(dt, 1e-3))))
    return {"value": len(px) / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle fwd+bwd (MSE loss) on {len(px)} random pixels of the "
                      f"{cam.width}x{cam.height} view, {dt:.1f} s"}


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

    scene = S.config_scene(args.workload, n_sites=args.sites or None)
    cam = rank_camera(args.workload, 0)
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
                                       f"{cam.width}x{cam.height} view, fwd+bwd"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------
SERVE_RATES = (50, 200, 1000, 2000)


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
                     f"training step replays a {RECORD_STEPS}-step walk record"}
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
    from paper_2502_01157_gb300.serve import Server, run_open_loop

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

    def step():
        foam.render(cams, out=tout)
        d, _ = rf.mse_grad(tout["rgb"], target, 1.0 / (3 * R))
        foam.backward(cams, tout, d, grads=grads)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    n = max(3, args.steps // 2)
    a, b, c = ev(), ev(), ev()
    a.record()
    for _ in range(n):
        foam.render(cams, out=out)
    b.record()
    for _ in range(n):
        step()
    c.record()
    torch.cuda.synchronize()
    res = {"scene": f"c4/c5 mixture, {scene.n_sites} sites, SH deg 3",
           "c4_cameras": "8 mixed (2x 640x480, 1280x720, 1600x900, 1920x1080) on a radius-12 sphere",
           "c4_rays": R,
           "c4_fwd_fp32_mrays_s": R * n / (a.elapsed_time(b) * 1e-3) / 1e6,
           "c4_fwdbwd_fp32_mrays_s": R * n / (b.elapsed_time(c) * 1e-3) / 1e6}
    # serving poses and resolutions
    rng = np.random.default_rng(1005)
    n_req = 4000
    poses = S.sphere_poses(n_req, 12.0, 1005)
    sizes = [S.C5_RESOLUTIONS[k] for k in rng.integers(0, 4, n_req)]
    scams = [S.pinhole(w, h, 60.0, c2w=p) for (w, h), p in zip(sizes, poses)]
    # batched forward of the first 64 serving requests, FP32 vs BF16 attributes
    batch = scams[:16]
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
    # open-loop Poisson serving with BF16 attributes (set just above)
    srv = Server(foam, mem_budget_bytes=4 << 30, max_inflight=512, n_streams=4, max_batch=8)
    rates = []
    for k, rate in enumerate(SERVE_RATES):
        m = int(min(n_req, max(100, rate * 2)))
        arr = S.poisson_arrivals(float(rate), m, 500 + k)
        st = run_open_loop(srv, scams[:m], arr, deadline_s=60.0)
        rates.append({"rate_req_s": rate, "offered": m, "completed": st["completed"],
                      "rejected": st["rejected_open_loop"], "p50_ms": st["p50_ms"],
                      "p99_ms": st["p99_ms"], "mrays_s": st["mrays_s"],
                      "mean_batch": st["mean_batch"], "max_busy_streams": st["max_busy_streams"]})
    srv.close()
    res["serving_bf16"] = {"budget_gb": 4, "streams": 4, "max_batch": 8,
                           "resolutions": "uniform over 320x240, 640x480, 1280x720, 1920x1080",
                           "poses": "uniform on the radius-12 sphere, looking at the origin",
                           "rates": rates}
    foam.close()
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
    target_np = S.random_target(cam.n_rays, 2024 + rank)
    mix_scene = None
    if not args.no_extras and world == 1:
        mix_scene = S.config_scene("c4")  # 3M-site mixture: batched and serving workloads

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2502_01157_gb300 import rf

    R = cam.n_rays
    deg = scene.sh_degree
    foam = rf.Foam.from_scene(scene)
    target = torch.from_numpy(target_np).to(dev)
    grads = dict(density=torch.zeros(scene.n_sites, device=dev),
                 sh=torch.zeros(scene.n_sites, (deg + 1) ** 2, 3, device=dev),
                 pos=torch.zeros(scene.n_sites, 3, device=dev))
    # the forward keeps a walk record (which face each step left by) that the
    # backward replays instead of searching the faces again
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
            for g in grads.values():
                dist.all_reduce(g)

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
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * R / (ms * 1e-3) / 1e6

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

    mixture = None
    if mix_scene is not None:
        mixture = mixture_extras(mix_scene, args, dev)

    # end to end through the public API with host buffers
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

    # roofline of the dominant kernel (the backward, replaying the walk record
    # for the first RECORD_STEPS steps of every ray and searching after them)
    attr_b = 4
    fwd_bytes = (bytes_per_step(k_bar, deg, attr_b) + 1) * steps_total + 20 * R
    steps_replayed = int(chk["steps"].clamp(max=RECORD_STEPS).sum().item())
    bwd_step_bytes = (replay_bytes_per_step(deg, attr_b) * steps_replayed
                      + bytes_per_step(k_bar, deg, attr_b) * (steps_total - steps_replayed)) / steps_total
    bwd_bytes = (bwd_step_bytes + bwd_extra_bytes_per_step(deg)) * steps_total + 32 * R
    import json as _j

    peaks = {}
    try:
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        peak, peak_src = 6800.0, "fallback"
    dominant = "bwd" if bwd_ms >= fwd_ms else "fwd"
    kb = bwd_bytes if dominant == "bwd" else fwd_bytes
    kms = bwd_ms if dominant == "bwd" else fwd_ms
    achieved = kb / (kms * 1e-3) / 1e9
    roof = {"kernel": f"rf::{dominant}_kernel<float,{deg}>", "bound": "hbm", "achieved": achieved,
            "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(f"{dominant}_kernel<float,{deg}>", args.workload if not args.sites else f"{args.workload}@{scene.n_sites}"),
            "algorithmic_bytes_per_launch": kb, "kernel_source": kernel_source_hash(),
            "note": "algorithmic bytes are served >99% by L1/L2 (traffic = ncu DRAM bytes per "
                    "launch); the binding unit is the L1 load data path, see profiles/",
            "bytes_per_cell_step": (bwd_step_bytes + bwd_extra_bytes_per_step(deg) if dominant == "bwd"
                                    else bytes_per_step(k_bar, deg, attr_b) + 1),
            "steps_replayed_frac": steps_replayed / steps_total,
            "cell_steps_per_launch": steps_total, "ms_per_launch": kms}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}"
                                   + (f" (with {scene.n_sites} sites)" if args.sites else ""),
                       "n_sites": scene.n_sites, "n_edges": scene.n_edges, "rays_per_step": R,
                       "cell_steps_per_ray": steps_total / R, "sh_degree": deg,
                       "step": f"fwd + mse grad + bwd (FP32 attributes; the backward replays a "
                               f"{RECORD_STEPS}-step walk record of the forward)",
                       "l2": "inputs larger than L2 (packed foam %.2f GB)" % (foam.info()["device_bytes"] / 1e9),
                       "parallelism": f"dp{world}" if world > 1 else "single"},
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "cell_steps_per_s": steps_total / (ms * 1e-3),
            **res,
            "mixture_3m": mixture,
            "gpu_launches": args.steps * 6,
            "roofline": roof,
            "clocks": clk,
            "e2e": {"value": R / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(pin_t.numel() * 4),
                    "d2h_bytes_per_step": int(pin_rgb.numel() * 4 + 4)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cam, target_np)
        if not args.no_extras:
            line["cpu_baseline"]["adjacency"] = cpu_adjacency_baseline(scene.pos)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
