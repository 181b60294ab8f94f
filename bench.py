#!/usr/bin/env python
"""Throughput of the Siddon projector, its transpose and the CG solver.

One step = one ``tomo_solve`` call on the 256^3 workload: FP64 ray setup,
b = P^T M y, then ``--iters`` CG iterations (each one P, one D^T D, one P^T
and the vector updates), all through the C ABI.  The reported value is
voxel-intersections (Siddon segments) per second over P and P^T:
segments per projection x (2 iters + 1) per step.

Default workload ``cg256``: cube 256^3 float32 over [-1.5, 1.5]^3 R_sun,
240 images 512 x 512 from two observer groups 40 degrees apart (1.5 degree
steps, 215 R_sun, FOV 3.2 R_sun), occulter mask r < 1 R_sun, data = P x +
Gaussian noise at SNR 50, lambda 1e-2, 3-axis finite-difference prior.

``--impl reference`` times the FP64 CPU oracle instead (P and P^T over a
seeded ray sample of the same workload) on the host cores.

Multi-GPU: the path has no exchange step that this benchmark needs; with
``--gpus N`` under torchrun every rank runs an independent replica of the
workload (weak scaling), and the value counts the work of all ranks over the
slowest rank's time.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("Siddon voxel-intersections/s (P and P^T) and CG s/iter at 256^3, "
          "vs FP64 oracle")
UNIT = "voxel-intersections/s"
HBM_FALLBACK_GBS = 6800.0

WORKLOAD_TEXT = {
    "cg256": ("cg256: cube 256^3 f32 over [-1.5,1.5]^3 R_sun; 240 images "
              "512x512 from two observer groups 40 deg apart (1.5 deg steps, "
              "215 R_sun, FOV 3.2 R_sun); occulter mask r<1 R_sun; y = Px + "
              "noise at SNR 50; lambda 1e-2, 3-axis finite-difference prior"),
    "single": ("single: cube 128^3 f32; 60 images 256x256, lon 0-177 deg, "
               "lat jitter +-7 deg; 6 streamers; occulter r<1; SNR 50; "
               "lambda 1e-2"),
    "temporal": ("temporal: 8 frames of 256^3 f32 over [-1.5,1.5]^3 R_sun; "
                 "240 images 512x512, time stamps U[0,7]; two observer "
                 "groups 40 deg apart"),
    "coronagraph": ("coronagraph: cube 512^3 f32 over [-4,4]^3 R_sun; 360 "
                    "images 1024x1024 from two groups 86 deg apart; occulter "
                    "r<1.5 and field edge r>4 masks; SNR 30; lambda 1e-2"),
    "batched": ("batched: 32 independent problems (seeds 100-131), cube side "
                "from {32,48,64,96,128}, 16-120 images of side "
                "{64,128,256,512}, observers evenly spaced on the ecliptic; "
                "10 CG iterations each, lambda 1e-2"),
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cg256", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--iters", type=int, default=20,
                    help="CG iterations per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the comparisons timed after the headline "
                         "(bf16, autograd, temporal, batched, Thomson)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--plane-sync", type=int, default=None,
                    help="walk of P / P^T (TOMO_OPT_PLANE_SYNC bit mask: "
                         "bit 0 P^T, bit 1 P on every image, bit 2 P on the "
                         "images where it is faster; library default 5)")
    ap.add_argument("--sweep", action="store_true",
                    help="measurement table instead of the benchmark line: "
                         "P, P^T (f32 / bf16), CG s/iter and the oracle's "
                         "rate on 1 and all host cores for every config")
    ap.add_argument("--images", type=int, default=0,
                    help="keep only this many images (evenly spaced) of the "
                         "workload: a reduced case for profiler captures")
    return ap.parse_args(argv)


# ------------------------------------------------------------- distributed

def dist_env():
    return (int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def aggregate(units, seconds, world):
    """Whole-job throughput: units of all ranks over the slowest rank's
    time.  Returns (total_units, max_seconds)."""
    if world <= 1:
        return float(units), float(seconds)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
             "sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv",
                                               delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-i", self.index,
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None,
                    "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.out.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- workload

def make_workload(name, n_images=0):
    import synth
    c = (synth.configs.batched_problem(100) if name == "batched"
         else synth.make_config(name))
    if n_images and n_images < c["pointing"].shape[0]:
        keep = np.linspace(0, c["pointing"].shape[0] - 1, n_images).astype(int)
        c["pointing"] = np.ascontiguousarray(c["pointing"][keep])
        if c["mask"] is not None:
            c["mask"] = np.ascontiguousarray(c["mask"][keep])
        c["name"] += "-%dimg" % n_images
    return c


def algorithmic_bytes(n_rays, n_live, segments, kind):
    """Bytes a launch must move if nothing is cached (gather model):
    4 B per segment (voxel gather, or atomic payload for the transpose),
    the 32-byte ray record of every live ray, 1 mask byte per pixel, and
    the 4-byte pixel (written by P for every pixel, read by P^T per live
    ray)."""
    per_pixel = 4 * n_rays if kind == "forward" else 4 * n_live
    return 4.0 * segments + 32.0 * n_live + 1.0 * n_rays + per_pixel


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def _profile_record(name):
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def ncu_reduction_sectors(kernel, workload):
    """Reduction sectors that `kernel` sends from L1 to the crossbar per
    Siddon segment on `workload`, recorded in profiles/, or None.  The
    ratio was captured on a subset of the workload's images and holds per
    segment for any subset; another workload's geometry changes it."""
    rec = _profile_record("reduction_sectors.json").get(kernel)
    if not rec or rec.get("workload") != workload:
        return None
    return rec.get("l1_to_crossbar_reduction_sectors_per_segment")


def ncu_traffic(kernel, workload, n_img):
    """DRAM bytes per launch of `kernel` recorded in profiles/ for this
    workload at this image count, or None (the bytes are those of one full
    launch, which another image count or workload does not repeat)."""
    rec = _profile_record("traffic.json")
    if rec.get("workload") != workload or rec.get("images") != n_img:
        return None
    return rec.get("bytes_per_launch", {}).get(kernel)


# ----------------------------------------------------------- oracle legs

def oracle_sample(c, seconds, seed=0):
    """Time the FP64 oracle (P then P^T) on a seeded ray sample sized to
    take about `seconds`.  Returns (segments/s, threads, description)."""
    from oracle import siddon
    g, ptg, nu, nv, mask = c["geom"], c["pointing"], c["nu"], c["nv"], c["mask"]
    n_all = ptg.shape[0] * nu * nv
    live = np.flatnonzero(mask.reshape(-1) == 0) if mask is not None else \
        np.arange(n_all)
    cube = c["cube"].astype(np.float64)
    rng = np.random.default_rng(seed)
    images = np.zeros(n_all)

    def run(frac):
        ids = np.sort(rng.choice(live, max(1, int(frac * live.size)),
                                 replace=False))
        segs = siddon.count_segments(g, ptg, nu, nv, None, ray_ids=ids)
        t0 = time.perf_counter()
        vals = siddon.project(g, cube, ptg, nu, nv, None, ray_ids=ids)
        images[ids] = vals
        siddon.backproject(g, images, ptg, nu, nv, None, ray_ids=ids)
        dt = time.perf_counter() - t0
        images[ids] = 0.0
        return ids.size, segs, dt

    f_cal = min(2e-4, 4000.0 / live.size)
    n, segs, dt = run(f_cal)  # calibrate
    frac = min(1.0, f_cal * seconds / max(dt, 1e-6))
    n, segs, dt = run(frac)
    desc = ("FP64 oracle P then P^T over a seeded sample of %d unmasked rays "
            "(%.3f %% of %s, %d segments each way)"
            % (n, 100.0 * n / live.size, c["name"], segs))
    return 2 * segs / dt, siddon.get_threads(), desc, 2 * segs, dt


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, on the host cores."""
    if rank != 0:
        return 0
    c = make_workload(args.workload, args.images)
    per_step = max(0.5, min(5.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(c, per_step, seed=1)
    rates, times, units, descs, cores = [], [], [], [], 1
    for k in range(args.steps):
        rate, cores, desc, segs, dt = oracle_sample(c, per_step, seed=100 + k)
        units.append(segs)
        times.append(dt)
        descs.append(desc)
    value = float(sum(units) / sum(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": descs[0]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm

def run_gpu(args, rank, local_rank, world):
    import torch
    import synth
    import paper_1103_5904_gb300 as T
    from paper_1103_5904_gb300 import build as lib_build

    lib_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = make_workload(args.workload, args.images)
    g, ptg, nu, nv = c["geom"], c["pointing"], c["nu"], c["nv"]
    tf = c.get("n_frames", 1)  # time frames (the temporal workload)
    n_img = ptg.shape[0]
    ctx = T.Context(local_rank)
    if args.plane_sync is not None:
        ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, args.plane_sync)
    mask_h = c["mask"]
    mask = torch.from_numpy(mask_h).to(dev) if mask_h is not None else None
    x_true = torch.from_numpy(c["cube"]).to(dev)
    # data: P x + Gaussian noise (seeded draws, SNR of the workload)
    y0 = T.tomo_project(x_true, g, ptg, nu, nv, mask=mask, n_frames=tf,
                        ctx=ctx)
    keep = (mask == 0) if mask is not None else torch.ones_like(y0, dtype=bool)
    rms = torch.sqrt(torch.mean(y0[keep].double() ** 2)).item()
    z = torch.from_numpy(synth.noise_draw(c["noise_seed"] or 0, y0.shape)).to(dev)
    y = (y0.double() + (rms / (c["snr"] or 50.0)) * z).float()
    lam = c["lam"] or 1e-2
    if mask is not None:
        y[mask != 0] = 0.0
    del z, y0
    n_rays = n_img * nu * nv
    n_live = int(keep.sum().item())
    segments = T.tomo_count_segments(g, ptg, nu, nv, mask=mask, ctx=ctx)
    units_per_step = segments * (2 * args.iters + 1)
    x = torch.empty_like(x_true)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.clear_cache()  # every step redoes the FP64 ray setup
        T.tomo_solve(y, g, ptg, mask=mask, lam=lam, max_iter=args.iters,
                     out=x, report=False, n_frames=tf, ctx=ctx)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    _, info = T.tomo_solve(y, g, ptg, mask=mask, lam=lam,
                           max_iter=args.iters, out=x, n_frames=tf, ctx=ctx)
    ctx.set_option(T.tomo.TOMO_OPT_PROFILE, 1)
    ctx.profile(reset=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between steps (outside the step events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof = ctx.profile(reset=True)
    ctx.set_option(T.tomo.TOMO_OPT_PROFILE, 0)
    local_s = sum(step_ms) / 1e3
    tot_units, max_s = aggregate(units_per_step * args.steps, local_s, world)
    value = tot_units / max_s
    ms_per_step = 1e3 * max_s / args.steps

    # roofline of the dominant Siddon kernel (launch-averaged device time)
    kern = {}
    # projections per step: P once per CG iteration, P^T once more for b;
    # a projection may take more than one launch (the forward runs the
    # per-ray and the plane-synchronous kernels on their own images)
    n_proj = {"forward": args.iters * args.steps,
              "adjoint": (args.iters + 1) * args.steps}
    for kind in ("forward", "adjoint"):
        launches, ms = prof[kind]
        if launches == 0:
            continue
        per_launch_s = ms / 1e3 / n_proj[kind]
        b = algorithmic_bytes(n_rays, n_live, segments, kind)
        kern[kind] = {"launches": launches, "projections": n_proj[kind],
                      "ms_per_projection": 1e3 * per_launch_s,
                      "segments_per_s": segments / per_launch_s,
                      "rays_per_s": n_rays / per_launch_s,
                      "algorithmic_bytes": b,
                      "achieved_gbs": b / per_launch_s / 1e9,
                      "time_share": ms / sum(v[1] for v in prof.values())}
    dom = max(kern, key=lambda k: kern[k]["ms_per_projection"] * kern[k]["projections"])
    kern["layout"] = {"launches": prof["layout"][0], "ms": prof["layout"][1],
                      "what": "cube layout copies of the plane-synchronous "
                              "walk (most return at once when no image "
                              "uses their layout)"}
    peak, peak_src = peak_hbm()
    plane = 5 if args.plane_sync is None else args.plane_sync
    kname = {"forward": ("k_forward_plane<float,false>" if plane & 2 else
                         "k_forward<float,false>+k_forward_plane<float,false>"
                         if plane & 4 else "k_forward<float,false>"),
             "adjoint": ("k_adjoint_plane<false>" if plane & 1
                         else "k_adjoint<false>")}
    if tf > 1:  # time frames: the frame-pair plane walks
        kname = {"forward": "k_forward_plane_pair<float,float2>",
                 "adjoint": "k_adjoint_plane_pair"}
    roofline = {"bound": "hbm", "kernel": kname[dom],
                "achieved": kern[dom]["achieved_gbs"], "peak": peak,
                "unit": "GB/s", "frac": kern[dom]["achieved_gbs"] / peak,
                "traffic": ncu_traffic(kname[dom], args.workload, n_img),
                "peak_source": peak_src + " HBM copy bandwidth",
                "bytes_model": "4 B/segment + 37 B/live ray + 1 B/pixel"}
    if dom == "adjoint":
        # the transpose read-modify-write model: 8 B per segment (each
        # reduction reads and writes its voxel), same per-ray bytes
        per_launch_s = kern["adjoint"]["ms_per_projection"] / 1e3
        rmw = (algorithmic_bytes(n_rays, n_live, segments, "adjoint") +
               4.0 * segments)
        roofline["achieved_rmw"] = rmw / per_launch_s / 1e9
        roofline["frac_rmw"] = roofline["achieved_rmw"] / peak
    # the resource that binds the plane transpose: each SM's L1 sends at
    # most one 32-byte reduction sector per cycle to the crossbar; sectors
    # per segment from the committed capture, time from this run, clock the
    # median sampled during the timed region
    red = (ncu_reduction_sectors(kname[dom], args.workload)
           if dom == "adjoint" else None)
    if red is not None and clk.get("sm_mhz"):
        per_launch_s = kern["adjoint"]["ms_per_projection"] / 1e3
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_sec = sms * clk["sm_mhz"] * 1e6
        got_sec = red * segments / per_launch_s
        roofline["binding"] = {
            "resource": "L1 -> crossbar reduction sectors (32 B, one per "
                        "cycle per SM)",
            "achieved": got_sec, "peak": peak_sec, "unit": "sectors/s",
            "frac": got_sec / peak_sec, "sectors_per_segment": red,
            "source": "profiles/k_plane_cg256_24img.md"}
    # compulsory bytes of one projection: the cube and the images once (and
    # the mask), far below the gather model
    comp = 4.0 * x_true.numel() + 4.0 * n_rays + (n_rays if mask is not None
                                                 else 0)
    roofline["compulsory_bytes"] = comp
    roofline["compulsory_ms_at_peak"] = comp / (peak * 1e9) * 1e3
    launches = int(sum(v[0] for v in prof.values()))

    # end to end through the C ABI with host buffers: H2D of y and mask from
    # pinned memory, solve, D2H of x, every step
    e2e = None
    if not args.no_e2e:
        y_h = y.cpu().pin_memory()
        m_h = mask.cpu().pin_memory() if mask is not None else None
        x_h = torch.empty(x.shape, dtype=torch.float32).pin_memory()
        y_d = torch.empty_like(y)
        m_d = torch.empty_like(mask) if mask is not None else None
        h2d = y_h.numel() * 4 + (m_h.numel() if m_h is not None else 0)
        d2h = x_h.numel() * 4
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def e2e_step():
            y_d.copy_(y_h, non_blocking=True)
            if m_h is not None:
                m_d.copy_(m_h, non_blocking=True)
            ctx.clear_cache()
            T.tomo_solve(y_d, g, ptg, mask=m_d, lam=lam,
                         max_iter=args.iters, out=x, report=False,
                         n_frames=tf, ctx=ctx)
            x_h.copy_(x, non_blocking=True)

        # the same untimed warm-up as the device-timed steps (the first
        # copies from freshly pinned buffers pay one-time costs)
        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_units, e_s = aggregate(units_per_step * args.steps,
                                 e0.elapsed_time(e1) / 1e3, world)
        e2e = {"value": e_units / e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * e_s / args.steps}

    extras = None
    if rank == 0 and world == 1 and not args.no_extras and \
            args.workload == "cg256" and not args.images:
        extras = run_extras(ctx, dev, c, y, mask, args.iters, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc, _, _ = oracle_sample(c, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": WORKLOAD_TEXT[args.workload] + (
                    " (reduced to %d images)" % args.images if args.images
                    else ""),
                "step": ("one tomo_solve: FP64 ray setup, b = P^T M y, %d CG "
                         "iterations" % args.iters),
                "cg_iters_per_step": args.iters,
                "rays": n_rays, "live_rays": n_live,
                "segments_per_projection": segments,
                "segments_per_step": units_per_step,
                "l2": "flushed between steps (512 MiB write)",
                "parallelism": "replicas" if world > 1 else "single GPU"},
            "cg_s_per_iter": ms_per_step / 1e3 / args.iters,
            "final_J_over_J0": float(info["J"][-1] / info["J"][0]),
            "kernels": kern,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": t_wall,
        }
        if extras is not None:
            line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_batched(args, rank, local_rank, world):
    """Config 3: all problems in one graph-captured batched solve, against
    the one-problem-at-a-time loop of tomo_solve on the same GPU."""
    import torch
    import synth
    import paper_1103_5904_gb300 as T
    from paper_1103_5904_gb300 import build as lib_build

    lib_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = T.Context(local_rank)
    iters = 10
    probs, segs = [], 0
    for c in synth.configs.batched():
        cube = torch.from_numpy(c["cube"]).to(dev)
        n_img = c["pointing"].shape[0]
        y = T.tomo_project(cube, c["geom"], c["pointing"], c["nu"], c["nv"],
                           ctx=ctx)
        segs += T.tomo_count_segments(c["geom"], c["pointing"], c["nu"],
                                      c["nv"], ctx=ctx)
        probs.append({"geom": c["geom"], "pointing": c["pointing"],
                      "nu": c["nu"], "nv": c["nv"], "images": y,
                      "cube": torch.zeros_like(cube), "lam": c["lam"],
                      "n_img": n_img})
        del cube
    units = segs * (2 * iters + 1)
    stream = torch.cuda.current_stream(dev)
    # batched: autotune once (first call), then graph replays
    T.tomo_solve_batched(probs, iters, autotune=True, report=False, ctx=ctx)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    def batched():
        T.tomo_solve_batched(probs, iters, report=False, ctx=ctx)

    def sequential():
        for p in probs:
            T.tomo_solve(p["images"], p["geom"], p["pointing"], lam=p["lam"],
                         max_iter=iters, out=p["cube"], report=False, ctx=ctx)

    for _ in range(args.warmup):
        batched()
        sequential()
    ctx.profile(reset=True)
    ms_b = timed(batched, args.steps)
    launches = sum(v[0] for v in ctx.profile(reset=True).values())
    ms_s = timed(sequential, args.steps)
    # per-kernel device time of one sequential pass (CUDA events)
    ctx.set_option(T.tomo.TOMO_OPT_PROFILE, 1)
    ctx.profile(reset=True)
    sequential()
    seq_prof = ctx.profile(reset=True)
    ctx.set_option(T.tomo.TOMO_OPT_PROFILE, 0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": units / (ms_b / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["batched"],
                       "step": "one tomo_solve_batched (one CUDA graph replay "
                               "of %d CG iterations for all 32 problems)"
                               % iters,
                       "segments_per_projection_all_problems": segs},
            "sequential": {"value": units / (ms_s / 1e3), "unit": UNIT,
                           "ms_per_step": ms_s,
                           "what": "tomo_solve per problem, one after another",
                           "kernels_ms": {k: v[1] for k, v in seq_prof.items()},
                           "launches": {k: v[0] for k, v in seq_prof.items()}},
            "batched_speedup": ms_s / ms_b,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ------------------------------------------------ comparisons (extras)

def _med_ms(fn, reps, flush):
    """Median device time of fn() over reps calls (CUDA events on the
    current stream), L2 flushed before each call outside the events."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def run_extras(ctx, dev, c, y, mask, iters, flush):
    """The forms compared against the plain FP32 single-instance path on the
    same GPU, timed after the headline (which they do not change):
      bf16:     P with the cube stored in bf16, and CG with a bf16 copy of
                the direction run to the FP32 criterion of `iters` iterations
      temporal: P and P^T of the 8-frame time-interpolated workload (frame
                pairs side by side), f32 and bf16 frames
      autograd: forward + backward of 0.5 ||P X||^2 through the autograd
                Function against the plain P and P^T calls (temporal)
      thomson:  pB and B operators (one walk for B) against P, photosphere
                geometry
      batched:  the 32-problem workload: one graph replay of 10 CG
                iterations and one batched P / P^T against the per-problem
                calls."""
    import torch
    import synth
    import paper_1103_5904_gb300 as T
    out = {}
    g, ptg, nu, nv = c["geom"], c["pointing"], c["nu"], c["nv"]
    X = torch.from_numpy(c["cube"]).to(dev)
    segs = T.tomo_count_segments(g, ptg, nu, nv, mask=mask, ctx=ctx)
    yy = torch.empty_like(y)
    p32 = _med_ms(lambda: T.tomo_project(X, g, ptg, nu, nv, mask=mask,
                                         out=yy, ctx=ctx), 5, flush)
    Xb = X.to(torch.bfloat16)
    p16 = _med_ms(lambda: T.tomo_project(Xb, g, ptg, nu, nv, mask=mask,
                                         out=yy, ctx=ctx), 5, flush)
    del Xb
    x = torch.empty_like(X)
    _, i32 = T.tomo_solve(y, g, ptg, mask=mask, lam=c["lam"], max_iter=iters,
                          out=x, ctx=ctx)
    _, i16 = T.tomo_solve(y, g, ptg, mask=mask, lam=c["lam"],
                          max_iter=int(1.5 * iters), out=x, bf16=True, ctx=ctx)
    target = i32["J"][iters] * (1 + 1e-4)
    hit = np.flatnonzero(i16["J"] <= target)
    k16 = int(hit[0]) if hit.size else -1
    cg32 = _med_ms(lambda: T.tomo_solve(y, g, ptg, mask=mask, lam=c["lam"],
                                        max_iter=iters, out=x, report=False,
                                        ctx=ctx), 3, flush)
    cg16 = (_med_ms(lambda: T.tomo_solve(y, g, ptg, mask=mask, lam=c["lam"],
                                         max_iter=k16, out=x, bf16=True,
                                         report=False, ctx=ctx), 3, flush)
            if k16 > 0 else None)
    out["bf16"] = {"P_f32_ms": p32, "P_bf16_ms": p16,
                   "cg_f32_iters": iters, "cg_bf16_iters_to_f32_criterion": k16,
                   "cg_f32_ms": cg32, "cg_bf16_ms_to_f32_criterion": cg16,
                   "what": "%s: bf16-stored cube against float32 (P), and CG "
                           "with a bf16 copy of the direction run until its "
                           "criterion reaches the float32 criterion after %d "
                           "iterations" % (c["name"], iters)}
    # Thomson operators on the same geometry with the photosphere
    go = dict(g, r_obs=1.0)
    th = {}
    for kind in ("emission", "pB", "B"):
        kw = {} if kind == "emission" else {"kind": kind, "limb_u": 0.6}
        yk = T.tomo_project(X, go, ptg, nu, nv, mask=mask, ctx=ctx, **kw)
        th[kind + "_P_ms"] = _med_ms(lambda: T.tomo_project(
            X, go, ptg, nu, nv, mask=mask, out=yk, ctx=ctx, **kw), 5, flush)
        th[kind + "_PT_ms"] = _med_ms(lambda: T.tomo_backproject(
            yk, go, ptg, mask=mask, out=x, ctx=ctx, **kw), 5, flush)
        del yk
    th["B_over_pB"] = {"P": th["B_P_ms"] / th["pB_P_ms"],
                       "PT": th["B_PT_ms"] / th["pB_PT_ms"]}
    th["what"] = ("%s with the opaque photosphere r_obs = 1, limb darkening "
                  "0.6: emission P, T_pB = O P M and T_B = P M' - O P M (one "
                  "walk on (m' x, m x) pairs)" % c["name"])
    out["thomson"] = th
    del X, x, yy
    torch.cuda.empty_cache()
    # time-interpolated workload and the autograd Function
    ct = synth.make_config("temporal")
    gt, pt, tf = ct["geom"], ct["pointing"], ct["n_frames"]
    Xt = torch.from_numpy(ct["cube"]).to(dev)
    st = T.tomo_count_segments(gt, pt, ct["nu"], ct["nv"], ctx=ctx)
    yt = T.tomo_project(Xt, gt, pt, ct["nu"], ct["nv"], n_frames=tf, ctx=ctx)
    xt = torch.empty_like(Xt)
    tp = _med_ms(lambda: T.tomo_project(Xt, gt, pt, ct["nu"], ct["nv"],
                                        n_frames=tf, out=yt, ctx=ctx), 5, flush)
    ta = _med_ms(lambda: T.tomo_backproject(yt, gt, pt, n_frames=tf, out=xt,
                                            ctx=ctx), 5, flush)
    Xtb = Xt.to(torch.bfloat16)
    tpb = _med_ms(lambda: T.tomo_project(Xtb, gt, pt, ct["nu"], ct["nv"],
                                         n_frames=tf, out=yt, ctx=ctx), 5, flush)
    del Xtb
    out["temporal"] = {"segments": int(st), "P_ms": tp, "PT_ms": ta,
                       "P_bf16_ms": tpb,
                       "P_segments_per_s": st / (tp / 1e3),
                       "PT_segments_per_s": st / (ta / 1e3),
                       "what": WORKLOAD_TEXT["temporal"]}
    Xg = Xt.clone().requires_grad_(True)

    def fwd_bwd():
        Xg.grad = None
        P = T.autograd.project(Xg, gt, pt, ct["nu"], ct["nv"], n_frames=tf,
                               ctx=ctx)
        P.backward(P.detach())
    out["autograd"] = {"fwd_bwd_ms": _med_ms(fwd_bwd, 5, flush),
                       "plain_P_plus_PT_ms": tp + ta,
                       "what": "temporal: forward + backward of 0.5 ||P X||^2 "
                               "through the autograd Function (backward = the "
                               "transpose kernel) against the plain P and P^T "
                               "calls"}
    del Xt, xt, yt, Xg
    torch.cuda.empty_cache()
    out["batched"] = batched_compare(T, ctx, dev, flush, steps=3, warmup=1)
    return out


def batched_compare(T, ctx, dev, flush, steps, warmup, iters=10):
    """The 32-problem workload: graph-replayed batched CG against the
    per-problem loop, and one batched P and P^T over all problems against
    the per-problem calls (ray records cached in both)."""
    import torch
    import synth
    probs, segs = [], 0
    for c in synth.configs.batched():
        cube = torch.from_numpy(c["cube"]).to(dev)
        y = T.tomo_project(cube, c["geom"], c["pointing"], c["nu"], c["nv"],
                           ctx=ctx)
        segs += T.tomo_count_segments(c["geom"], c["pointing"], c["nu"],
                                      c["nv"], ctx=ctx)
        probs.append({"geom": c["geom"], "pointing": c["pointing"],
                      "nu": c["nu"], "nv": c["nv"], "images": y,
                      "cube": torch.zeros_like(cube), "lam": c["lam"],
                      "x_true": cube})
    T.tomo_solve_batched(probs, iters, autotune=True, report=False, ctx=ctx)

    def batched_cg():
        T.tomo_solve_batched(probs, iters, report=False, ctx=ctx)

    def sequential_cg():
        for p in probs:
            T.tomo_solve(p["images"], p["geom"], p["pointing"], lam=p["lam"],
                         max_iter=iters, out=p["cube"], report=False, ctx=ctx)
    fwd_b = [dict(p, cube=p["x_true"], images=torch.empty_like(p["images"]))
             for p in probs]
    adj_b = [dict(p, cube=torch.empty_like(p["x_true"])) for p in probs]

    def batched_p():
        T.tomo_project_batched(fwd_b, ctx=ctx)

    def batched_pt():
        T.tomo_backproject_batched(adj_b, ctx=ctx)

    def seq_p():
        for p, d in zip(probs, fwd_b):
            T.tomo_project(p["x_true"], p["geom"], p["pointing"], p["nu"],
                           p["nv"], out=d["images"], ctx=ctx)

    def seq_pt():
        for p, d in zip(probs, adj_b):
            T.tomo_backproject(p["images"], p["geom"], p["pointing"],
                               out=d["cube"], ctx=ctx)
    res = {}
    for name, fn in (("cg_graph_ms", batched_cg), ("cg_sequential_ms",
                                                   sequential_cg),
                     ("P_batched_ms", batched_p), ("P_sequential_ms", seq_p),
                     ("PT_batched_ms", batched_pt),
                     ("PT_sequential_ms", seq_pt)):
        for _ in range(warmup):
            fn()
        res[name] = _med_ms(fn, steps, flush)
    res["cg_speedup"] = res["cg_sequential_ms"] / res["cg_graph_ms"]
    res["segments_per_projection_all_problems"] = int(segs)
    res["cg_iters"] = iters
    res["what"] = (WORKLOAD_TEXT["batched"] + "; batched = one graph replay "
                   "(CG) or one persistent launch (P, P^T) over all problems, "
                   "sequential = the single-problem calls one after another; "
                   "ray records cached, L2 flushed before each timing")
    return res


# ------------------------------------------------------- measurement table

SWEEP = [
    # name, CG iterations (0: none), bf16 variant
    ("small", 0, False),
    ("single", 20, False),
    ("temporal", 0, True),
    ("coronagraph", 50, True),
    ("paper128", 0, False),
    ("paper256", 0, False),
    ("cg256", 20, True),
]
# configs also measured with the photosphere and a map mask inside it
SOLAR_SETTING = ("paper128", "cg256")


def run_sweep(args, local_rank):
    """One JSON line per config: device time and segments/s of P and P^T
    (median of repeated calls with the ray records cached, L2 flushed between
    calls), the bf16-stored cube where the config has one, CG seconds per
    iteration (ray setup excluded), bf16 against f32 CG at equal criterion,
    the autograd form against the plain calls (time-varying config), and
    the FP64 oracle's segments/s on one host core and on all of them."""
    import torch
    import synth
    import paper_1103_5904_gb300 as T
    from oracle import siddon
    from paper_1103_5904_gb300 import build as lib_build

    lib_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    ctx = T.Context(local_rank)

    def med_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for name, cg_iters, has_bf16 in SWEEP:
        c = synth.make_config(name)
        g, ptg, nu, nv = c["geom"], c["pointing"], c["nu"], c["nv"]
        T_frames = c["n_frames"]
        mask = (torch.from_numpy(c["mask"]).to(dev)
                if c["mask"] is not None else None)
        X = torch.from_numpy(c["cube"]).to(dev)
        segs = T.tomo_count_segments(g, ptg, nu, nv, mask=mask, ctx=ctx)
        rays = ptg.shape[0] * nu * nv
        reps = 10 if segs < 2e10 else 5
        y = T.tomo_project(X, g, ptg, nu, nv, mask=mask, n_frames=T_frames,
                           ctx=ctx)
        out = torch.empty_like(X)
        line = {"sweep": name, "segments": int(segs), "rays": int(rays)}
        p_ms = med_ms(lambda: T.tomo_project(X, g, ptg, nu, nv, mask=mask,
                                             n_frames=T_frames, out=y,
                                             ctx=ctx), reps)
        a_ms = med_ms(lambda: T.tomo_backproject(y, g, ptg, mask=mask,
                                                 n_frames=T_frames, out=out,
                                                 ctx=ctx), reps)
        line.update({"P_ms": p_ms, "PT_ms": a_ms,
                     "P_segments_per_s": segs / (p_ms / 1e3),
                     "PT_segments_per_s": segs / (a_ms / 1e3),
                     "P_rays_per_s": rays / (p_ms / 1e3)})
        if has_bf16:
            Xb = X.to(torch.bfloat16)
            line["P_bf16_ms"] = med_ms(lambda: T.tomo_project(
                Xb, g, ptg, nu, nv, mask=mask, n_frames=T_frames, out=y,
                ctx=ctx), reps)
            line["P_bf16_segments_per_s"] = segs / (line["P_bf16_ms"] / 1e3)
            del Xb
        if T_frames > 1:
            # the projector as a torch.autograd.Function: forward + backward
            # of 0.5 ||P X||^2 against the plain P and P^T calls
            Xg = X.clone().requires_grad_(True)

            def fwd_bwd():
                Xg.grad = None
                P = T.autograd.project(Xg, g, ptg, nu, nv, mask=mask,
                                       n_frames=T_frames, ctx=ctx)
                P.backward(P.detach())
            line["autograd_fwd_bwd_ms"] = med_ms(fwd_bwd, reps)
            line["plain_P_plus_PT_ms"] = p_ms + a_ms
            del Xg
        if cg_iters:
            # data: the projection of the cube (noise-free here: the solver's
            # speed does not depend on the noise)
            yd = y if T_frames == 1 else None
            x = torch.empty_like(X)
            cg_ms = med_ms(lambda: T.tomo_solve(
                yd, g, ptg, mask=mask, lam=c["lam"], max_iter=cg_iters,
                out=x, report=False, ctx=ctx), 3)
            line["cg_iters"] = cg_iters
            line["cg_s_per_iter"] = cg_ms / 1e3 / cg_iters
            if has_bf16:
                _, i32 = T.tomo_solve(yd, g, ptg, mask=mask, lam=c["lam"],
                                      max_iter=cg_iters, out=x, ctx=ctx)
                _, i16 = T.tomo_solve(yd, g, ptg, mask=mask, lam=c["lam"],
                                      max_iter=int(1.5 * cg_iters), out=x,
                                      bf16=True, ctx=ctx)
                target = i32["J"][cg_iters] * (1 + 1e-4)
                hit = np.flatnonzero(i16["J"] <= target)
                k16 = int(hit[0]) if hit.size else -1
                line["bf16_iters_to_f32_criterion"] = k16
                if k16 > 0:
                    b_ms = med_ms(lambda: T.tomo_solve(
                        yd, g, ptg, mask=mask, lam=c["lam"], max_iter=k16,
                        out=x, bf16=True, report=False, ctx=ctx), 3)
                    line["cg_bf16_s_to_f32_criterion"] = b_ms / 1e3
                    line["cg_f32_s"] = cg_ms / 1e3
            del x
        if name in SOLAR_SETTING:
            # the solar-tomography setting: opaque photosphere (lines of
            # sight end at r = 1) and a map mask that excludes the voxels
            # inside it; segments, P and P^T times, CG seconds per iteration
            go = dict(g, r_obs=1.0)
            mm = torch.from_numpy(synth.shell_map_mask(go, 1.0)).to(dev)
            segs_o = T.tomo_count_segments(go, ptg, nu, nv, mask=mask, ctx=ctx)
            yo = T.tomo_project(X, go, ptg, nu, nv, mask=mask, ctx=ctx)
            line["solar_segments"] = int(segs_o)
            line["solar_P_ms"] = med_ms(lambda: T.tomo_project(
                X, go, ptg, nu, nv, mask=mask, map_mask=mm, out=yo, ctx=ctx),
                reps)
            line["solar_PT_ms"] = med_ms(lambda: T.tomo_backproject(
                yo, go, ptg, mask=mask, map_mask=mm, out=out, ctx=ctx), reps)
            if cg_iters:
                x = torch.empty_like(X)
                cg_o = med_ms(lambda: T.tomo_solve(
                    yo, go, ptg, mask=mask, lam=c["lam"], max_iter=cg_iters,
                    out=x, report=False, map_mask=mm, ctx=ctx), 3)
                line["solar_cg_s_per_iter"] = cg_o / 1e3 / cg_iters
                del x
            # white-light images (Thomson pB and B operators, limb
            # darkening 0.6) on the same geometry
            for kind in ("pB", "B"):
                yk = T.tomo_project(X, go, ptg, nu, nv, mask=mask, kind=kind,
                                    limb_u=0.6, ctx=ctx)
                line[kind + "_P_ms"] = med_ms(lambda: T.tomo_project(
                    X, go, ptg, nu, nv, mask=mask, kind=kind, limb_u=0.6,
                    out=yk, ctx=ctx), reps)
                line[kind + "_PT_ms"] = med_ms(lambda: T.tomo_backproject(
                    yk, go, ptg, mask=mask, kind=kind, limb_u=0.6, out=out,
                    ctx=ctx), reps)
                del yk
            del yo, mm
        if T_frames == 1:
            # the autotuner's schedule for this size bucket (tile shape and
            # walk rules), P and P^T timed again under it
            best = T.tomo_autotune(X, y, g, ptg, mask=mask, ctx=ctx)
            line["tuned_rules"] = best["rules"]
            line["P_tuned_ms"] = med_ms(lambda: T.tomo_project(
                X, g, ptg, nu, nv, mask=mask, out=y, ctx=ctx), reps)
            line["PT_tuned_ms"] = med_ms(lambda: T.tomo_backproject(
                y, g, ptg, mask=mask, out=out, ctx=ctx), reps)
            T.tomo_set_plane_rules(None, g, nu, nv, ctx=ctx)
        # the oracle on one core and on all host cores (seeded ray sample)
        c_host = dict(c)
        nthreads = siddon.get_threads()
        if T_frames == 1:
            siddon.set_threads(1)
            line["oracle_segments_per_s_1core"] = oracle_sample(c_host, 1.0, 7)[0]
            siddon.set_threads(nthreads)
            r, cores, _, _, _ = oracle_sample(c_host, 2.0, 8)
            line["oracle_segments_per_s_all"] = r
            line["oracle_cores"] = cores
        print(json.dumps(line), flush=True)
        del X, y, out
        torch.cuda.empty_cache()
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, local_rank, world = dist_env()
    if world != args.gpus:
        if world == 1 and args.gpus > 1:
            print("run --gpus %d under torchrun (one process per GPU)"
                  % args.gpus, file=sys.stderr)
            return 2
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args, local_rank) if rank == 0 else 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batched":
            return run_batched(args, rank, local_rank, world)
        return run_gpu(args, rank, local_rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
