#!/usr/bin/env python3
"""Benchmark: one timestep of the grey radiative LB scheme (stream + exact
implicit collision) on the radiating-sphere workload, 128^3 sites x 42
directions (icosahedral geodesic level 1), float32 populations, vacuum
faces, kappa_a = eta = 40 inside R = 0.25 (kappa_a R = 10), cfl 0.5.

Prints one JSON line.  `value` is site-direction updates per second over
the timed steps (inputs resident in HBM, 705 MB of populations per step,
larger than L2); `e2e` is the same metric through the C ABI with host
buffers: every step hands new fluid coefficients (kappa_a, eta) over in
pinned host memory (lb_rt_set_fluid with LB_RT_HOST_MAPPED: the step kernel
reads them across the host link), steps, and returns E and F to pinned host
memory (lb_rt_step_moments: the collision epilogue writes them across the
host link), as a coupled hydrodynamics code does each step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun) runs independent replicas, one per GPU (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 128
LEVEL = 1
NDIR = 42
KAPPA_R = 10.0
CFL = 0.5
METRIC = "site-direction updates/s"
UNIT = "sd/s"
WORKLOAD = "3D radiating sphere 128^3 x 42 dirs (icosahedral L1), FP32 populations, kappa_a R = 10, vacuum faces, cfl 0.5"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            v = d.get("hbm_gbs") or d.get("hbm_GBs") or d.get("hbm")
            if v:
                return float(v), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


PROFILE = os.path.join(ROOT, "profiles", "step_static_f32_sphere128_42.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2007_05718_gb300", "csrc", f)
                  for f in ("kernels_tma.cu", "tma_common.cuh")]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _traffic_from_profiles():
    """Per-launch DRAM bytes of the step kernel from the committed ncu
    summary, or None when the kernel source changed after the capture."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    for line in open(PROFILE):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha256_16")):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % os.getpid())
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # wait (up to 5 s) until the sampler runs, and count only the samples
        # taken from here on, i.e. during the timed region
        self.skip = 0
        if self.proc:
            t_end = time.time() + 5.0
            while time.time() < t_end:
                self.f.flush()
                n = sum(1 for _ in open(self.path))
                if n > 0:
                    self.skip = n
                    break
                time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.06)  # one more sample interval
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for i, line in enumerate(open(self.path)):
            if i < self.skip:
                continue
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, v):
    """Maximum of a per-rank value over the replicas (NCCL on GPUs, gloo on CPU)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_step_per_rank, ws, ms_max, steps):
    """Whole-job rate of N independent replicas: all ranks' units over the
    slowest rank's time (weak scaling)."""
    return units_per_step_per_rank * ws * steps / (ms_max * 1e-3)


def _workload_fields():
    from paper_2007_05718_gb300 import workloads as W
    return W.radiating_sphere(N_SIDE, KAPPA_R)


def oracle_sample_time(n_side, steps=1):
    """Time the FP64 oracle (as it stands) on an n_side^3 sub-box of the same
    workload, single thread; returns (seconds per step, sd per step)."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import directions as D, lb
from paper_2007_05718_gb300 import workloads as W
n = %d
sp = W.radiating_sphere(n, %r)
nv, w = D.icosphere(%d)
lat = lb.Lattice(3, (n, n, n), nv, w, cfl=%r, dx=1.0 / n, bc=(lb.VACUUM,) * 3)
co = lb.Static(kappa_a=sp["kappa_a"].astype(float), eta=sp["eta"].astype(float))
I = lb.isotropic(sp["E0"].astype(float), lat)
t0 = time.perf_counter()
for _ in range(%d):
    I = lb.step(I, lat, co)
dt = time.perf_counter() - t0
print(json.dumps({"sec": dt / %d, "sd": n ** 3 * len(w)}))
""" % (ROOT, n_side, KAPPA_R, LEVEL, CFL, steps, steps)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["sec"], d["sd"]


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n_sample = 48
    for _ in range(max(args.warmup, 0) and 1):
        oracle_sample_time(16, 1)
    sec, sd = oracle_sample_time(n_sample, max(args.steps, 1))
    value = sd / sec
    ncores = len(os.sched_getaffinity(0))
    sample = "%d^3 sub-box of the same workload (42 dirs), %d oracle steps, FP64 numpy, 1 thread" % (
        n_sample, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sites": N_SIDE ** 3, "ndir": NDIR},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cores": ncores},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def collision_mode_costs(steps=20, warmup=3, n=128):
    """Step time of the three collision forms on one workload (128^3 x 42,
    periodic, kappa_a = 1, kappa_0 = 1e3, lambda = 0.5, eta = 1, FP32): the
    exact implicit closed form, the explicit update and the paper's
    Lambda iteration with 5 cycles (its timing runs use 5)."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    E0 = torch.from_numpy(W.gaussian_E0((n, n, n), 8.0)).cuda()
    out = {}
    for name, coll, iters in (("implicit_exact", lbrt.LB_RT_IMPLICIT_EXACT, 1),
                              ("explicit", lbrt.LB_RT_EXPLICIT, 1),
                              ("lambda_5", lbrt.LB_RT_LAMBDA_K, 5)):
        stream = torch.cuda.Stream()
        h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=1, cfl=CFL,
                              collision=coll, lambda_iters=iters, stream=stream.cuda_stream)
        lbrt.lb_rt_set_fluid(h, kappa_a=1.0, kappa_0=1000.0, lam=0.5, eta=1.0)
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        lbrt.lb_rt_step(h, warmup)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lbrt.lb_rt_step(h, steps)
        b.record(stream)
        b.synchronize()
        out[name + "_ms"] = a.elapsed_time(b) / steps
        lbrt.lb_rt_destroy(h)
    out["implicit_over_explicit"] = out["implicit_exact_ms"] / out["explicit_ms"]
    out["lambda5_over_explicit"] = out["lambda_5_ms"] / out["explicit_ms"]
    out["workload"] = "128^3 x 42 periodic, kappa_a 1, kappa_0 1e3, lambda 0.5, eta 1, FP32"
    return out


def moving_fluid_costs(n=256, level=2, steps=10, warmup=3):
    """Moving background fluid (mixed frame, App. B), 256^3 x 162 periodic,
    the seeded shear flow: step time with FP32 and with FP16 populations."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    mf = W.moving_fluid(n)
    fields = {k: torch.from_numpy(mf[k]).cuda() for k in ("v", "kt_a", "kt_0", "eta_t")}
    E0 = torch.ones((n, n, n), dtype=torch.float32, device="cuda")
    out = {}
    for name, st in (("fp32", lbrt.LB_RT_F32), ("fp16", lbrt.LB_RT_F16_DEV)):
        stream = torch.cuda.Stream()
        h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=level, cfl=CFL,
                              moving=True, storage=st, stream=stream.cuda_stream)
        lbrt.lb_rt_set_fluid(h, **fields)
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        lbrt.lb_rt_step(h, warmup)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lbrt.lb_rt_step(h, steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "sd_s": n ** 3 * N / (ms * 1e-3)}
        lbrt.lb_rt_destroy(h)
        torch.cuda.empty_cache()
    out["fp16_over_fp32"] = out["fp32"]["ms_per_step"] / out["fp16"]["ms_per_step"]
    out["workload"] = "256^3 x 162 periodic shear flow (|v| <= 0.6), density-scaled opacities"
    return out


def diffusion_costs(n=256, level=2, steps=10, warmup=3):
    """Optically thick diffusion, 256^3 x 162 periodic, kappa_0 = 1e3 /L,
    Gaussian E0 (sigma 8 cells): step time with FP32, FP16 and BF16
    populations, and the 16-bit over FP32 rate."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    E0 = torch.from_numpy(W.gaussian_E0((n, n, n), 8.0)).cuda()
    out = {}
    for name, st in (("fp32", lbrt.LB_RT_F32), ("fp16", lbrt.LB_RT_F16_DEV),
                     ("bf16", lbrt.LB_RT_BF16_DEV)):
        stream = torch.cuda.Stream()
        h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=level, cfl=CFL,
                              dx=1.0 / n, bc=(lbrt.LB_RT_PERIODIC,) * 3, storage=st,
                              stream=stream.cuda_stream)
        lbrt.lb_rt_set_fluid(h, kappa_0=1000.0)
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        lbrt.lb_rt_step(h, warmup)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lbrt.lb_rt_step(h, steps)
        b.record(stream)
        b.synchronize()
        lbrt.lb_rt_sync(h)
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "sd_s": n ** 3 * N / (ms * 1e-3)}
        lbrt.lb_rt_destroy(h)
        torch.cuda.empty_cache()
    out["fp16_over_fp32"] = out["fp32"]["ms_per_step"] / out["fp16"]["ms_per_step"]
    out["bf16_over_fp32"] = out["fp32"]["ms_per_step"] / out["bf16"]["ms_per_step"]
    out["workload"] = "256^3 x 162 periodic diffusion, kappa_0 = 1e3 /L, Gaussian E0 (8 cells)"
    return out


def serving_measurement(n_capacity=16, n_open=40, seed=20200711):
    """Batched serving on the seeded request stream (sphere/shadow, n in
    {32..128}^3, 42 or 162 directions, kappa log-uniform 1e-1..1e4, 200-2000
    steps, FP16 storage): capacity from a closed-loop run of the first
    n_capacity requests (all present at t = 0), then the first n_open
    requests with Poisson arrivals at 0.8 x that capacity."""
    from paper_2007_05718_gb300 import serve
    from paper_2007_05718_gb300 import workloads as W
    closed = W.serving_requests(n_capacity, seed=seed, rate=1e9)
    for r in closed:
        r["arrival"] = 0.0
    rc = serve.serve(closed, steps_per_tick=50, max_problems=64)
    cap = rc["throughput_req_s"]
    rate = 0.8 * cap
    stream = W.serving_requests(n_open, seed=seed, rate=rate)
    ro = serve.serve(stream, steps_per_tick=50, max_problems=64)
    return {
        "capacity_req_s": cap, "capacity_sd_s": rc["throughput_sd_s"],
        "arrival_rate_req_s": rate, "requests": ro["requests"], "completed": ro["completed"],
        "p50_s": ro["p50_s"], "p99_s": ro["p99_s"], "throughput_req_s": ro["throughput_req_s"],
        "throughput_sd_s": ro["throughput_sd_s"], "max_concurrent": ro["max_concurrent"],
        "storage": "fp16", "steps_per_tick": 50,
        "sample": "first %d requests of the seed-%d stream (closed loop) and first %d with Poisson "
                  "arrivals at 0.8 x capacity; the configured stream has 2000" % (n_capacity, seed, n_open),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=20, help="coupled steps of the end-to-end run")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched serving run")
    ap.add_argument("--no-collision-modes", action="store_true",
                    help="skip the implicit / explicit / Lambda-5 timing")
    ap.add_argument("--no-moving", action="store_true",
                    help="skip the 256^3 x 162 runs (diffusion FP32/FP16/BF16, moving fluid)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_05718_gb300 import build, lbrt
    build.build()
    sp = _workload_fields()
    stream = torch.cuda.Stream()
    sites = N_SIDE ** 3
    with torch.cuda.stream(stream):
        h = lbrt.lb_rt_create(3, N_SIDE, N_SIDE, N_SIDE, dirset=lbrt.LB_RT_ICOSPHERE, level=LEVEL,
                              cfl=CFL, dx=1.0 / N_SIDE, bc=(lbrt.LB_RT_VACUUM,) * 3,
                              stream=stream.cuda_stream)
        ka = torch.from_numpy(sp["kappa_a"]).cuda()
        eta = torch.from_numpy(sp["eta"]).cuda()
        E0 = torch.from_numpy(sp["E0"]).cuda()
        lbrt.lb_rt_set_fluid(h, kappa_a=ka, eta=eta)
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        # warm-up
        lbrt.lb_rt_step(h, args.warmup)
        stream.synchronize()
        _barrier(ws)
        clocks = Clocks(local)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        _barrier(ws)
        t0.record(stream)
        for _ in range(args.steps):
            lbrt.lb_rt_step(h, 1)
        t1.record(stream)
        t1.synchronize()
        torch.cuda.synchronize()
        _barrier(ws)
        ms = t0.elapsed_time(t1)
        ck = clocks.stop()
        ms_max = _max_over_ranks(ws, ms)
        ms_step = ms_max / args.steps
        sd_step = sites * N
        value = aggregate_rate(sd_step, ws, ms_max, args.steps)

        # the same workload with FP16 populations (16-bit deviation storage)
        h16 = lbrt.lb_rt_create(3, N_SIDE, N_SIDE, N_SIDE, dirset=lbrt.LB_RT_ICOSPHERE, level=LEVEL,
                                cfl=CFL, dx=1.0 / N_SIDE, bc=(lbrt.LB_RT_VACUUM,) * 3,
                                storage=lbrt.LB_RT_F16_DEV, stream=stream.cuda_stream)
        lbrt.lb_rt_set_fluid(h16, kappa_a=ka, eta=eta)
        lbrt.lb_rt_set_state(h16, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        lbrt.lb_rt_step(h16, args.warmup)
        stream.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            lbrt.lb_rt_step(h16, 1)
        f1.record(stream)
        f1.synchronize()
        ms16 = _max_over_ranks(ws, f0.elapsed_time(f1)) / args.steps
        lbrt.lb_rt_destroy(h16)

        # end to end through the C ABI with host buffers
        ka_h = torch.from_numpy(sp["kappa_a"]).pin_memory()
        eta_h = torch.from_numpy(sp["eta"]).pin_memory()
        E_h = torch.empty(sites, dtype=torch.float32).pin_memory()
        F_h = torch.empty((3, sites), dtype=torch.float32).pin_memory()
        for _ in range(2):
            lbrt.lb_rt_set_fluid(h, kappa_a=ka_h, eta=eta_h, mapped=True)
            lbrt.lb_rt_step_moments(h, 1, E_h, F_h)
        torch.cuda.synchronize()
        _barrier(ws)
        te = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            lbrt.lb_rt_set_fluid(h, kappa_a=ka_h, eta=eta_h, mapped=True)
            lbrt.lb_rt_step_moments(h, 1, E_h, F_h)
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - te
        e_ms = _max_over_ranks(ws, max(e0.elapsed_time(e1), wall * 1e3))
        e2e_value = sd_step * ws / (e_ms * 1e-3 / args.e2e_steps)
        lbrt.lb_rt_destroy(h)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    bytes_per_launch = sites * N * 8.0 + sites * 8.0   # populations r+w, kappa_a and eta fields
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch / (ms_step * 1e-3) / 1e9
    traffic = _traffic_from_profiles()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": sites, "ndir": N, "global_batch": ws,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (%.0f MB of populations per step)" % (sites * N * 4 / 1e6)},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * sites,
                "d2h_bytes_per_step": 4 * 4 * sites, "steps": args.e2e_steps,
                "route": "lb_rt_set_fluid(kappa_a, eta in pinned host memory, read in place "
                         "by the step kernel) + lb_rt_step_moments(1 step, E and F written "
                         "to pinned host memory by the step kernel)"},
        "clocks": ck,
        "f16": {"value": sd_step * ws / (ms16 * 1e-3), "unit": UNIT, "ms_per_step": ms16,
                "ratio_vs_f32": ms_step / ms16,
                "storage": "FP16 deviation from w_i E, float32 E per site, float32 arithmetic"},
    }
    if not args.no_collision_modes and ws == 1:
        try:
            line["collision_modes"] = collision_mode_costs()
        except Exception as e:  # report, do not hide
            line["collision_modes"] = {"error": str(e)[:300]}
    if not args.no_moving and ws == 1:
        try:
            line["diffusion_256"] = diffusion_costs()
        except Exception as e:  # report, do not hide
            line["diffusion_256"] = {"error": str(e)[:300]}
        try:
            line["moving_fluid"] = moving_fluid_costs()
        except Exception as e:  # report, do not hide
            line["moving_fluid"] = {"error": str(e)[:300]}
    if not args.no_serving and ws == 1:
        try:
            line["serving"] = serving_measurement()
        except Exception as e:  # report, do not hide
            line["serving"] = {"error": str(e)[:300]}
    if not args.no_cpu_baseline:
        try:
            sec, sd = oracle_sample_time(64, 1)
            line["cpu_baseline"] = {"value": sd / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "1 oracle step (FP64 numpy) of a 64^3 sub-box of the same workload, 42 dirs",
                                    "host_cores": len(os.sched_getaffinity(0))}
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
