#!/usr/bin/env python3
"""Benchmark of the grey radiative LB step (fused pull-stream + exact implicit
collision, Sec. 3.3) on its largest single-GPU configuration: optically thick
diffusion, 256^3 periodic sites x 162 directions (icosahedral geodesic level
2), pure isotropic scattering kappa_0 = 1e3 /L (kappa_0 dx = 3.9), Gaussian
initial E (sigma 8 cells) with isotropic populations, cfl 0.5.

Prints one JSON line.  The headline `value` is site-direction updates per
second of the float32-population step over the timed steps (inputs resident
in HBM: 22 GB of populations per step, far larger than L2).  Sub-lines, each
with its own roofline: the same configuration with FP16 and BF16
equilibrium-deviation storage (the storage the configuration names; float32
arithmetic), the radiating sphere 128^3 x 42 (FP32 and FP16) and the moving
background fluid 256^3 x 162 (App. B; FP32 and FP16).  `e2e` is the headline
metric through the C ABI with host buffers: every step hands a per-site
scattering opacity over in pinned host memory (lb_rt_set_fluid with
LB_RT_HOST_MAPPED, read in place by the step kernel), steps, and returns E
and F to pinned host memory (lb_rt_step_moments), as a coupled fluid code
does each step.  The FP64 oracle is timed on the host cores beside it, with
one thread and with every core.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun) runs independent replicas, one per GPU (weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 256
LEVEL = 2
KAPPA0_DX = 3.90625          # kappa_0 dx of the diffusion configuration (kappa_0 = 1e3 /L at 256^3)
SIGMA_CELLS = 8.0
CFL = 0.5
METRIC = "site-direction updates/s"
UNIT = "sd/s"
WORKLOAD = ("3D optically thick diffusion 256^3 x 162 dirs (icosahedral L2), periodic, pure "
            "scattering kappa_0 = 1e3 /L, Gaussian E0 (sigma 8 cells), cfl 0.5")


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


CSRC = os.path.join(ROOT, "paper_2007_05718_gb300", "csrc")
# the ncu summary of each timed kernel (traffic per launch, scaled to the
# bench size where the summary says so) and the sources it was captured from
PROFILES = {
    "c3_fp32": ("step_static_f32_diffusion256_162.md", ("kernels_tma.cu", "tma_common.cuh")),
    "c3_fp16": ("step_static_f16_diffusion256_162.md", ("kernels_tma16.cu", "tma_common.cuh")),
    "c3_bf16": ("step_static_bf16_diffusion256_162.md", ("kernels_tma16.cu", "tma_common.cuh")),
    "c2_fp32": ("step_static_f32_sphere128_42.md", ("kernels_tma.cu", "tma_common.cuh")),
    "c2_fp16": ("step_static_f16_sphere128_42.md", ("kernels_sc.cu", "tma_common.cuh")),
    "c5_fp32": ("step_moving_f32_shear128_162.md", ("kernels_tma_moving.cu", "tma_common.cuh")),
    "c5_fp16": ("step_moving_f16_shear128_162.md", ("kernels_tma16.cu", "tma_common.cuh")),
}


def kernel_source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(key):
    """DRAM bytes per launch of a line's kernel from its committed ncu
    summary, or None when there is none or the kernel source changed after
    the capture."""
    if key not in PROFILES:
        return None
    name, files = PROFILES[key]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        s = line.strip()
        if s.startswith(("traffic_bytes_per_launch", "kernel_source_sha256_16")) and ":" in s:
            k, v = s.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash(files):
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def roofline(key, bytes_per_launch, ms_per_launch):
    peak, kind = _peaks()
    achieved = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic(key), "peak_kind": kind, "algorithmic_bytes_per_launch": bytes_per_launch}


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
                 "--format=csv,noheader,nounits", "-lms", "20"],
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
                time.sleep(0.01)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.03)  # one more sample interval
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


# ---------------------------------------------------------------------------
# FP64 oracle on the host cores (the reference arm and the CPU baseline)
# ---------------------------------------------------------------------------

ORACLE_CODE = r"""
import sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import directions as D, lb
from paper_2007_05718_gb300 import workloads as W
n, steps = %(n)d, %(steps)d
nv, w = D.icosphere(%(level)d)
lat = lb.Lattice(3, (n, n, n), nv, w, cfl=%(cfl)r, dx=1.0 / n, bc=(lb.PERIODIC,) * 3)
co = lb.Static(kappa_0=%(k0dx)r * n)
I = lb.isotropic(W.gaussian_E0((n, n, n), %(sigma)r).astype(float), lat)
I = lb.step(I, lat, co)
t0 = time.perf_counter()
for _ in range(steps):
    I = lb.step(I, lat, co)
dt = time.perf_counter() - t0
print(json.dumps({"sec": dt, "sd": n ** 3 * len(w) * steps}))
"""


def oracle_time(n_side, steps, procs):
    """Run `procs` copies of the FP64 oracle (numpy as it stands, one thread
    each) at once, each on an n_side^3 periodic sub-box of the diffusion
    configuration (same kappa_0 dx, sigma and cfl), each in a fresh
    interpreter; returns (aggregate sd/s, seconds of the slowest copy)."""
    code = ORACLE_CODE % dict(root=ROOT, n=n_side, steps=steps, level=LEVEL, cfl=CFL, k0dx=KAPPA0_DX,
                              sigma=SIGMA_CELLS * n_side / N_SIDE if n_side < 64 else SIGMA_CELLS)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    sd, sec = 0.0, 0.0
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        d = json.loads(out.strip().splitlines()[-1])
        sd += d["sd"]
        sec = max(sec, d["sec"])
    return sd / sec, sec


def cpu_baselines(n_side=48, steps=6):
    cores = len(os.sched_getaffinity(0))
    one, t1 = oracle_time(n_side, steps, 1)
    allc, tall = oracle_time(n_side, steps, cores)
    sample = ("%d oracle steps (FP64 numpy) of a %d^3 periodic sub-box of the diffusion configuration "
              "(162 dirs, same kappa_0 dx and cfl)" % (steps, n_side))
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample + ", one copy per core at once; seconds %.1f" % tall,
            "one_thread": {"value": one, "unit": UNIT, "cores": 1, "sample": sample + ", seconds %.1f" % t1}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    n_sample = 40
    oracle_time(16, 1, 1)  # warm-up of the interpreter and numpy
    vals = []
    for _ in range(max(args.steps, 1) if args.steps <= 3 else 3):
        v, sec = oracle_time(n_sample, 2, cores)
        vals.append((v, sec))
    value = statistics.median(v for v, _ in vals)
    sec = statistics.median(s for _, s in vals)
    sample = ("%d^3 periodic sub-box of the diffusion configuration (162 dirs), 2 oracle steps per "
              "copy, one FP64 numpy copy per host core (%d) at once" % (n_sample, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (N_SIDE ** 3 * 162) / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sites": N_SIDE ** 3, "ndir": 162},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample + "; seconds per copy %.1f" % sec},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU lines
# ---------------------------------------------------------------------------

def _time_steps(lbrt, h, stream, steps):
    """CUDA-event time (ms) of `steps` single-step launches on the handle's stream."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        lbrt.lb_rt_step(h, 1)
    b.record(stream)
    b.synchronize()
    lbrt.lb_rt_sync(h)
    return a.elapsed_time(b), None


def diffusion_line(key, storage, steps, warmup, n=N_SIDE):
    """The diffusion configuration with the given storage: ms per step and its roofline."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    stream = torch.cuda.Stream()
    E0 = torch.from_numpy(W.gaussian_E0((n, n, n), SIGMA_CELLS)).cuda()
    h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=LEVEL, cfl=CFL, dx=1.0 / n,
                          bc=(lbrt.LB_RT_PERIODIC,) * 3, storage=storage, stream=stream.cuda_stream)
    try:
        lbrt.lb_rt_set_fluid(h, kappa_0=KAPPA0_DX * n)
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        lbrt.lb_rt_step(h, warmup)
        ms, _ = _time_steps(lbrt, h, stream, steps)
    finally:
        lbrt.lb_rt_destroy(h)
        torch.cuda.empty_cache()
    ms /= steps
    sites = n ** 3
    per_sd = 8.0 if storage == lbrt.LB_RT_F32 else 4.0
    per_site = 0.0 if storage == lbrt.LB_RT_F32 else 8.0   # E read + written (16-bit storage)
    nbytes = sites * (N * per_sd + per_site)
    return {"ms_per_step": ms, "value": sites * N / (ms * 1e-3), "unit": UNIT,
            "roofline": roofline(key, nbytes, ms)}


def sphere_line(key, storage, steps, warmup, n=128, kappa_r=10.0):
    """Radiating sphere 128^3 x 42 (vacuum faces, kappa_a R = 10): ms per step and roofline."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    sp = W.radiating_sphere(n, kappa_r)
    stream = torch.cuda.Stream()
    h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=1, cfl=CFL, dx=1.0 / n,
                          bc=(lbrt.LB_RT_VACUUM,) * 3, storage=storage, stream=stream.cuda_stream)
    try:
        lbrt.lb_rt_set_fluid(h, kappa_a=torch.from_numpy(sp["kappa_a"]).cuda(),
                             eta=torch.from_numpy(sp["eta"]).cuda())
        lbrt.lb_rt_set_state(h, torch.from_numpy(sp["E0"]).cuda(), lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        lbrt.lb_rt_step(h, warmup)
        ms, _ = _time_steps(lbrt, h, stream, steps)
    finally:
        lbrt.lb_rt_destroy(h)
        torch.cuda.empty_cache()
    ms /= steps
    sites = n ** 3
    per_sd = 8.0 if storage == lbrt.LB_RT_F32 else 4.0
    per_site = 8.0 if storage == lbrt.LB_RT_F32 else 16.0   # kappa_a, eta (+ E r/w in 16-bit)
    nbytes = sites * (N * per_sd + per_site)
    return {"ms_per_step": ms, "value": sites * N / (ms * 1e-3), "unit": UNIT,
            "roofline": roofline(key, nbytes, ms),
            "workload": "radiating sphere 128^3 x 42, vacuum faces, kappa_a R = 10"}


def moving_line(key, storage, steps, warmup, n=256, level=2):
    """Moving background fluid (App. B), 256^3 x 162 periodic, the seeded
    shear flow: ms per step and roofline."""
    import torch
    from paper_2007_05718_gb300 import lbrt
    from paper_2007_05718_gb300 import workloads as W
    mf = W.moving_fluid(n)
    fields = {k: torch.from_numpy(mf[k]).cuda() for k in ("v", "kt_a", "kt_0", "eta_t")}
    stream = torch.cuda.Stream()
    h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=level, cfl=CFL,
                          moving=True, storage=storage, stream=stream.cuda_stream)
    try:
        lbrt.lb_rt_set_fluid(h, **fields)
        lbrt.lb_rt_set_state(h, torch.ones((n, n, n), dtype=torch.float32, device="cuda"),
                             lbrt.LB_RT_STATE_ISOTROPIC)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        lbrt.lb_rt_step(h, warmup)
        ms, _ = _time_steps(lbrt, h, stream, steps)
    finally:
        lbrt.lb_rt_destroy(h)
        del fields
        torch.cuda.empty_cache()
    ms /= steps
    sites = n ** 3
    per_sd = 8.0 if storage == lbrt.LB_RT_F32 else 4.0
    per_site = 24.0 if storage == lbrt.LB_RT_F32 else 32.0   # v, kt_a, kt_0, eta_t (+ E r/w)
    nbytes = sites * (N * per_sd + per_site)
    return {"ms_per_step": ms, "value": sites * N / (ms * 1e-3), "unit": UNIT,
            "roofline": roofline(key, nbytes, ms),
            "workload": "moving fluid 256^3 x 162 periodic shear flow (|v| <= 0.6), density-scaled opacities"}


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
        ms, _ = _time_steps(lbrt, h, stream, steps)
        out[name + "_ms"] = ms / steps
        lbrt.lb_rt_destroy(h)
    out["implicit_over_explicit"] = out["implicit_exact_ms"] / out["explicit_ms"]
    out["lambda5_over_explicit"] = out["lambda_5_ms"] / out["explicit_ms"]
    out["workload"] = "128^3 x 42 periodic, kappa_a 1, kappa_0 1e3, lambda 0.5, eta 1, FP32"
    return out


def serving_measurement(n_capacity=24, n_open=150, seed=20200711, steps_per_tick=50):
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
    # capacity with one launch per direction group and step, then with the
    # autotuner free to pair the 42- and 162-direction groups in one launch
    rs = serve.serve(closed, steps_per_tick=steps_per_tick, max_problems=64, pair_groups=0)
    rc = serve.serve(closed, steps_per_tick=steps_per_tick, max_problems=64, pair_groups=2)
    cap = rc["throughput_req_s"]
    rate = 0.8 * cap
    stream = W.serving_requests(n_open, seed=seed, rate=rate)
    ro = serve.serve(stream, steps_per_tick=steps_per_tick, max_problems=64)
    return {
        "capacity_req_s": cap, "capacity_sd_s": rc["throughput_sd_s"],
        "capacity_separate_launches_req_s": rs["throughput_req_s"],
        "capacity_paired_ticks": rc["paired_ticks"], "capacity_ticks": rc["ticks"],
        "paired_ticks": ro["paired_ticks"],
        "arrival_rate_req_s": rate, "requests": ro["requests"], "completed": ro["completed"],
        "p50_s": ro["p50_s"], "p99_s": ro["p99_s"], "throughput_req_s": ro["throughput_req_s"],
        "throughput_sd_s": ro["throughput_sd_s"], "max_concurrent": ro["max_concurrent"],
        "ticks": ro["ticks"], "storage": "fp16",
        "steps_per_tick": steps_per_tick,
        "sample": "first %d requests of the seed-%d stream (closed loop) and first %d with Poisson "
                  "arrivals at 0.8 x capacity; the configured stream has 2000" % (n_capacity, seed, n_open),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle samples")
    ap.add_argument("--e2e-steps", type=int, default=10, help="coupled steps of the end-to-end run")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched serving run")
    ap.add_argument("--serving-requests", type=int, default=150,
                    help="requests of the seed-20200711 stream served in the open-loop run (2000 = all)")
    ap.add_argument("--no-collision-modes", action="store_true",
                    help="skip the implicit / explicit / Lambda-5 timing")
    ap.add_argument("--no-sublines", action="store_true",
                    help="skip the FP16/BF16, sphere and moving-fluid sub-lines")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_05718_gb300 import build, lbrt
    from paper_2007_05718_gb300 import workloads as W
    build.build()
    n = N_SIDE
    sites = n ** 3
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = lbrt.lb_rt_create(3, n, n, n, dirset=lbrt.LB_RT_ICOSPHERE, level=LEVEL, cfl=CFL,
                              dx=1.0 / n, bc=(lbrt.LB_RT_PERIODIC,) * 3, stream=stream.cuda_stream)
        lbrt.lb_rt_set_fluid(h, kappa_0=KAPPA0_DX * n)
        E0 = torch.from_numpy(W.gaussian_E0((n, n, n), SIGMA_CELLS)).cuda()
        lbrt.lb_rt_set_state(h, E0, lbrt.LB_RT_STATE_ISOTROPIC)
        del E0
        N = lbrt.lb_rt_directions(h)[0].shape[0]
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
        lbrt.lb_rt_sync(h)
        ms_max = _max_over_ranks(ws, ms)
        ms_step = ms_max / args.steps
        sd_step = sites * N
        value = aggregate_rate(sd_step, ws, ms_max, args.steps)

        # end to end through the C ABI with host buffers: a per-site kappa_0
        # field in from pinned host memory, E and F out to pinned host memory
        k0_h = torch.full((n, n, n), KAPPA0_DX * n, dtype=torch.float32).pin_memory()
        E_h = torch.empty(sites, dtype=torch.float32).pin_memory()
        F_h = torch.empty((3, sites), dtype=torch.float32).pin_memory()
        for _ in range(2):
            lbrt.lb_rt_set_fluid(h, kappa_0=k0_h, mapped=True)
            lbrt.lb_rt_step_moments(h, 1, E_h, F_h)
        torch.cuda.synchronize()
        _barrier(ws)
        te = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            lbrt.lb_rt_set_fluid(h, kappa_0=k0_h, mapped=True)
            lbrt.lb_rt_step_moments(h, 1, E_h, F_h)
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - te
        e_ms = _max_over_ranks(ws, max(e0.elapsed_time(e1), wall * 1e3))
        e2e_value = sd_step * ws / (e_ms * 1e-3 / args.e2e_steps)
        lbrt.lb_rt_destroy(h)
        del k0_h, E_h, F_h
        torch.cuda.empty_cache()

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    bytes_per_launch = sites * N * 8.0   # populations read and written; kappa_0 is a scalar
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + ", FP32 populations", "sites": sites, "ndir": N,
                   "storage": "fp32", "global_batch": ws,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (%.1f GB of populations per step)" % (sites * N * 4 / 1e9)},
        "gpu_launches": args.steps,
        "roofline": roofline("c3_fp32", bytes_per_launch, ms_step),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * sites,
                "d2h_bytes_per_step": 4 * 4 * sites, "steps": args.e2e_steps,
                "route": "lb_rt_set_fluid(kappa_0 per site in pinned host memory, read in place by "
                         "the step kernel) + lb_rt_step_moments(1 step, E and F written to pinned "
                         "host memory by the step kernel)"},
        "clocks": ck,
    }
    if not args.no_sublines and ws == 1:
        sub = {}
        few = max(3, min(args.steps, 20))
        for key, fn, st, steps in (
                ("c3_fp16", diffusion_line, lbrt.LB_RT_F16_DEV, few),
                ("c3_bf16", diffusion_line, lbrt.LB_RT_BF16_DEV, few),
                ("c2_fp32", sphere_line, lbrt.LB_RT_F32, max(3, min(args.steps, 200))),
                ("c2_fp16", sphere_line, lbrt.LB_RT_F16_DEV, max(3, min(args.steps, 200))),
                ("c5_fp32", moving_line, lbrt.LB_RT_F32, few),
                ("c5_fp16", moving_line, lbrt.LB_RT_F16_DEV, few)):
            try:
                sub[key] = fn(key, st, steps, args.warmup)
            except Exception as e:  # report, do not hide
                sub[key] = {"error": str(e)[:300]}
        line["sublines"] = sub
        try:
            line["fp16_over_fp32"] = {
                "diffusion_256_162": ms_step / sub["c3_fp16"]["ms_per_step"],
                "bf16_diffusion_256_162": ms_step / sub["c3_bf16"]["ms_per_step"],
                "sphere_128_42": sub["c2_fp32"]["ms_per_step"] / sub["c2_fp16"]["ms_per_step"],
                "moving_256_162": sub["c5_fp32"]["ms_per_step"] / sub["c5_fp16"]["ms_per_step"]}
        except Exception:
            pass
    if not args.no_collision_modes and ws == 1:
        try:
            line["collision_modes"] = collision_mode_costs()
        except Exception as e:  # report, do not hide
            line["collision_modes"] = {"error": str(e)[:300]}
    if not args.no_serving and ws == 1:
        try:
            line["serving"] = serving_measurement(n_open=args.serving_requests)
        except Exception as e:  # report, do not hide
            line["serving"] = {"error": str(e)[:300]}
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baselines()
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
