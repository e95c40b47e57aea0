"""Continuous-batching request loop over the batch C ABI (lb_rt_batch_*).

Radiative-transfer solves arrive over time (each a radiating-sphere or
shadow problem of its own grid size, direction count, opacity and step
count); the loop admits every arrived request whose device buffers fit the
batch's memory budget (first come, first served), keeps admitted problems
resident, advances all of them together one tick at a time (one persistent
kernel launch per direction group and step, replayed from a CUDA graph) and
retires a problem as soon as the tick with its last step has completed.
Ticks are pipelined: the loop enqueues the next tick while the previous one
runs (the batch keeps two in flight), and admissions run on the problems'
own streams meanwhile, so the device does not wait for the host between
ticks.  Requests that arrive while others are on the GPU join at the next
tick.  Reported: per-request time to solution (completion minus arrival),
its p50/p99, and throughput in requests/s and site-direction updates/s.

All stepping runs in liblbrt.so; this module schedules and marshals only.
"""
import collections
import time

import numpy as np

from . import lbrt
from . import workloads as W


def request_problem(req, cfl=0.5):
    """(problem kwargs, fluid kwargs, initial E0) of one serving request:
    sphere = homogeneous radiating sphere of radius 0.25 with kappa_a = eta =
    kappa inside (1/L units); shadow = emitting sphere (radius 0.125,
    kappa_a = eta = kappa) in front of a black absorber (kappa_a = 1e4)."""
    n = req["n"]
    if req["kind"] == "sphere":
        f = W.radiating_sphere(n, req["kappa"] * 0.25)
    else:
        f = W.shadow(n, req["kappa"])
    level = 1 if req["ndir"] == 42 else 2
    problem = dict(dims=3, nx=n, ny=n, nz=n, dirset=lbrt.LB_RT_ICOSPHERE, level=level, cfl=cfl,
                   bc=(lbrt.LB_RT_VACUUM,) * 3)
    return problem, dict(kappa_a=f["kappa_a"], eta=f["eta"]), f["E0"]


def percentile(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else None


def serve(requests, *, storage=lbrt.LB_RT_F16_DEV, steps_per_tick=50, max_problems=64,
          mem_budget=0, use_graph=True, autotune=True, keep_results=False, timeout_s=None,
          pair_groups=2):
    """Run the request stream (dicts with id, arrival [s], kind, n, ndir,
    kappa, steps) through one batch.  Arrival times are honoured on the wall
    clock from the call's start.  Returns a report dict; with keep_results
    the final E [n^3] and F [3, n^3] of every request are included.
    pair_groups as lb_rt_batch_create: by default the autotuner decides
    whether the 42- and 162-direction requests share one launch per step."""
    b = lbrt.lb_rt_batch_create(max_problems=max_problems, storage=storage,
                                steps_per_tick=steps_per_tick, mem_budget=mem_budget,
                                use_graph=use_graph, autotune=autotune, pair_groups=pair_groups)
    pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
    waiting = collections.deque()
    active = {}
    done = {}
    results = {}
    ticks = 0
    paired_ticks = 0
    max_active = 0
    t0 = time.perf_counter()
    try:
        while pending or waiting or active:
            now = time.perf_counter() - t0
            if timeout_s is not None and now > timeout_s:
                break
            while pending and pending[0]["arrival"] <= now:
                waiting.append(pending.popleft())
            while waiting:
                req = waiting[0]
                problem, fluid, E0 = request_problem(req)
                slot = lbrt.lb_rt_batch_admit(b, problem, fluid, E0, lbrt.LB_RT_STATE_ISOTROPIC,
                                              req["steps"])
                if slot is None:
                    if not active:
                        raise RuntimeError("request %d does not fit an empty batch" % req["id"])
                    break
                waiting.popleft()
                active[slot] = (req, time.perf_counter() - t0)
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0]["arrival"] - now)))
                continue
            max_active = max(max_active, len(active))
            if lbrt.lb_rt_batch_tick(b) > 0:
                ticks += 1
                if pair_groups and any(lbrt.lb_rt_batch_plan(b, s)[2] for s in active):
                    paired_ticks += 1
            else:
                # every step of the admitted problems is enqueued: wait for
                # the ticks in flight so that the finished ones can retire
                lbrt.lb_rt_batch_sync(b)
            for slot in lbrt.lb_rt_batch_poll(b):
                req, t_admit = active.pop(slot)
                if keep_results:
                    S = req["n"] ** 3
                    E = np.zeros(S, dtype=np.float32)
                    F = np.zeros((3, S), dtype=np.float32)
                    lbrt.lb_rt_batch_moments(b, slot, E, F)
                    results[req["id"]] = (E, F)
                lbrt.lb_rt_batch_release(b, slot)
                t_done = time.perf_counter() - t0
                done[req["id"]] = dict(arrival=req["arrival"], admitted=t_admit, done=t_done,
                                       latency=t_done - req["arrival"])
    finally:
        lbrt.lb_rt_batch_destroy(b)
    wall = time.perf_counter() - t0
    lat = [d["latency"] for d in done.values()]
    sd = sum(r["n"] ** 3 * r["ndir"] * r["steps"] for r in requests if r["id"] in done)
    t_first = min((r["arrival"] for r in requests), default=0.0)
    span = max((d["done"] for d in done.values()), default=wall) - t_first
    rep = {
        "requests": len(requests), "completed": len(done), "ticks": ticks,
        "paired_ticks": paired_ticks,
        "max_concurrent": max_active, "wall_s": wall,
        "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
        "throughput_req_s": len(done) / span if span > 0 else None,
        "throughput_sd_s": sd / span if span > 0 else None,
        "site_direction_updates": sd, "storage": storage, "steps_per_tick": steps_per_tick,
        "per_request": done,
    }
    if keep_results:
        rep["results"] = results
    return rep


def run_alone(req, *, storage=lbrt.LB_RT_F16_DEV, steps_per_tick=50):
    """The request solved by itself in a fresh batch (for the alone-vs-mix check)."""
    r = dict(req, arrival=0.0)
    rep = serve([r], storage=storage, steps_per_tick=steps_per_tick, max_problems=1,
                keep_results=True)
    return rep["results"][req["id"]]
