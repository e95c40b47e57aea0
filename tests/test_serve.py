"""Continuous-batching serving loop: requests arrive while others run, are
admitted as memory frees up, and each result equals the same request solved
alone; small requests are also checked against the FP64 oracle."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt, serve
from paper_2007_05718_gb300 import workloads as W
from parity import Problem, oracle_run, pad_F, rel_l2

pytestmark = pytest.mark.gpu


def _stream(count, seed, rate):
    return W.serving_requests(count, seed=seed, sizes=(16, 24, 32, 40), steps=(20, 90), rate=rate)


def test_mix_equals_alone_and_overlap(cuda):
    reqs = _stream(24, 20200711, rate=400.0)
    b = lbrt.lb_rt_batch_create(max_problems=4, storage=lbrt.LB_RT_F16_DEV)
    try:
        # a memory budget for roughly six mid-size problems: admission waits
        per = lbrt.lb_rt_batch_problem_bytes(b, dims=3, nx=32, ny=32, nz=32,
                                             dirset=lbrt.LB_RT_ICOSPHERE, level=2)
    finally:
        lbrt.lb_rt_batch_destroy(b)
    rep = serve.serve(reqs, steps_per_tick=16, max_problems=16, mem_budget=6 * per,
                      keep_results=True)
    assert rep["completed"] == len(reqs)
    assert rep["max_concurrent"] > 1                 # work overlapped on the device
    assert rep["p99_s"] >= rep["p50_s"] > 0
    for req in reqs[::3]:
        E, F = serve.run_alone(req, steps_per_tick=16)
        Em, Fm = rep["results"][req["id"]]
        assert np.array_equal(E, Em) and np.array_equal(F, Fm)


def test_served_results_against_oracle(cuda):
    reqs = [dict(id=0, arrival=0.0, kind="sphere", n=16, ndir=42, kappa=40.0, steps=30),
            dict(id=1, arrival=0.0, kind="shadow", n=16, ndir=162, kappa=3.0, steps=25)]
    rep = serve.serve(reqs, steps_per_tick=8, keep_results=True)
    for req in reqs:
        problem, fluid, E0 = serve.request_problem(req)
        n = req["n"]
        p = Problem(3, (n, n, n), "ico", level=problem["level"], bc="vvv", coef=fluid,
                    state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=E0)
        Io, Eo, Fo, Po, bo, lat = oracle_run(p, req["steps"])
        E, F = rep["results"][req["id"]]
        assert rel_l2(E.reshape(n, n, n), Eo) <= 2e-3
        assert rel_l2(F.reshape(3, n, n, n), pad_F(Fo, 3)) <= 2e-3
