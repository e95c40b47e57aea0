"""The allocation-free energy reduction (lb_rt_total_energy_noalloc).

Callers that cannot allocate device memory where they need the number use
this entry point; it must agree with the library's regular FP64 energy
reduction (the total reported by lb_rt_moments right after lb_rt_set_state),
on two calls in a row since all calls share one static scratch array."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import TOL_F32, Problem, make_handle

pytestmark = pytest.mark.gpu


def _reference_total(p):
    h = make_handle(p)
    try:
        total = lbrt.lb_rt_moments(h, budget=True)["total"]
        return h, total
    except Exception:
        lbrt.lb_rt_destroy(h)
        raise


@pytest.mark.parametrize("shape,level", [((9, 13, 40), 1), ((24, 24, 24), 2)])
def test_noalloc_total_matches_regular_reduction(cuda, shape, level):
    import torch
    N = 42 if level == 1 else 162
    p = Problem(3, shape, "ico", level=level, state=W.random_populations(N, shape, 61))
    h, expected = _reference_total(p)
    try:
        sites = int(np.prod(shape))
        pops = torch.empty((N, sites), device="cuda", dtype=torch.float32)
        lbrt.lb_rt_get_populations(h, pops)
        torch.cuda.synchronize()
        first = lbrt.lb_rt_total_energy_noalloc(pops, N, sites)
        out = torch.zeros(1, device="cuda", dtype=torch.float64)
        lbrt.lb_rt_total_energy_noalloc(pops, N, sites, out=out)
        torch.cuda.synchronize()
        second = float(out.item())
    finally:
        lbrt.lb_rt_destroy(h)
    assert abs(first - expected) <= TOL_F32 * abs(expected)
    assert abs(second - expected) <= TOL_F32 * abs(expected)


def test_noalloc_rejects_oversize_and_bad_arguments(cuda):
    import torch
    pops = torch.zeros((1, 8), device="cuda", dtype=torch.float32)
    with pytest.raises(lbrt.LBRTError):
        lbrt.lb_rt_total_energy_noalloc(pops, 1, 16_777_217)
    with pytest.raises(lbrt.LBRTError):
        lbrt.lb_rt_total_energy_noalloc(pops, 0, 8)
