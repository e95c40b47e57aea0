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
        # an independent FP64 sum of the very same array, on the host
        host_sum = float(np.sum(pops.cpu().numpy().astype(np.float64)))
    finally:
        lbrt.lb_rt_destroy(h)
    assert abs(first - expected) <= TOL_F32 * abs(expected)
    assert abs(second - expected) <= TOL_F32 * abs(expected)
    # the kernel sums a site's directions in float32, then sites in FP64
    assert abs(first - host_sum) <= TOL_F32 * abs(host_sum)
    assert abs(second - host_sum) <= TOL_F32 * abs(host_sum)


def test_noalloc_rejects_oversize_and_bad_arguments(cuda):
    """The C entry point itself refuses, before any launch, sizes beyond its
    fixed scratch array, a zero direction count and host memory where it
    needs device memory (called here through the raw C ABI, since the
    binding refuses most of these on its own)."""
    import ctypes as C
    import torch
    lib = lbrt.load()
    pops = torch.zeros((1, 8), device="cuda", dtype=torch.float32)
    res = C.c_double()
    st = lib.lb_rt_total_energy_noalloc(pops.data_ptr(), 1, 16_777_217, C.byref(res),
                                        lbrt.LB_RT_HOST, None)
    assert st == lbrt.LB_RT_EINVAL and "limit" in lbrt.lb_rt_last_error(None)
    st = lib.lb_rt_total_energy_noalloc(pops.data_ptr(), 0, 8, C.byref(res), lbrt.LB_RT_HOST, None)
    assert st == lbrt.LB_RT_EINVAL
    host = np.zeros(8, dtype=np.float32)
    st = lib.lb_rt_total_energy_noalloc(host.ctypes.data, 1, 8, C.byref(res), lbrt.LB_RT_HOST, None)
    assert st == lbrt.LB_RT_EINVAL and "device" in lbrt.lb_rt_last_error(None)
    hout = np.zeros(1, dtype=np.float64)
    st = lib.lb_rt_total_energy_noalloc(pops.data_ptr(), 1, 8, hout.ctypes.data,
                                        lbrt.LB_RT_DEVICE, None)
    assert st == lbrt.LB_RT_EINVAL
    # a valid call still works after the refusals
    assert lbrt.lb_rt_total_energy_noalloc(pops, 1, 8) == 0.0
