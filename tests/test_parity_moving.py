"""GPU moving-fluid step (mixed-frame equation, App. B) against the FP64 oracle."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import Problem, TOL_F32, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level", [1, 2])
def test_moving_shear_reduced(cuda, level):
    """The moving-background generator on a 20^3 periodic box (|v| <= 0.6),
    density-scaled kt_a in [0.1, 100], kt_0 in [0, 100], eta_t = kt_a."""
    n = 20
    mf = W.moving_fluid(n)
    N = 42 if level == 1 else 162
    p = Problem(3, (n, n, n), "ico", level=level, moving=dict(v=mf["v"], kt_a=mf["kt_a"],
                kt_0=mf["kt_0"], eta_t=mf["eta_t"]),
                state=W.random_populations(N, (n, n, n), 31), budget=True)
    I, E, F, P, b = gpu_run(p, 12)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, 12)
    assert rel_l2(E, Eo) <= TOL_F32
    assert rel_l2(F, Fo) <= TOL_F32
    assert rel_l2(I, Io) <= TOL_F32
    assert abs(b["source"] - bo["source"]) <= 1e-5 * abs(bo["source"])


def test_moving_at_rest_equals_static(cuda):
    shape = (6, 8, 32)
    ka = W.random_fields(shape, 32, 0.0, 20.0)
    k0 = W.random_fields(shape, 33, 0.0, 30.0)
    eta = W.random_fields(shape, 34, 0.0, 3.0)
    st = W.random_populations(42, shape, 35)
    pm = Problem(3, shape, "ico", level=1, bc="vpv",
                 moving=dict(v=np.zeros((3,) + shape, dtype=np.float32), kt_a=ka, kt_0=k0, eta_t=eta),
                 state=st)
    ps = Problem(3, shape, "ico", level=1, bc="vpv", coef=dict(kappa_a=ka, kappa_0=k0, eta=eta),
                 state=st)
    Im = gpu_run(pm, 5)[0]
    Is = gpu_run(ps, 5)[0]
    assert rel_l2(Im, Is) < 1e-6


def test_moving_uniform_scalars_and_no_velocity(cuda):
    shape = (4, 5, 33)
    p = Problem(3, shape, "ico", level=1, moving=dict(v=None, kt_a=2.0, kt_0=5.0, eta_t=1.5),
                state=W.random_populations(42, shape, 36))
    I, E, F, P, b = gpu_run(p, 4)
    Io, Eo, *_ = oracle_run(p, 4)
    assert rel_l2(I, Io) <= TOL_F32
