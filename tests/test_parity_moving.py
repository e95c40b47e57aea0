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


@pytest.mark.parametrize("storage,tol", [(lbrt.LB_RT_F32, TOL_F32), (lbrt.LB_RT_F16_DEV, 2e-3)])
def test_moving_large_direction_set_site_kernel(cuda, storage, tol):
    """192 Gauss-Legendre directions (12 in mu x 16 in phi, four upwind
    classes of 48) fit none of the tile plans of the moving kernels (at most
    176 internal directions), so the step runs on the one-thread-per-site
    kernel; it must match the oracle like the tiled kernels do."""
    shape = (6, 7, 9)
    v = 0.5 * np.stack([W.smooth_field(shape, 81 + k) for k in range(3)]).astype(np.float32) / 3.0
    p = Problem(3, shape, "gl", gl=(12, 16), bc="pvp", storage=storage,
                moving=dict(v=v, kt_a=W.random_fields(shape, 85, 0.0, 10.0),
                            kt_0=W.random_fields(shape, 86, 0.0, 20.0), eta_t=1.0),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC,
                state=(1.0 + 0.5 * W.smooth_field(shape, 87)).astype(np.float32))
    I, E, F, P, b = gpu_run(p, 6)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, 6)
    assert rel_l2(E, Eo) <= tol
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Eo) <= tol


@pytest.fixture(scope="module")
def c5_48():
    """The moving-fluid configuration's generator on 48^3 (ico-162, periodic),
    a seeded P1 start, and the oracle's 10 steps of it (computed once)."""
    n, steps = 48, 10
    mf = W.moving_fluid(n)
    E0, F0 = W.random_moments((n, n, n), 49)
    mov = dict(v=mf["v"], kt_a=mf["kt_a"], kt_0=mf["kt_0"], eta_t=mf["eta_t"])
    state = np.concatenate([E0[None], F0]).astype(np.float32)
    p = Problem(3, (n, n, n), "ico", level=2, moving=mov, state_kind=lbrt.LB_RT_STATE_P1, state=state)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, steps)
    return dict(mov=mov, state=state, steps=steps, Eo=Eo, Fo=Fo, n=n)


@pytest.mark.parametrize("storage,tol", [(lbrt.LB_RT_F32, TOL_F32), (lbrt.LB_RT_F16_DEV, 2e-3)])
def test_c5_48_cubed_ten_steps(cuda, c5_48, storage, tol):
    """Ten mixed-frame steps (App. B) of the 48^3 instance of the moving-fluid
    configuration against the FP64 oracle: E and F within 1e-5 (FP32
    populations) or 2e-3 (FP16)."""
    n = c5_48["n"]
    p = Problem(3, (n, n, n), "ico", level=2, storage=storage, moving=c5_48["mov"],
                state_kind=lbrt.LB_RT_STATE_P1, state=c5_48["state"])
    I, E, F, P, b = gpu_run(p, c5_48["steps"])
    assert rel_l2(E, c5_48["Eo"]) <= tol
    assert np.linalg.norm(F - c5_48["Fo"]) / np.linalg.norm(c5_48["Eo"]) <= tol
