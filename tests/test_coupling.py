"""Coupling outputs on the GPU (lb_rt_coupling) against the oracle's
transform of the oracle's moments after a few moving-fluid steps."""
import numpy as np
import pytest

from oracle import coupling as CP
from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import Problem, TOL_F32, make_handle, oracle_run, pad_F, rel_l2

pytestmark = pytest.mark.gpu


def _gpu_coupling(p, steps):
    h = make_handle(p)
    try:
        lbrt.lb_rt_step(h, steps)
        S_ = int(np.prod(p.shape))
        J = np.zeros(S_, dtype=np.float32)
        H = np.zeros((3, S_), dtype=np.float32)
        S = np.zeros((4, S_), dtype=np.float32)
        lbrt.lb_rt_coupling(h, J, H, S)
        return J.reshape(p.shape), H.reshape((3,) + p.shape), S.reshape((4,) + p.shape)
    finally:
        lbrt.lb_rt_destroy(h)


@pytest.mark.parametrize("storage,tol", [(lbrt.LB_RT_F32, 1e-5), (lbrt.LB_RT_F16_DEV, 2e-3)])
def test_coupling_moving_shear(cuda, storage, tol):
    n = 16
    mf = W.moving_fluid(n)
    shape = (n, n, n)
    E0 = 1.0 + W.smooth_field(shape, 61).astype(np.float32)
    F0 = 0.2 * np.stack([W.smooth_field(shape, 62 + k) for k in range(3)]).astype(np.float32)
    p = Problem(3, shape, "ico", level=1, storage=storage,
                moving=dict(v=mf["v"], kt_a=mf["kt_a"], kt_0=mf["kt_0"], eta_t=mf["eta_t"]),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]))
    J, H, S = _gpu_coupling(p, 6)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, 6)
    v = mf["v"].astype(np.float64)
    S0, Sj, Jo, Ho, H0 = CP.four_force(Eo, Fo, Po, v,
                                       mf["kt_a"].astype(np.float64), mf["kt_0"].astype(np.float64),
                                       mf["eta_t"].astype(np.float64))
    assert rel_l2(J, Jo) <= tol
    # H and S are differences of nearly equal terms: scale by |J|
    scale = np.linalg.norm(Jo)
    assert np.linalg.norm(H - Ho) / scale <= tol
    assert np.linalg.norm(S[0] - S0) / np.linalg.norm(S0) <= tol
    assert np.linalg.norm(S[1:] - Sj) / np.linalg.norm(S0) <= tol


def test_coupling_static_handle_is_rest_frame(cuda):
    shape = (6, 7, 33)
    ka = W.random_fields(shape, 71, 0.0, 5.0)
    p = Problem(3, shape, "ico", level=1, bc="vpv", coef=dict(kappa_a=ka, kappa_0=3.0, eta=1.0),
                state=W.random_populations(42, shape, 72))
    J, H, S = _gpu_coupling(p, 3)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, 3)
    assert rel_l2(J, Eo) <= TOL_F32
    assert np.linalg.norm(H - pad_F(Fo, 3)) / np.linalg.norm(Eo) <= TOL_F32
    S0 = ka.astype(np.float64) * Eo - 1.0
    assert np.linalg.norm(S[0] - S0) / np.linalg.norm(S0) <= TOL_F32
    Sj = (ka.astype(np.float64) + 3.0)[None] * pad_F(Fo, 3)
    assert np.linalg.norm(S[1:] - Sj) / np.linalg.norm(S0) <= TOL_F32
