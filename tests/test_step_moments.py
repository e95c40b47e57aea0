"""lb_rt_step_moments: E and F of the new state written by the step kernel's
collision epilogue (E' = alpha E* + c0, F' = alpha F* + c1 / d for an
isotropic table), against lb_rt_step + lb_rt_moments and the FP64 oracle,
for every output route (device buffers, page-locked host memory written by
the kernel, other host memory written directly where the device addresses it
and through a device buffer elsewhere) and for the cases
that fall back to the separate moments pass."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import TOL_F32, Problem, make_handle, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _plain(p, steps):
    """lb_rt_step + lb_rt_moments (the reference route), host outputs."""
    h = make_handle(p)
    try:
        lbrt.lb_rt_step(h, steps)
        S = int(np.prod(p.shape))
        E = np.zeros(S, dtype=np.float32)
        F = np.zeros((3, S), dtype=np.float32)
        lbrt.lb_rt_moments(h, E, F)
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        I = np.zeros((N, S), dtype=np.float32)
        lbrt.lb_rt_get_populations(h, I)
        return E, F, I
    finally:
        lbrt.lb_rt_destroy(h)


def _fused(p, steps, route):
    import torch
    h = make_handle(p)
    try:
        S = int(np.prod(p.shape))
        if route == "device":
            E = torch.zeros(S, dtype=torch.float32, device="cuda")
            F = torch.zeros((3, S), dtype=torch.float32, device="cuda")
        elif route == "pinned":
            E = torch.zeros(S, dtype=torch.float32).pin_memory()
            F = torch.zeros((3, S), dtype=torch.float32).pin_memory()
        else:
            E = np.zeros(S, dtype=np.float32)
            F = np.zeros((3, S), dtype=np.float32)
        lbrt.lb_rt_step_moments(h, steps, E, F)
        if route == "device":
            torch.cuda.synchronize()
        E = E.cpu().numpy() if hasattr(E, "cpu") else E
        F = F.cpu().numpy() if hasattr(F, "cpu") else F
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        I = np.zeros((N, S), dtype=np.float32)
        lbrt.lb_rt_get_populations(h, I)
        return E, F, I
    finally:
        lbrt.lb_rt_destroy(h)


def _sphere(n=32):
    sp = W.radiating_sphere(n, 10.0)
    return Problem(3, (n, n, n), "ico", level=1, cfl=0.5, bc="vvv",
                   coef=dict(kappa_a=sp["kappa_a"], eta=sp["eta"]),
                   state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=sp["E0"])


def test_routes_agree_and_match_the_separate_pass_and_the_oracle(cuda):
    p = _sphere()
    steps = 12
    E2, F2, I2 = _plain(p, steps)
    got = {r: _fused(p, steps, r) for r in ("device", "pinned", "pageable")}
    for r in ("pinned", "pageable"):
        np.testing.assert_array_equal(got[r][0], got["device"][0])
        np.testing.assert_array_equal(got[r][1], got["device"][1])
    E1, F1, I1 = got["device"]
    # the populations are those of the plain step, bit for bit
    np.testing.assert_array_equal(I1, I2)
    assert rel_l2(E1, E2) < 2e-6 and rel_l2(F1, F2) < 2e-6
    _, Eo, Fo, _, _, _ = oracle_run(p, steps)
    assert rel_l2(E1.reshape(p.shape), Eo) <= TOL_F32
    assert rel_l2(F1.reshape((3,) + p.shape), Fo) <= TOL_F32


@pytest.mark.parametrize("collision", ["implicit", "explicit", "lambda"])
def test_ragged_periodic_random_fields(cuda, collision):
    shape = (13, 21, 37)
    co = dict(kappa_a=W.random_fields(shape, 1), kappa_0=W.random_fields(shape, 2, 0.5, 3.0),
              lam=W.random_fields(shape, 3, -0.5, 0.5), eta=W.random_fields(shape, 4))
    if collision == "explicit":
        co = {k: v * 0.3 for k, v in co.items()}
    p = Problem(3, shape, "ico", level=1, cfl=0.5, bc="ppv", collision=collision,
                lambda_iters=3, coef=co, state=W.random_populations(42, shape, 5))
    E2, F2, _ = _plain(p, 7)
    E1, F1, _ = _fused(p, 7, "pinned")
    assert rel_l2(E1, E2) < 3e-6 and rel_l2(F1, F2) < 3e-6


@pytest.mark.parametrize("bc", ["ppp", "vvv"])
def test_162_directions_epilogue(cuda, bc):
    """The E, F epilogue of the 162-direction tile plan (16 direction warps,
    one plane per batch), periodic and vacuum faces."""
    shape = (10, 12, 70)
    co = dict(kappa_a=W.random_fields(shape, 21), kappa_0=W.random_fields(shape, 22, 0.5, 3.0),
              eta=W.random_fields(shape, 23))
    p = Problem(3, shape, "ico", level=2, cfl=0.5, bc=bc, coef=co,
                state=W.random_populations(162, shape, 24))
    E2, F2, I2 = _plain(p, 4)
    E1, F1, I1 = _fused(p, 4, "device")
    np.testing.assert_array_equal(I1, I2)
    assert rel_l2(E1, E2) < 3e-6
    assert np.linalg.norm(F1 - F2) / np.linalg.norm(E2) < 3e-6
    _, Eo, Fo, _, _, _ = oracle_run(p, 4)
    assert rel_l2(E1.reshape(p.shape), Eo) <= TOL_F32


def test_2d_ring_with_forward_peaked_scattering(cuda):
    shape = (1, 24, 40)
    p = Problem(2, shape, "ring", ndir=16, ring_offset=0.3, cfl=0.7, bc="ppp",
                coef=dict(kappa_0=2.0 * 40, lam=0.5), state=W.random_populations(16, shape, 7))
    E2, F2, _ = _plain(p, 9)
    E1, F1, _ = _fused(p, 9, "device")
    # near isotropy |F| ~ 1e-3 E: the two summation orders differ by float32
    # rounding of E-sized terms, so F is compared on the scale of E
    assert rel_l2(E1, E2) < 2e-6
    assert np.linalg.norm(F1 - F2) / np.linalg.norm(E2) < 2e-6
    assert np.all(F1[2] == 0.0)


@pytest.mark.parametrize("case", ["f16", "frozen", "moving", "zero_steps"])
def test_fallback_cases_equal_the_separate_pass(cuda, case):
    n = 16
    sp = W.radiating_sphere(n, 10.0)
    kw = dict(coef=dict(kappa_a=sp["kappa_a"], eta=sp["eta"]),
              state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=sp["E0"])
    p = Problem(3, (n, n, n), "ico", level=1, cfl=0.5, bc="vvv", **kw)
    steps = 0 if case == "zero_steps" else 5
    if case == "f16":
        p.storage = lbrt.LB_RT_F16_DEV
    elif case == "frozen":
        cells = np.array([0, 7, n * n * n - 1], dtype=np.int32)
        p.frozen = (cells, np.full((3, 42), 0.1, dtype=np.float32))
    elif case == "moving":
        mf = W.moving_fluid(n)
        p.moving = dict(v=mf["v"], kt_a=mf["kt_a"], kt_0=mf["kt_0"], eta_t=mf["eta_t"])
    E2, F2, _ = _plain(p, steps)
    E1, F1, _ = _fused(p, steps, "pageable")
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(F1, F2)


def test_fields_read_in_place_from_page_locked_host_memory(cuda):
    """lb_rt_set_fluid with LB_RT_HOST_MAPPED: the kernels read kappa_a and
    eta from pinned host memory; the run is bit-identical to copied fields
    and new field values take effect at the next step."""
    import torch
    p = _sphere(24)
    ka = torch.from_numpy(p.coef["kappa_a"]).pin_memory()
    eta = torch.from_numpy(p.coef["eta"]).pin_memory()
    S = int(np.prod(p.shape))
    h1, h2 = make_handle(p), make_handle(p)
    try:
        out = []
        for h, mapped in ((h1, True), (h2, False)):
            E = torch.zeros(S, dtype=torch.float32).pin_memory()
            F = torch.zeros((3, S), dtype=torch.float32).pin_memory()
            for k in range(3):
                scale = 1.0 + 0.5 * k
                if mapped:
                    ka.copy_(torch.from_numpy(p.coef["kappa_a"] * scale))
                    lbrt.lb_rt_set_fluid(h, kappa_a=ka, eta=eta, mapped=True)
                else:
                    lbrt.lb_rt_set_fluid(h, kappa_a=p.coef["kappa_a"] * scale, eta=p.coef["eta"])
                lbrt.lb_rt_step_moments(h, 2, E, F)
            out.append((E.numpy().copy(), F.numpy().copy()))
        np.testing.assert_array_equal(out[0][0], out[1][0])
        np.testing.assert_array_equal(out[0][1], out[1][1])
        # an unknown pointer kind is refused
        import ctypes
        f, _, keep = lbrt._make_fluid(kappa_a=1.0)
        assert lbrt.load().lb_rt_set_fluid(h1, ctypes.byref(f), 7) == lbrt.LB_RT_EINVAL
    finally:
        lbrt.lb_rt_destroy(h1)
        lbrt.lb_rt_destroy(h2)


def test_full_size_bench_problem(cuda):
    """The bench's 128^3 x 42 radiating sphere (vacuum faces, kappa_a R = 10):
    the epilogue moments written to pinned host memory agree with the
    separate moments pass after the same steps."""
    p = _sphere(128)
    E2, F2, I2 = _plain(p, 3)
    E1, F1, I1 = _fused(p, 3, "pinned")
    np.testing.assert_array_equal(I1, I2)
    assert rel_l2(E1, E2) < 2e-6
    assert np.linalg.norm(F1 - F2) / np.linalg.norm(E2) < 2e-6
