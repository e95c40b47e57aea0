"""16-bit population storage (FP16 and BF16, the populations kept as the
relative deviation from the static equilibrium w_i E, float32 arithmetic)
against the FP64 oracle on the same seeded inputs: relative L2 of E and F
within 2e-3."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import Problem, gpu_run, make_handle, oracle_run, pad_F, rel_l2

pytestmark = pytest.mark.gpu

TOL_16 = 2e-3
STORAGES = [pytest.param(lbrt.LB_RT_F16_DEV, id="fp16"), pytest.param(lbrt.LB_RT_BF16_DEV, id="bf16")]


def _check(p, steps, f_scale="F", tol_f=TOL_16):
    I, E, F, P, b = gpu_run(p, steps)
    Io, Eo, Fo, Po, bo, lat = oracle_run(p, steps)
    eE = rel_l2(E, Eo)
    Fo3 = pad_F(Fo, p.dims)
    eF = rel_l2(F, Fo3) if f_scale == "F" else np.linalg.norm(F - Fo3) / np.linalg.norm(Eo)
    assert eE <= TOL_16, eE
    assert eF <= tol_f, eF
    return E, F, b, Eo, bo, eE, eF


def test_sphere_reduced(cuda):
    """Radiating sphere (kappa_a R = 10), 32^3, 42 directions, vacuum faces,
    150 steps, FP16 storage.  Outside the sphere the field streams freely and
    is strongly beamed, so the deviations from isotropy are of order one.
    BF16 (8 significant bits) is not validated in this regime (its flux error
    here is about 5e-3; the header says to use FP16 for it) and is tested on
    the near-isotropic problems below, at the same 2e-3 bar."""
    sp = W.radiating_sphere(32, 10.0)
    p = Problem(3, (32, 32, 32), "ico", level=1, bc="vvv", storage=lbrt.LB_RT_F16_DEV,
                coef=dict(kappa_a=sp["kappa_a"], eta=sp["eta"]),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=sp["E0"], budget=True)
    _check(p, 150)


@pytest.mark.parametrize("storage", STORAGES)
def test_thick_sphere_with_scattering_reduced(cuda, storage):
    """A scattering-dominated sphere: kappa_a R = 10 inside with kappa_0 = 400
    /L everywhere, so the field stays near isotropy and both 16-bit formats
    are in their validated regime; 32^3, 42 directions, vacuum faces, 150
    steps, E and F at 2e-3."""
    sp = W.radiating_sphere(32, 10.0)
    p = Problem(3, (32, 32, 32), "ico", level=1, bc="vvv", storage=storage,
                coef=dict(kappa_a=sp["kappa_a"], kappa_0=400.0, eta=sp["eta"]),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=sp["E0"], budget=True)
    _check(p, 150)


@pytest.mark.parametrize("storage", STORAGES)
def test_diffusion_reduced(cuda, storage):
    """Pure scattering kappa_0 dx = 3.9, 162 directions, 24^3 periodic Gaussian, 40 steps."""
    n = 24
    E0 = W.gaussian_E0((n, n, n), 3.0)
    p = Problem(3, (n, n, n), "ico", level=2, storage=storage, coef=dict(kappa_0=3.90625 * n),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=E0, budget=True)
    E, F, b, Eo, bo, eE, eF = _check(p, 40)
    # the float32 E field is conserved by the collision; the stream sees the
    # 16-bit rounding of the deviations only
    assert abs(b["total"] / b["initial"] - 1) < 1e-4


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("bc", ["ppp", "vpv", "pvv"])
def test_random_fields_ragged_grid(cuda, storage, bc):
    """Ragged grid, random per-site opacities, mixed boundaries; the initial
    state is a P1 field (smooth E, F) so that the deviations are those of a
    radiation field rather than of white noise."""
    shape = (5, 11, 37)
    coef = dict(kappa_a=W.random_fields(shape, 1, 0.0, 30.0), kappa_0=W.random_fields(shape, 2, 0.0, 80.0),
                lam=W.random_fields(shape, 3, -1.0, 1.0), eta=W.random_fields(shape, 4, 0.0, 5.0))
    E0 = 1.0 + W.smooth_field(shape, 5).astype(np.float32)
    F0 = 0.2 * np.stack([W.smooth_field(shape, 6 + k) for k in range(3)]).astype(np.float32)
    state = np.concatenate([E0[None], F0]).astype(np.float32)
    p = Problem(3, shape, "ico", level=1, bc=bc, storage=storage, coef=coef,
                state_kind=lbrt.LB_RT_STATE_P1, state=state, budget=True)
    _check(p, 6, f_scale="E")


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("mode,iters", [("explicit", 1), ("lambda", 5)])
def test_collision_modes(cuda, storage, mode, iters):
    shape = (6, 9, 33)
    coef = dict(kappa_a=W.random_fields(shape, 6, 0.0, 10.0), kappa_0=W.random_fields(shape, 7, 0.0, 40.0),
                lam=W.random_fields(shape, 8, -1.0, 1.0), eta=W.random_fields(shape, 9, 0.0, 2.0))
    E0 = 1.0 + W.smooth_field(shape, 10).astype(np.float32)
    p = Problem(3, shape, "ico", level=1, bc="pvp", storage=storage, collision=mode,
                lambda_iters=iters, coef=coef, state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=E0)
    _check(p, 5, f_scale="E")


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("nx", [36, 37, 8])
@pytest.mark.parametrize("bc", ["ppp", "vvv"])
def test_kernel_paths_by_row_width(cuda, storage, nx, bc):
    """Row widths that leave a partial pair, a partial tile or a single short
    tile; periodic rows exercise the ghost mirrors."""
    shape = (7, 5, nx)
    E0 = 1.0 + W.smooth_field(shape, 15).astype(np.float32)
    p = Problem(3, shape, "ico", level=1, bc=bc, storage=storage,
                coef=dict(kappa_a=2.0, kappa_0=30.0, eta=1.5),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=E0)
    _check(p, 7, f_scale="E")


@pytest.mark.parametrize("storage", STORAGES)
def test_populations_round_trip(cuda, storage):
    """set_state(populations) then get_populations returns each value within
    the 16-bit rounding of its deviation from w_i E."""
    shape = (4, 5, 9)
    N = 42
    Ipop = W.random_populations(N, shape, 31)
    p = Problem(3, shape, "ico", level=1, storage=storage, state=Ipop)
    h = make_handle(p)
    try:
        out = np.zeros((N, int(np.prod(shape))), dtype=np.float32)
        lbrt.lb_rt_get_populations(h, out)
    finally:
        lbrt.lb_rt_destroy(h)
    ref = Ipop.reshape(N, -1).astype(np.float64)
    eps = 2.0 ** -11 if storage == lbrt.LB_RT_F16_DEV else 2.0 ** -8
    E = ref.sum(axis=0)
    # |I - I_ref| <= w E |q| eps  with w E |q| = |I - w E|
    w = 1.0 / N
    bound = np.abs(ref - w * E) * eps + 1e-6 * w * E
    assert np.all(np.abs(out - ref) <= bound)


@pytest.mark.parametrize("storage", STORAGES)
def test_checkpoint_resume_bit_exact(cuda, storage):
    shape = (6, 8, 40)
    E0 = 1.0 + W.smooth_field(shape, 21).astype(np.float32)
    p = Problem(3, shape, "ico", level=1, bc="pvp", storage=storage,
                coef=dict(kappa_a=1.0, kappa_0=20.0, eta=0.5),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=E0, budget=True)
    h = make_handle(p)
    h2 = make_handle(p)
    try:
        lbrt.lb_rt_step(h, 3)
        buf = lbrt.lb_rt_save_state(h)
        lbrt.lb_rt_step(h, 4)
        lbrt.lb_rt_restore_state(h2, buf)
        lbrt.lb_rt_step(h2, 4)
        S = int(np.prod(shape))
        a = np.zeros((42, S), dtype=np.float32)
        b = np.zeros((42, S), dtype=np.float32)
        lbrt.lb_rt_get_populations(h, a)
        lbrt.lb_rt_get_populations(h2, b)
        assert np.array_equal(a, b)
    finally:
        lbrt.lb_rt_destroy(h)
        lbrt.lb_rt_destroy(h2)


@pytest.mark.parametrize("storage", STORAGES)
def test_frozen_beam_injection(cuda, storage):
    """Sec. 4.1.1 beam on a ring-8 40 x 24 grid, direction 0 held at 1 on the
    left column for |y - 12| < 6, vacuum in x, cfl 0.2 (frozen cells re-encode
    the whole site)."""
    nx, ny = 40, 24
    N = 8
    cells = np.array([y * nx for y in range(ny) if abs(y - 12) < 6], dtype=np.int64)
    vals = np.zeros((len(cells), N), dtype=np.float32)
    vals[:, 0] = 1.0
    state = np.zeros((N, 1, ny, nx), dtype=np.float32)
    p = Problem(2, (1, ny, nx), "ring", ndir=N, cfl=0.2, bc="vpp", storage=storage,
                state=state, frozen=(cells, vals), budget=True)
    _check(p, 60)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("level", [1, 2])
def test_moving_shear_reduced(cuda, storage, level):
    """Moving background (App. B) with 16-bit storage: the shear-flow
    generator on a 20^3 periodic box, smooth initial E and F (P1 state)."""
    n = 20
    mf = W.moving_fluid(n)
    shape = (n, n, n)
    E0 = 1.0 + W.smooth_field(shape, 41).astype(np.float32)
    F0 = 0.2 * np.stack([W.smooth_field(shape, 42 + k) for k in range(3)]).astype(np.float32)
    p = Problem(3, shape, "ico", level=level, storage=storage,
                moving=dict(v=mf["v"], kt_a=mf["kt_a"], kt_0=mf["kt_0"], eta_t=mf["eta_t"]),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]), budget=True)
    _check(p, 12)


@pytest.mark.parametrize("storage", STORAGES)
def test_moving_with_vacuum_faces(cuda, storage):
    shape = (6, 9, 35)
    v = 0.4 * np.stack([W.smooth_field(shape, 51 + k) for k in range(3)]).astype(np.float32) / 3.0
    p = Problem(3, shape, "ico", level=1, bc="vpv", storage=storage,
                moving=dict(v=v, kt_a=W.random_fields(shape, 55, 0.0, 10.0),
                            kt_0=W.random_fields(shape, 56, 0.0, 20.0), eta_t=1.0),
                state_kind=lbrt.LB_RT_STATE_ISOTROPIC,
                state=(1.0 + 0.5 * W.smooth_field(shape, 57)).astype(np.float32))
    _check(p, 8, f_scale="E")
