"""Parity at the full benchmark sizes, in the launch configuration the bench
times: one step from a seeded P1 state, checked on sampled sites that the
oracle computes one by one (stream_sites + the exact collision)."""
import numpy as np
import pytest

from oracle import lb as OL
from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import Problem, make_handle, rel_l2

pytestmark = pytest.mark.gpu


def _sampled(p, E0, F0, co_fields, nsample, seed, collide=None):
    """(GPU, oracle) populations after one step at sampled sites; the oracle
    streams the P1 state one site at a time (stream_sites) and applies the
    exact collision (static by default, or `collide(Is, lat, sites)`)."""
    import torch
    lat = p.lattice()
    h = make_handle(p)
    try:
        lbrt.lb_rt_step(h, 1)
        lbrt.lb_rt_sync(h)
        N = lat.N
        out = torch.empty((N,) + p.shape, device="cuda")
        lbrt.lb_rt_get_populations(h, out)
        torch.cuda.synchronize()
        g = np.random.default_rng(seed)
        nz, ny, nx = p.shape
        # random interior sites plus every corner and face-centre site
        z = np.concatenate([g.integers(0, nz, nsample), [0, nz - 1, 0, nz - 1, nz // 2]])
        y = np.concatenate([g.integers(0, ny, nsample), [0, ny - 1, ny - 1, 0, 0]])
        x = np.concatenate([g.integers(0, nx, nsample), [0, nx - 1, nx - 1, 0, nx // 2]])
        idx = torch.from_numpy((z * ny + y) * nx + x).cuda()
        got = out.reshape(N, -1)[:, idx].cpu().numpy().astype(np.float64)
        del out
    finally:
        lbrt.lb_rt_destroy(h)
    E0d, F0d = E0.astype(np.float64), F0.astype(np.float64)
    n, w = lat.n, lat.w

    def value_at(i, zz, yy, xx):
        return w[i] * (E0d[zz, yy, xx] + 3.0 * (n[i, 0] * F0d[0, zz, yy, xx] + n[i, 1] * F0d[1, zz, yy, xx]
                                                + n[i, 2] * F0d[2, zz, yy, xx]))

    Is = OL.stream_sites(value_at, (z, y, x), lat)
    if collide is not None:
        return got, collide(Is, lat, (z, y, x))
    co = OL.Static(**{k: (v[z, y, x].astype(np.float64) if isinstance(v, np.ndarray) else v)
                      for k, v in co_fields.items()})
    ref = OL.collide_implicit(Is, lat, co)
    return got, ref


def test_c2_full_128_cubed_42(cuda):
    n = 128
    sp = W.radiating_sphere(n, 10.0)
    E0, F0 = W.random_moments((n, n, n), 41)
    p = Problem(3, (n, n, n), "ico", level=1, bc="vvv",
                coef=dict(kappa_a=sp["kappa_a"], eta=sp["eta"]),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]))
    got, ref = _sampled(p, E0, F0, dict(kappa_a=sp["kappa_a"], eta=sp["eta"]), 4000, 42)
    assert rel_l2(got, ref) < 1e-6
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_c3_full_256_cubed_162(cuda):
    n = 256
    E0, F0 = W.random_moments((n, n, n), 43)
    k0 = 3.90625 * n
    p = Problem(3, (n, n, n), "ico", level=2, coef=dict(kappa_0=k0),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]))
    got, ref = _sampled(p, E0, F0, dict(kappa_0=k0), 3000, 44)
    assert rel_l2(got, ref) < 1e-6
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("storage", [pytest.param(lbrt.LB_RT_F16_DEV, id="fp16"),
                                     pytest.param(lbrt.LB_RT_BF16_DEV, id="bf16")])
def test_c3_full_256_cubed_162_16bit(cuda, storage):
    """The diffusion configuration with 16-bit storage at full size: the P1
    state is encoded in 16 bits on the device, stepped once and decoded; the
    oracle streams the exact P1 state.  The 16-bit rounding of the deviations
    from w_i E (which are small here, |F| <= 0.2 E / 3) stays within 2e-3."""
    n = 256
    E0, F0 = W.random_moments((n, n, n), 45)
    k0 = 3.90625 * n
    p = Problem(3, (n, n, n), "ico", level=2, storage=storage, coef=dict(kappa_0=k0),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]))
    got, ref = _sampled(p, E0, F0, dict(kappa_0=k0), 3000, 46)
    assert rel_l2(got, ref) < 2e-3
    assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max()


@pytest.mark.parametrize("storage,tol", [pytest.param(lbrt.LB_RT_F32, 1e-5, id="fp32"),
                                         pytest.param(lbrt.LB_RT_F16_DEV, 2e-3, id="fp16")])
def test_c5_full_256_cubed_162_moving(cuda, storage, tol):
    """The moving-fluid configuration at full size (the seeded relativistic
    shear flow, |v| <= 0.6, density-scaled opacities): one mixed-frame step
    (App. B) from a P1 state, checked on sampled sites against the oracle's
    exact moving collision."""
    n = 256
    mf = W.moving_fluid(n)
    E0, F0 = W.random_moments((n, n, n), 47)
    p = Problem(3, (n, n, n), "ico", level=2, storage=storage,
                moving=dict(v=mf["v"], kt_a=mf["kt_a"], kt_0=mf["kt_0"], eta_t=mf["eta_t"]),
                state_kind=lbrt.LB_RT_STATE_P1, state=np.concatenate([E0[None], F0]))

    def collide(Is, lat, sites):
        z, y, x = sites
        mo = OL.Moving(v=mf["v"][:, z, y, x].astype(np.float64),
                       kt_a=mf["kt_a"][z, y, x].astype(np.float64),
                       kt_0=mf["kt_0"][z, y, x].astype(np.float64),
                       eta_t=mf["eta_t"][z, y, x].astype(np.float64))
        return OL.collide_moving(Is, lat, mo)

    got, ref = _sampled(p, E0, F0, None, 3000, 48, collide=collide)
    assert rel_l2(got, ref) < tol
    assert np.abs(got - ref).max() <= 10 * tol * np.abs(ref).max()
