"""The oracle against the paper's analytic solutions: radiating sphere
(Sec. 4.2.2) and Gaussian diffusion (Sec. 4.2.3 with the diffusion
coefficient of App. A)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import analytic as A
from oracle import directions as D
from oracle import lb
from paper_2007_05718_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def test_sphere_profile_closed_forms():
    R = 0.25
    for kappa in (4.0, 40.0, 400.0):
        E, F = A.sphere_EF([0.0], R, kappa)
        assert abs(E[0] - (1 - math.exp(-kappa * R))) < 1e-13   # s = R at the centre
        assert abs(F[0]) < 1e-15
    # optically thick limit: f = 1 inside the cone mu > mu_c outside the sphere
    for r in (0.3, 0.5, 1.0):
        E, F = A.sphere_EF([r], R, 1e6)
        mu_c = math.sqrt(1 - (R / r) ** 2)
        assert abs(E[0] - 0.5 * (1 - mu_c)) < 1e-9
        assert abs(F[0] - 0.25 * (R / r) ** 2) < 1e-9
    # optically thin limit: E = kappa * (mean chord) / ... -> E ~ kappa * <s>;
    # at the centre <s> = R exactly
    E, _ = A.sphere_EF([0.0], R, 1e-6)
    assert abs(E[0] / (1e-6 * R) - 1) < 1e-5


def _run_sphere(nn, kR, steps):
    n, w = D.icosphere(1)
    sp = W.radiating_sphere(nn, kR)
    lat = lb.Lattice(3, (nn,) * 3, n, w, cfl=0.5, dx=1 / nn, bc=(lb.VACUUM,) * 3)
    co = lb.Static(kappa_a=sp["kappa_a"].astype(float), eta=sp["eta"].astype(float))
    I = lb.isotropic(sp["E0"].astype(float), lat)
    for _ in range(steps):
        prev, I = I, lb.step(I, lat, co)
    r = W.radius((nn,) * 3, (0.5, 0.5, 0.5), 1 / nn)
    Ea, _ = A.sphere_EF(r.ravel(), 0.25, kR / 0.25)
    return I.sum(0), prev.sum(0), Ea.reshape(r.shape), r


@pytest.mark.slow
@pytest.mark.parametrize("kR,tol", [(1.0, 0.05), (10.0, 0.10)])
def test_radiating_sphere_steady_state(kR, tol):
    """32^3, 42 directions, vacuum boundaries, cfl 0.5: after ~2.3 light
    crossings the state is steady and E(r) follows the analytic profile
    (discretisation-limited: R is 8 cells)."""
    E, Eprev, Ea, r = _run_sphere(32, kR, 150)
    assert np.abs(E - Eprev).max() < 1e-8
    m = r < 1.5 * 0.25
    assert np.linalg.norm((E - Ea)[m]) / np.linalg.norm(Ea[m]) < tol
    core = r < 0.5 * 0.25
    assert np.abs(E - Ea)[core].max() < 0.02


def _run_gauss_2d(N, kdx, steps, scheme="implicit", L=128):
    n, w = D.ring2d(N, 0.0)
    lat = lb.Lattice(2, (1, L, L), n, w, cfl=0.5, dx=1 / L)
    k0 = kdx * L
    E0 = W.gaussian_E0((1, L, L), 8.0).astype(np.float64)
    I = lb.run(lb.isotropic(E0, lat), lat, lb.Static(kappa_0=k0), steps, collision=scheme)
    Dc = A.diffusion_coefficient(k0, lat.dt, lat.dx, 2, np.sum(w * np.abs(n[:, 0])), scheme)
    r2 = W.radius((1, L, L), (0.5, 0.5, 0.5 / L), 1 / L) ** 2
    Ea = A.gaussian_E(r2, steps * lat.dt, 8 / L, Dc, dims=2)
    E = I.sum(0)
    return np.linalg.norm(E - Ea) / np.linalg.norm(Ea), E, Ea


@pytest.mark.slow
def test_gaussian_diffusion_2d_implicit():
    crit = json.load(open(GOLDEN))["diffusion_criterion"]["rel_l2"]
    err, E, Ea = _run_gauss_2d(16, 4.0, 400)
    assert err < crit
    # without the interpolation term the prediction is far off
    L = 128
    n, w = D.ring2d(16, 0.0)
    r2 = W.radius((1, L, L), (0.5, 0.5, 0.5 / L), 1 / L) ** 2
    Ebad = A.gaussian_E(r2, 400 * 0.5 / L, 8 / L, 1 / (2 * 4.0 * L), dims=2)
    assert np.linalg.norm(E - Ebad) / np.linalg.norm(Ebad) > 5 * crit


@pytest.mark.slow
def test_gaussian_diffusion_2d_explicit():
    crit = json.load(open(GOLDEN))["diffusion_criterion"]["rel_l2"]
    err, _, _ = _run_gauss_2d(16, 1.5, 400, scheme="explicit")
    assert err < crit


@pytest.mark.slow
def test_gaussian_diffusion_3d_implicit():
    """48^3 periodic, 42 directions, sigma0 = 4 cells; the d = 3 amplitude
    factor (sigma0^2 / (sigma0^2 + sigma_D^2))^{3/2} is required."""
    crit = json.load(open(GOLDEN))["diffusion_criterion"]["rel_l2"]
    L = 48
    n, w = D.icosphere(1)
    lat = lb.Lattice(3, (L,) * 3, n, w, cfl=0.5, dx=1 / L)
    k0 = 4.0 * L
    E0 = W.gaussian_E0((L,) * 3, 4.0).astype(np.float64)
    steps = 60
    I = lb.run(lb.isotropic(E0, lat), lat, lb.Static(kappa_0=k0), steps)
    Dc = A.diffusion_coefficient(k0, lat.dt, lat.dx, 3, np.sum(w * np.abs(n[:, 0])))
    r2 = W.radius((L,) * 3, (0.5, 0.5, 0.5), 1 / L) ** 2
    t = steps * lat.dt
    Ea = A.gaussian_E(r2, t, 4 / L, Dc, dims=3)
    E = I.sum(0)
    assert np.linalg.norm(E - Ea) / np.linalg.norm(Ea) < crit
    E2 = A.gaussian_E(r2, t, 4 / L, Dc, dims=2)   # the 2D amplitude is wrong in 3D
    assert np.linalg.norm(E - E2) / np.linalg.norm(E2) > 2 * crit


def test_free_streaming_wave_exact_moments():
    """Radiation wave (Sec. 4.1.2) in vacuum: energy is conserved exactly and
    the energy-weighted second moment grows exactly as the binomial walk of
    each direction predicts; the shell-averaged profile follows the
    direction-set independent closed form within the interpolation blur."""
    from oracle import analytic as A
    from oracle import directions as D
    from oracle import lb
    from paper_2007_05718_gb300 import workloads as W
    n, R, steps = 48, 5.0, 16   # the walk reaches at most R + steps < n / 2: no outflow
    E0, c = W.wave_ball(n, R)
    nv, w = D.icosphere(1)
    lat = lb.Lattice(3, (n, n, n), nv, w, cfl=0.2, dx=1.0, bc=(lb.VACUUM,) * 3)
    I = lb.isotropic(E0.astype(float), lat)
    idx = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    m = float(E0.sum())
    S2 = float((E0 * r2).sum())
    I = lb.run(I, lat, lb.Static(), steps)
    E = I.sum(axis=0)
    assert abs(E.sum() - m) < 1e-12 * m
    M2 = float((E * r2).sum())
    assert abs(M2 - A.wave_second_moment(lat, m, S2, steps)) < 1e-10 * M2
    # first moment stays at the centre (symmetric direction set)
    assert abs(float((E * (X - c[0])).sum())) < 1e-9 * m
    # the closed form's peak tends to the inverse-square law
    assert abs(A.wave_peak(1000.0, 5.0) * 4 * 1000.0 ** 2 / 25.0 - 1.0) < 1e-4
    # shell average of the closed form conserves the ball's energy
    rr = np.linspace(0.01, 40, 20001)
    tot = np.trapezoid(A.wave_shell_E(rr, 12.0, 5.0) * 4 * np.pi * rr ** 2, rr)
    assert abs(tot / (4.0 / 3.0 * np.pi * 125.0) - 1.0) < 1e-3
