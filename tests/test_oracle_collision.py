"""Pins for the oracle's collisions (Eqs. collision-step, rte_implicit, the
Lambda iteration of Sec. 3.3, and the mixed-frame equation of App. B)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import analytic as A
from oracle import directions as D
from oracle import lb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def _sites(N, S, seed):
    g = np.random.default_rng(seed)
    Is = g.random((N, S)) / N
    co = lb.Static(kappa_a=10 ** g.uniform(-2, 4, S), kappa_0=10 ** g.uniform(-2, 4, S),
                   lam=g.uniform(-1, 1, S), eta=10 ** g.uniform(-2, 3, S))
    return Is, co


@pytest.mark.parametrize("dirs", ["ico1", "ring16", "gl"])
def test_implicit_matches_dense_solve(dirs):
    if dirs == "ico1":
        n, w = D.icosphere(1); d = 3
    elif dirs == "ring16":
        n, w = D.ring2d(16, 0.3); d = 2
    else:
        n, w = D.gauss_legendre_product(3, 6); d = 3
    S = 12
    Is, co = _sites(len(w), S, 7)
    lat = lb.Lattice(d, (1, 1, S), n, w, cfl=0.5, dx=0.01)
    got = lb.collide_implicit(Is, lat, co)
    for s in range(S):
        ref = A.dense_static_solve(Is[:, s], n[:, :d], w, lat.dt, co.kappa_a[s],
                                   co.kappa_0[s], co.lam[s], co.eta[s])
        assert np.allclose(got[:, s], ref, rtol=1e-11, atol=1e-14)


def test_implicit_isotropic_closed_form():
    """For an isotropic table the exact step has E = (E* + dt eta)/(1 + dt kappa_a)
    and F = F* / (1 + dt (kappa_a + kappa_0) - dt kappa_0 lambda / d)."""
    n, w = D.icosphere(2)
    S = 50
    Is, co = _sites(len(w), S, 8)
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=0.5, dx=0.01)
    E, F = lb.implicit_moments(Is, lat, co)
    Es, Fs, _ = lb.moments(Is, lat)
    dt = lat.dt
    assert np.allclose(E, (Es + dt * co.eta) / (1 + dt * co.kappa_a), rtol=1e-12)
    den = 1 + dt * (co.kappa_a + co.kappa_0) - dt * co.kappa_0 * co.lam / 3
    assert np.allclose(F, Fs / den, rtol=1e-11, atol=1e-16)
    # and the populations really have those moments
    I = lb.collide_implicit(Is, lat, co)
    E2, F2, _ = lb.moments(I, lat)
    assert np.allclose(E2, E, rtol=1e-12) and np.allclose(F2, F, rtol=1e-10, atol=1e-16)


def test_lambda_iteration_converges_to_exact():
    n, w = D.icosphere(1)
    S = 20
    Is, co = _sites(len(w), S, 9)
    co.kappa_0 = np.minimum(co.kappa_0, 50.0)   # keep the contraction well below 1
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=0.5, dx=0.01)
    I_it, it = lb.collide_lambda(Is, lat, co, tol=1e-15)
    assert it > 3
    assert np.allclose(I_it, lb.collide_implicit(Is, lat, co), rtol=1e-12, atol=1e-16)


def test_lambda_iteration_shadow_cycles():
    f = json.load(open(GOLDEN))["lambda_iteration_shadow"]
    n, w = D.icosphere(1)
    S = 30
    g = np.random.default_rng(10)
    Is = g.random((len(w), S))
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=f["cfl"], dx=1.0 / 150)
    co = lb.Static(kappa_a=f["kappa_a"])
    _, it = lb.collide_lambda(Is, lat, co, tol=f["tol"])
    assert it <= f["max_cycles"]


def test_explicit_moments():
    """Eq. (collision-step) moves the moments as E = E* + dt (eta - kappa_a E*)
    and F = F* (1 - dt kappa_0 (1 - lambda/d) - dt kappa_a) for an isotropic table."""
    n, w = D.icosphere(1)
    S = 10
    Is, co = _sites(len(w), S, 11)
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=0.5, dx=1e-5)
    I = lb.collide_explicit(Is, lat, co)
    E, F, _ = lb.moments(I, lat)
    Es, Fs, _ = lb.moments(Is, lat)
    dt = lat.dt
    assert np.allclose(E, Es + dt * (co.eta - co.kappa_a * Es), rtol=1e-12)
    assert np.allclose(F, Fs * (1 - dt * co.kappa_0 * (1 - co.lam / 3) - dt * co.kappa_a),
                       rtol=1e-10, atol=1e-15)


def _moving_sites(N, S, seed, vmax=0.6):
    g = np.random.default_rng(seed)
    Is = g.random((N, S)) / N
    v = g.normal(size=(3, S))
    v *= (vmax * g.random(S) / np.linalg.norm(v, axis=0))[None]
    mo = lb.Moving(v=v, kt_a=10 ** g.uniform(-1, 3, S), kt_0=10 ** g.uniform(-1, 2, S),
                   eta_t=10 ** g.uniform(-1, 3, S))
    return Is, mo


def test_moving_matches_dense_solve():
    n, w = D.icosphere(1)
    S = 10
    Is, mo = _moving_sites(len(w), S, 12)
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=0.5, dx=1 / 64)
    got = lb.collide_moving(Is, lat, mo)
    for s in range(S):
        ref = A.dense_moving_solve(Is[:, s], n, w, lat.dt, mo.v[:, s], mo.kt_a[s],
                                   mo.kt_0[s], mo.eta_t[s])
        assert np.allclose(got[:, s], ref, rtol=1e-11, atol=1e-15)


def test_moving_lambda_iteration_converges_to_exact():
    n, w = D.icosphere(1)
    Is, mo = _moving_sites(len(w), 10, 13)
    mo.kt_0 = np.minimum(mo.kt_0, 20.0)
    lat = lb.Lattice(3, (1, 1, 10), n, w, cfl=0.5, dx=1 / 64)
    I_it, it = lb.collide_moving_lambda(Is, lat, mo, tol=1e-15)
    assert it > 2
    assert np.allclose(I_it, lb.collide_moving(Is, lat, mo), rtol=1e-12, atol=1e-16)


def test_moving_reduces_to_static_at_rest():
    n, w = D.icosphere(1)
    S = 10
    Is, mo = _moving_sites(len(w), S, 14)
    mo.v = np.zeros((3, S))
    lat = lb.Lattice(3, (1, 1, S), n, w, cfl=0.5, dx=1 / 64)
    co = lb.Static(kappa_a=mo.kt_a, kappa_0=mo.kt_0, lam=0.0, eta=mo.eta_t)
    assert np.allclose(lb.collide_moving(Is, lat, mo), lb.collide_implicit(Is, lat, co),
                       rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("vmag", [0.1, 0.3, 0.6])
def test_lab_frame_emission_integrates_to_W(vmag):
    """sum_i w_i (W beta_i)^-3 -> (1/2) int dmu / (W^3 (1 - v mu)^3) = W: the
    lab-frame emission of an isotropic fluid-frame emitter is W eta_t."""
    n, w = D.icosphere(2)
    v = vmag * np.array([0.36, 0.48, 0.8])
    W = 1 / math.sqrt(1 - v @ v)
    beta = 1 - n @ v
    q = np.sum(w / (W * beta) ** 3)
    tol = {0.1: 1e-6, 0.3: 1e-4, 0.6: 2e-2}[vmag]
    assert abs(q / W - 1) < tol


def test_pure_scattering_conserves_energy():
    n, w = D.icosphere(1)
    shape = (6, 6, 6)
    lat = lb.Lattice(3, shape, n, w, cfl=0.5, dx=1 / 6)
    I = np.random.default_rng(15).random((len(w),) + shape)
    co = lb.Static(kappa_0=300.0, lam=0.4)
    e0 = I.sum()
    for _ in range(5):
        I = lb.step(I, lat, co)
    assert abs(I.sum() / e0 - 1) < 1e-13


def test_energy_budget_identity():
    """sum E^{n+1} - sum E^n = source - outflow + injection, with source =
    dt sum (eta - kappa_a E^{n+1}) for the isotropic implicit step."""
    n, w = D.icosphere(1)
    shape = (6, 7, 8)
    lat = lb.Lattice(3, shape, n, w, cfl=0.5, dx=1 / 8, bc=(lb.VACUUM,) * 3)
    g = np.random.default_rng(16)
    I = g.random((len(w),) + shape)
    ka = g.random(shape) * 20
    eta = g.random(shape) * 5
    co = lb.Static(kappa_a=ka, kappa_0=3.0, lam=0.2, eta=eta)
    fz = lb.Frozen(cells=np.array([[1, 2, 3], [4, 4, 4]]), values=g.random((2, len(w))))
    e0 = I.sum()
    b = {}
    I1 = lb.step(I, lat, co, frozen=fz, budget=b)
    assert abs(I1.sum() - e0 - (b["source"] - b["outflow"] + b["injection"])) < 1e-12 * e0
    # the source term equals dt sum(eta - kappa_a E_coll)
    Is = lb.stream(I, lat)
    Ec = lb.collide_implicit(Is, lat, co).sum(0)
    assert abs(b["source"] - lat.dt * np.sum(eta - ka * Ec)) < 1e-11 * e0
