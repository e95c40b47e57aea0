"""Host-side fits of the diffusion study (paper_2007_05718_gb300.diffusion_study)
against the oracle's independent fits, on data with a known answer."""
import math

import numpy as np

from oracle import diffusion as Df
from paper_2007_05718_gb300 import diffusion_study as S


def test_hill_and_gaussian_fit_match_the_oracle():
    n, sigma0, Dtrue = 96, 6.0, 0.61
    x = np.arange(n) + 0.5 - 0.5 * n
    for t in (5.0, 40.0):
        np.testing.assert_allclose(S.hill(n, sigma0, Dtrue, t),
                                   Df.gaussian_hill_periodic(x, x, (0.0, 0.0), (n, n), sigma0,
                                                             Dtrue, t), rtol=1e-12, atol=1e-300)
    steps, dt = (5, 10, 20, 50), 0.5
    snaps = [S.hill(n, sigma0, Dtrue, k * dt).astype(np.float32) for k in steps]
    D, err = S.fit_gaussian_D(snaps, steps, dt, sigma0, 0.3)
    assert abs(D / Dtrue - 1.0) < 1e-5 and err < 1e-6
    # a hill whose width follows another law: both fits land on the same D
    snaps2 = [S.hill(n, sigma0, Dtrue * (1.0 + 0.2 * math.exp(-k / 10.0)), k * dt) for k in steps]
    D1, e1 = S.fit_gaussian_D(snaps2, steps, dt, sigma0, 0.5)
    D2, e2 = Df.fit_gaussian_D(snaps2, [k * dt for k in steps], x, x, (0.0, 0.0), (n, n), sigma0)
    assert abs(D1 / D2 - 1.0) < 1e-6 and abs(e1 - e2) < 1e-9


def test_alpha_fit_matches_the_oracle():
    pts = S.sweep_points()
    k0 = np.array([p["kappa_0"] for p in pts])
    cfl = np.array([p["cfl"] for p in pts])
    lam = np.array([p["lam"] for p in pts])
    alpha = (-4.0 / 3.0, 0.48, 0.65)
    Dm = S.model_D(alpha, k0, lam, cfl)
    np.testing.assert_allclose(Dm, Df.model_D(alpha, k0, lam, cfl, 1.0, 2), rtol=1e-14)
    got, rms = S.fit_alphas(k0, lam, cfl, Dm)
    np.testing.assert_allclose(got, alpha, rtol=1e-7)
    Dc = Df.closed_form_D(k0, lam, cfl, 1.0, 2, 2.0 / math.pi)
    a_pkg, r_pkg = S.fit_alphas(k0, lam, cfl, Dc)
    a_orc, r_orc = Df.fit_alphas(k0, lam, cfl, 1.0, 2, Dc)
    np.testing.assert_allclose(a_pkg, a_orc, rtol=1e-6, atol=1e-8)
    assert abs(r_pkg - r_orc) < 1e-9


def test_variance_of_a_sampled_gaussian():
    n, sigma0 = 128, 7.0
    E = S.hill(n, sigma0, 0.0, 0.0)
    assert abs(S.variance(E, 0) - sigma0 ** 2) < 1e-9
    assert abs(S.variance(E, 1) - sigma0 ** 2) < 1e-9
