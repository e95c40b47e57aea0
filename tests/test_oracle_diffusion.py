"""Pins of oracle/diffusion.py (App. A): the spatial-moment recursion against
brute-force lattice runs and the free-streaming closed form, the closed-form
D against the recursion, and the two fits against data with a known answer."""
import math

import numpy as np
import pytest

from oracle import diffusion as Df
from oracle import directions as D
from oracle import lb


def _pulse_variances(n, w, cfl, k0, lam, steps, L=48, collision="implicit"):
    """Brute force: a unit isotropic pulse on an L x L periodic oracle
    lattice (no mass reaches the faces within `steps`), x and y variances."""
    lat = lb.Lattice(2, (1, L, L), n, w, cfl=cfl, dx=1.0)
    E0 = np.zeros((1, L, L))
    E0[0, L // 2, L // 2] = 1.0
    I = lb.isotropic(E0, lat)
    co = lb.Static(kappa_0=k0, lam=lam)
    x = np.arange(L) - L // 2
    Vx, Vy = [0.0], [0.0]
    for _ in range(steps):
        I = lb.step(I, lat, co, collision=collision)
        E = I.sum(0)[0]
        m0 = E.sum()
        mx, my = (E.sum(0) * x).sum() / m0, (E.sum(1) * x).sum() / m0
        Vx.append((E.sum(0) * x * x).sum() / m0 - mx * mx)
        Vy.append((E.sum(1) * x * x).sum() / m0 - my * my)
    return np.array(Vx), np.array(Vy)


@pytest.mark.parametrize("phi0,cfl,k0,lam", [(0.0, 0.5, 1.0, 0.5), (0.3, 0.8, 2.0, 0.25),
                                             (0.1, 1.0, 0.5, 0.0)])
def test_recursion_equals_brute_force_lattice(phi0, cfl, k0, lam):
    n, w = D.ring2d(16, phi0)
    steps = 20
    Vx, Vy = _pulse_variances(n, w, cfl, k0, lam, steps)
    Rx = Df.moment_recursion(n, w, 2, cfl, 1.0, k0, lam, steps, axis=0)
    Ry = Df.moment_recursion(n, w, 2, cfl, 1.0, k0, lam, steps, axis=1)
    np.testing.assert_allclose(Rx, Vx, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Ry, Vy, rtol=1e-11, atol=1e-12)


def test_recursion_free_streaming_closed_form():
    """kappa_0 = 0: each direction walks a Bernoulli shift of probability a
    per step, V(t) = t <a(1-a)>_w + t^2 cfl^2 <(n^x)^2>_w - t^2 (<a s>_w)^2."""
    n, w = D.ring2d(12, 0.2)
    cfl, steps = 0.7, 30
    V = Df.moment_recursion(n, w, 2, cfl, 1.0, 0.0, 0.0, steps)
    a = cfl * np.abs(n[:, 0])
    s = np.where(n[:, 0] >= 0, 1.0, -1.0)
    t = np.arange(steps + 1)
    want = t * np.sum(w * a * (1 - a)) + t * t * (np.sum(w * a * a) - np.sum(w * a * s) ** 2)
    np.testing.assert_allclose(V, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dirs", ["ring16", "ring120", "ring16rot", "ico42", "gl"])
def test_closed_form_D_equals_recursion(dirs):
    if dirs == "ring16":
        (n, w), d = D.ring2d(16, 0.0), 2
    elif dirs == "ring120":
        (n, w), d = D.ring2d(120, 0.0), 2
    elif dirs == "ring16rot":
        (n, w), d = D.ring2d(16, 0.3), 2
    elif dirs == "ico42":
        (n, w), d = D.icosphere(1), 3
    else:
        (n, w), d = D.gauss_legendre_product(4, 8), 3
    mabs = float(np.sum(w * np.abs(n[:, 0])))
    for k0, cfl, lam in ((1.0, 1.0, 0.0), (1.0, 0.5, 0.5), (0.5, 0.25, 0.75), (5.0, 1.0, 0.25),
                         (100.0, 0.1, 0.5)):
        Dr = Df.recursion_D(n, w, d, cfl, 1.0, k0, lam)
        Dc = Df.closed_form_D(k0, lam, cfl, 1.0, d, mabs)
        assert abs(Dr / Dc - 1.0) < 1e-10, (dirs, k0, cfl, lam, Dr, Dc)


@pytest.mark.parametrize("collision", ["implicit", "explicit"])
def test_explicit_and_implicit_against_brute_force_and_closed_form(collision):
    n, w = D.ring2d(16, 0.0)
    cfl, k0, lam = 0.5, 1.5, 0.5
    Vx, _ = _pulse_variances(n, w, cfl, k0, lam, 20, collision=collision)
    Rx = Df.moment_recursion(n, w, 2, cfl, 1.0, k0, lam, 20, collision=collision)
    np.testing.assert_allclose(Rx, Vx, rtol=1e-11, atol=1e-12)
    Dr = Df.recursion_D(n, w, 2, cfl, 1.0, k0, lam, collision=collision)
    Dc = Df.closed_form_D(k0, lam, cfl, 1.0, 2, float(np.sum(w * np.abs(n[:, 0]))), collision)
    assert abs(Dr / Dc - 1.0) < 1e-10


def test_closed_form_D_is_not_the_chapman_enskog_leading_term():
    """Eq. (numerical-diff-coeff) alone (no interpolation term, explicit
    relaxation) is off by tens of percent at kappa_0 dx = 1: the recursion
    tells the two apart."""
    n, w = D.ring2d(120, 0.0)
    Dr = Df.recursion_D(n, w, 2, 1.0, 1.0, 1.0, 0.0)
    ce = 1.0 / (2 * 1.0) * (1.0 - 0.5 * 1.0)
    assert Dr / ce > 2.0


def test_fit_gaussian_D_recovers_known_D():
    L, sigma0, Dtrue = 64, 5.0, 0.37
    x = np.arange(L) + 0.5 - 0.5 * L
    X, Y = np.meshgrid(x, x, indexing="xy")
    times = [5, 10, 20, 50]
    # the hill written out as the double sum over images
    snaps = []
    for t in times:
        s2 = sigma0 ** 2 + 2 * Dtrue * t
        G = sum(np.exp(-((X + jx * L) ** 2 + (Y + jy * L) ** 2) / (2 * s2))
                for jx in range(-2, 3) for jy in range(-2, 3))
        snaps.append(sigma0 ** 2 / s2 * G)
    np.testing.assert_allclose(Df.gaussian_hill_periodic(x, x, (0.0, 0.0), (L, L), sigma0, Dtrue, 20),
                               snaps[2], rtol=1e-13, atol=1e-300)
    Dfit, err = Df.fit_gaussian_D(snaps, times, x, x, (0.0, 0.0), (L, L), sigma0)
    assert abs(Dfit / Dtrue - 1.0) < 1e-7 and err < 1e-7
    # a wrong D leaves an error at every sample time
    wrong = Df.gaussian_errors(snaps, times, x, x, (0.0, 0.0), (L, L), sigma0, Dtrue * 1.5)
    assert wrong.min() > 1e-3


def test_fit_alphas_recovers_known_coefficients():
    pts = [(k, c, l) for k in (0.5, 1.0, 2.0, 5.0, 10.0) for c in (0.1, 0.25, 0.5, 1.0)
           for l in (0.0, 0.25, 0.5, 0.75)]
    k0, cfl, lam = (np.array(v) for v in zip(*pts))
    alpha = (-4.0 / 3.0, 0.48, 0.65)
    Dm = Df.model_D(alpha, k0, lam, cfl, 1.0, 2)
    assert np.all(Dm > 0)
    got, rms = Df.fit_alphas(k0, lam, cfl, 1.0, 2, Dm)
    np.testing.assert_allclose(got, alpha, rtol=1e-7, atol=1e-8)
    assert rms < 1e-10
    # the closed form of the scheme is not in the model's span, so it leaves a residual
    Dc = Df.closed_form_D(k0, lam, cfl, 1.0, 2, 2.0 / math.pi)
    got, rms = Df.fit_alphas(k0, lam, cfl, 1.0, 2, Dc)
    assert rms > 1e-3
