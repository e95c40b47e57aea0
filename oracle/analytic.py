"""Closed-form references the oracle is pinned against (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import math

import numpy as np


# ----------------------------------------------------------------------------
# homogeneous radiating sphere (Sec. 4.2.2)
# ----------------------------------------------------------------------------

def sphere_f(r, mu, R, kappa, b=1.0):
    """Steady intensity f(r, mu) = b (1 - exp(-kappa s(r, mu))), with the path
    length through the sphere s = r mu + R g inside, s = 2 R g outside for
    sqrt(1 - R^2/r^2) < mu < 1 and 0 otherwise, g = sqrt(1 - r^2/R^2 (1 - mu^2)).
    b = eta / kappa_a = 1 for eta = kappa_a."""
    r = np.asarray(r, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    g2 = 1.0 - (r / R) ** 2 * (1.0 - mu ** 2)
    g = np.sqrt(np.clip(g2, 0.0, None))
    inside = r < R
    ratio = np.where(inside, 1.0, R / np.where(inside, 1.0, r))
    mu_c = np.sqrt(np.clip(1.0 - ratio ** 2, 0.0, None))
    s = np.where(inside, r * mu + R * g, np.where(mu > mu_c, 2.0 * R * g, 0.0))
    return b * (1.0 - np.exp(-kappa * s))


def sphere_EF(r, R, kappa, order=200):
    """E(r) = 1/2 int f dmu and F(r) = 1/2 int mu f dmu (Eqs. radsph_1, radsph_2),
    by Gauss-Legendre quadrature split at the kink mu_c = sqrt(1 - R^2/r^2)."""
    x, wx = np.polynomial.legendre.leggauss(order)

    def integrate(lo, hi, rr, moment):
        mu = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        f = sphere_f(rr, mu, R, kappa)
        return 0.5 * (hi - lo) * np.sum(wx * f * mu ** moment)

    E, F = [], []
    for rr in np.atleast_1d(r):
        if rr < R:
            pieces = [(-1.0, 1.0)]
        else:
            mu_c = math.sqrt(max(0.0, 1.0 - (R / rr) ** 2))
            pieces = [(mu_c, 1.0)]
        E.append(0.5 * sum(integrate(lo, hi, rr, 0) for lo, hi in pieces))
        F.append(0.5 * sum(integrate(lo, hi, rr, 1) for lo, hi in pieces))
    return np.array(E), np.array(F)


# ----------------------------------------------------------------------------
# Gaussian diffusion (Sec. 4.2.3, App. A)
# ----------------------------------------------------------------------------

def gaussian_E(r2, t, sigma0, D, A=1.0, dims=2):
    """Eq. (gauss-hill-analytic) with sigma_D^2 = 2 D t.  The amplitude factor
    is (sigma0^2 / (sigma0^2 + sigma_D^2))^{d/2}; the printed exponent 1 is
    the d = 2 case."""
    s2 = sigma0 ** 2 + 2.0 * D * t
    return A * (sigma0 ** 2 / s2) ** (dims / 2.0) * np.exp(-r2 / (2.0 * s2))


def diffusion_coefficient(kappa_0, dt, dx, dims, mean_abs_nx, scheme="implicit"):
    """Diffusion coefficient of the scheme for lambda = 0, c = 1.

    The collision part follows the Chapman-Enskog result of App. A
    (Eq. numerical-diff-coeff): D = (1/(d kappa_0)) (1 - kappa_0 dt / 2) for the
    explicit relaxation omega = kappa_0 dt.  For the implicit collision the
    relaxation is omega' = kappa_0 dt / (1 + kappa_0 dt), which gives
    dt/d (1/omega' - 1/2).  The pull interpolation adds, per axis, the
    variance of a Bernoulli shift of probability a = cfl |n^x|, i.e.
    (dx^2 / (2 dt)) <a (1 - a)>_w; with <(n^x)^2>_w = 1/d its second part
    cancels the -dt/(2d) of the collision term.  Net:
        implicit: D = 1/(d kappa_0) + (dx/2) <|n^x|>_w
        explicit: D = (1 - kappa_0 dt)/(d kappa_0) + (dx/2) <|n^x|>_w
    (the interpolation term plays the role of the fitted background
    diffusivity of Eq. numerical-diff-coeff2)."""
    if scheme == "implicit":
        return 1.0 / (dims * kappa_0) + 0.5 * dx * mean_abs_nx
    return (1.0 - kappa_0 * dt) / (dims * kappa_0) + 0.5 * dx * mean_abs_nx


# ----------------------------------------------------------------------------
# dense brute-force collision solves
# ----------------------------------------------------------------------------

def dense_static_solve(Is, n, w, dt, kappa_a, kappa_0, lam, eta):
    """Solve Eq. (rte_implicit) at one site as the full N x N linear system
        (1 + dt (kappa_0 + kappa_a)) I_i - dt kappa_0 w_i sum_j (1 + lam n_i.n_j) I_j
            = I*_i + dt w_i eta
    with numpy.linalg.solve (LAPACK gesv)."""
    N = len(w)
    M = np.eye(N) * (1.0 + dt * (kappa_0 + kappa_a))
    M -= dt * kappa_0 * w[:, None] * (1.0 + lam * (n @ n.T))
    return np.linalg.solve(M, Is + dt * w * eta)


def dense_moving_solve(Is, n, w, dt, v, kt_a, kt_0, eta_t):
    """The mixed-frame implicit step (App. B) at one site as an N x N system:
        (1 + dt W beta_i (kt_a + kt_0)) I_i - dt w_i D_i kt_0 W^2 sum_j beta_j^2 I_j
            = I*_i + dt w_i D_i eta_t,
    beta_i = 1 - v.n_i, D_i = (W beta_i)^-3, solved with numpy.linalg.solve."""
    v = np.asarray(v, dtype=np.float64)
    W = 1.0 / math.sqrt(1.0 - v @ v)
    beta = 1.0 - n @ v
    D = 1.0 / (W * beta) ** 3
    N = len(w)
    M = np.diag(1.0 + dt * W * beta * (kt_a + kt_0))
    M -= dt * kt_0 * W ** 2 * (w * D)[:, None] * (beta ** 2)[None, :]
    return np.linalg.solve(M, Is + dt * w * D * eta_t)


def wave_shell_E(r, t, R):
    """Free streaming of a uniform isotropic ball (radius R, E = 1) in vacuum:
    E(r, t) is the fraction of directions n with |r - n t| < R, i.e.
    (1 - c*) / 2 with c* = (r^2 + t^2 - R^2) / (2 r t), clipped to [0, 1]
    (c* <= -1 inside the moving ball).  Any direction set gives this shell
    average, since every direction carries a translated copy of the ball."""
    r = np.asarray(r, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        c = (r ** 2 + t ** 2 - R ** 2) / (2.0 * r * t)
    c = np.where(r * t > 0, c, np.where(r < R, -1.0, 1.0))
    return np.clip((1.0 - np.clip(c, -1.0, 1.0)) / 2.0, 0.0, 1.0)


def wave_peak(t, R):
    """max_r wave_shell_E(r, t, R) = (1 - sqrt(1 - R^2 / t^2)) / 2 for t > R
    (at r = sqrt(t^2 - R^2)); tends to R^2 / (4 t^2), the inverse-square law."""
    return (1.0 - math.sqrt(1.0 - (R / t) ** 2)) / 2.0


def wave_second_moment(lat, ball_mass, ball_S2, steps):
    """Exact energy-weighted second moment sum_x E |x - c|^2 (cells^2) of the
    discrete pull scheme after `steps` steps in vacuum, before any energy
    leaves the box: each direction carries the ball shifted by a binomial
    walk with success probability a = cfl |n^a| per axis (Eq. interp), so
    sum_i w_i [S2 + m (steps^2 cfl^2 |n_i|^2 + steps sum_a a (1 - a))] with
    m and S2 the ball's mass and second moment about its centre."""
    a = lat.cfl * np.abs(lat.n[:, :lat.dims])
    walk = steps ** 2 * lat.cfl ** 2 * np.sum(lat.n[:, :lat.dims] ** 2, axis=1) \
        + steps * np.sum(a * (1.0 - a), axis=1)
    return float(np.sum(lat.w * (ball_S2 + ball_mass * walk)))

