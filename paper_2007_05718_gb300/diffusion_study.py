"""Diffusion-coefficient study of App. A.2, run through the batch C ABI.

A Gaussian energy hill (Sec. 4.2.3) diffuses under pure scattering
(kappa_a = eta = 0) on a periodic 2D grid, for a sweep of Peclet numbers
kappa_0 dx, time steps dt / dx (the CFL number) and lambda = 3 kappa_1 /
kappa_0.  Every sweep point is one problem of one batch (all points share
the direction table, so each step is one persistent launch over all of
them); E is read back at the sample times t / dt = 5 ... 200.  From the
snapshots two diffusion coefficients are taken per point:

- `variance_D`: the growth of the hill's variance along x between the last
  two samples, [V(t2) - V(t1)] / (2 (t2 - t1)); for a linear scheme this is
  the spreading of its Green's function, independent of the initial shape;
- `fit_gaussian_D`: App. A.2's procedure, the D whose analytic hill (Eq.
  gauss-hill-analytic, with the periodic images of the box) is closest to
  the snapshots in the largest relative L2 error over the sample times.

`fit_alphas` fits Eq. (numerical-diff-coeff2),
    chi = kappa_0 (1 + alpha_1 lambda / d),
    D = c / (d chi) [1 - (1/2 + alpha_2) dt c chi] + (dx^2 / dt) alpha_3,
to the per-point D by nonlinear least squares of the relative residual.

Lengths are in cells (dx = 1), c = 1, so dt = CFL and kappa_0 = kappa_0 dx.
The stepping runs in liblbrt.so; this module marshals, reads E back and
does the host-side fits.
"""
import itertools
import math

import numpy as np

from . import lbrt
from . import workloads as W

SAMPLE_STEPS = (5, 10, 20, 50, 100, 150, 200)


def sweep_points(kappa_0_dx=(0.5, 1.0, 2.0, 5.0, 10.0), cfl=(0.1, 0.25, 0.5, 1.0),
                 lam=(0.0, 0.25, 0.5, 0.75)):
    """All combinations, as dicts {kappa_0, cfl, lam}."""
    return [dict(kappa_0=k, cfl=c, lam=l) for k, c, l in itertools.product(kappa_0_dx, cfl, lam)]


def run_sweep(points, *, n=512, ndir=120, sigma0=10.0, sample_steps=SAMPLE_STEPS,
              storage=lbrt.LB_RT_F32, collision=lbrt.LB_RT_IMPLICIT_EXACT):
    """Run every point on an n x n periodic grid with the ndir-direction 2D
    ring; returns {"E": [points][samples] float32 (n, n) arrays, "steps",
    "sigma0", "n", "mean_abs_nx"}."""
    E0 = W.gaussian_E0((1, n, n), sigma0)
    tick = math.gcd(*sample_steps)
    last = max(sample_steps)
    b = lbrt.lb_rt_batch_create(max_problems=len(points), storage=storage, steps_per_tick=tick,
                                use_graph=True, autotune=False)
    snaps = [[None] * len(sample_steps) for _ in points]
    try:
        slots = []
        for p in points:
            problem = dict(dims=2, nx=n, ny=n, nz=1, dirset=lbrt.LB_RT_RING2D, ndir=ndir,
                           cfl=p["cfl"], dx=1.0, bc=(lbrt.LB_RT_PERIODIC,) * 3,
                           collision=collision)
            s = lbrt.lb_rt_batch_admit(b, problem, dict(kappa_0=p["kappa_0"], lam=p["lam"]), E0,
                                       lbrt.LB_RT_STATE_ISOTROPIC, last)
            if s is None:
                raise RuntimeError("sweep does not fit the device memory budget")
            slots.append(s)
        done = 0
        while done < last:
            lbrt.lb_rt_batch_tick(b)
            lbrt.lb_rt_batch_sync(b)
            done = lbrt.lb_rt_batch_steps(b, slots[0])
            if done in sample_steps:
                k = sample_steps.index(done)
                for j, s in enumerate(slots):
                    assert lbrt.lb_rt_batch_steps(b, s) == done
                    E = np.zeros(n * n, dtype=np.float32)
                    lbrt.lb_rt_batch_moments(b, s, E)
                    snaps[j][k] = E.reshape(n, n)
    finally:
        lbrt.lb_rt_batch_destroy(b)
    phi = 2.0 * math.pi * np.arange(ndir) / ndir
    return dict(E=snaps, steps=tuple(sample_steps), sigma0=sigma0, n=n,
                mean_abs_nx=float(np.mean(np.abs(np.cos(phi)))))


def centred_coords(n):
    """Cell-centre coordinates relative to the hill's centre (the box centre)."""
    x = np.arange(n) + 0.5 - 0.5 * n
    return np.meshgrid(x, x, indexing="xy")


def variance(E, axis=0):
    """Second central moment of E along x (axis 0) or y (axis 1), in cells^2."""
    X, Y = centred_coords(E.shape[0])
    q = X if axis == 0 else Y
    E = E.astype(np.float64)
    m0 = E.sum()
    m1 = (q * E).sum() / m0
    return float((q * q * E).sum() / m0 - m1 * m1)


def variance_D(snaps, steps, dt, axis=0):
    """[V(t2) - V(t1)] / (2 (t2 - t1)) from the last two snapshots."""
    V1, V2 = variance(snaps[-2], axis), variance(snaps[-1], axis)
    return (V2 - V1) / (2.0 * (steps[-1] - steps[-2]) * dt)


def hill(n, sigma0, D, t, images=2):
    """Eq. (gauss-hill-analytic) in 2D, amplitude 1, on the periodic n x n
    box (rows y, columns x); the image sum is separable in x and y."""
    x = np.arange(n) + 0.5 - 0.5 * n
    s2 = sigma0 * sigma0 + 2.0 * D * t
    g = sum(np.exp(-(x + j * n) ** 2 / (2.0 * s2)) for j in range(-images, images + 1))
    return (sigma0 * sigma0 / s2) * np.outer(g, g)


def hill_error(snaps, steps, dt, sigma0, D):
    """Largest relative L2 error of the snapshots against the hill with D."""
    n = snaps[0].shape[0]
    worst = 0.0
    for E, k in zip(snaps, steps):
        G = hill(n, sigma0, D, k * dt)
        E = np.asarray(E, dtype=np.float64)
        worst = max(worst, float(np.linalg.norm(E - G) / np.linalg.norm(G)))
    return worst


def fit_gaussian_D(snaps, steps, dt, sigma0, D_guess):
    """App. A.2: D minimising the largest relative L2 error over the sample
    times (bounded Brent search in log D around D_guess); returns (D, error)."""
    from scipy.optimize import minimize_scalar
    f = lambda u: hill_error(snaps, steps, dt, sigma0, math.exp(u))
    c = math.log(D_guess)
    r = minimize_scalar(f, bounds=(c - 2.0, c + 2.0), method="bounded",
                        options=dict(xatol=1e-10, maxiter=500))
    return math.exp(r.x), float(r.fun)


def model_D(alpha, kappa_0, lam, dt, dx=1.0, dims=2):
    """Eq. (numerical-diff-coeff2), c = 1."""
    chi = kappa_0 * (1.0 + alpha[0] * lam / dims)
    return 1.0 / (dims * chi) * (1.0 - (0.5 + alpha[1]) * dt * chi) + dx * dx / dt * alpha[2]


def fit_alphas(kappa_0, lam, dt, D, dx=1.0, dims=2, x0=(-1.0, 0.0, 0.3)):
    """(alpha_1, alpha_2, alpha_3) minimising the relative residual of Eq.
    (numerical-diff-coeff2); returns (alphas, rms relative residual)."""
    from scipy.optimize import least_squares
    kappa_0, lam, dt, D = (np.asarray(x, dtype=np.float64) for x in (kappa_0, lam, dt, D))

    def res(a):
        return model_D(a, kappa_0, lam, dt, dx, dims) / D - 1.0

    r = least_squares(res, np.asarray(x0, dtype=np.float64), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return tuple(float(v) for v in r.x), float(np.sqrt(np.mean(r.fun ** 2)))


def study(points=None, **kw):
    """Run the sweep and both fits; returns per-point rows and the alphas."""
    points = sweep_points() if points is None else points
    out = run_sweep(points, **kw)
    rows = []
    for p, snaps in zip(points, out["E"]):
        dv = variance_D(snaps, out["steps"], p["cfl"])
        dg, err = fit_gaussian_D(snaps, out["steps"], p["cfl"], out["sigma0"], dv)
        rows.append(dict(p, D_variance=dv, D_gauss=dg, gauss_err=err))
    k0 = [r["kappa_0"] for r in rows]
    lam = [r["lam"] for r in rows]
    dt = [r["cfl"] for r in rows]
    diffusive = [r for r in rows if r["gauss_err"] <= 0.01]
    fits = {
        "variance": fit_alphas(k0, lam, dt, [r["D_variance"] for r in rows]),
        "gauss": fit_alphas([r["kappa_0"] for r in diffusive], [r["lam"] for r in diffusive],
                            [r["cfl"] for r in diffusive], [r["D_gauss"] for r in diffusive])
        if len(diffusive) >= 3 else None,
    }
    return dict(rows=rows, fits=fits, n_diffusive=len(diffusive), raw=out)
