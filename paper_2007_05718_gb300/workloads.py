"""Seeded synthetic inputs for the radiative LB problems.

This module holds only input recipes (fields, masks, initial moments,
request streams).  It contains none of the method's arithmetic: no direction
tables, no streaming stencil, no collision.  Both the CUDA path and the CPU
checker take their inputs from here, so it imports nothing but numpy.

All fields are returned as float32 arrays of shape (nz, ny, nx) (x fastest);
lengths are in units of the domain length L along x, cell centres sit at
(i + 1/2) dx with dx = 1 / nx.
"""
import math

import numpy as np


def _centres(shape, dx):
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    x = (np.arange(nx) + 0.5) * dx
    return np.meshgrid(z, y, x, indexing="ij")


def radius(shape, centre, dx):
    """Distance of every cell centre from `centre` = (x, y, z)."""
    Z, Y, X = _centres(shape, dx)
    return np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)


def gaussian_E0(shape, sigma_cells, amplitude=1.0, centre=None):
    """E0 = A exp(-|r - r0|^2 / (2 sigma^2)), sigma in cells, centred in the box
    by default (the Gaussian-diffusion initial data)."""
    nz, ny, nx = shape
    dx = 1.0 / nx
    if centre is None:
        centre = (0.5 * nx * dx, 0.5 * ny * dx, 0.5 * nz * dx)
    r = radius(shape, centre, dx)
    s = sigma_cells * dx
    return (amplitude * np.exp(-r * r / (2.0 * s * s))).astype(np.float32)


def radiating_sphere(n, kappa_R, R=0.25, centre=(0.5, 0.5, 0.5)):
    """Homogeneous radiating sphere on an n^3 grid: kappa_a = eta = kappa_R / R
    for cell centres strictly inside radius R, 0 outside; initial E0 = 1
    inside and (R/r)^2 outside.  Returns dict of float32 fields."""
    shape = (n, n, n)
    dx = 1.0 / n
    r = radius(shape, centre, dx)
    inside = r < R
    k = np.where(inside, kappa_R / R, 0.0).astype(np.float32)
    E0 = np.where(inside, 1.0, (R / np.maximum(r, 1e-30)) ** 2).astype(np.float32)
    return {"kappa_a": k, "eta": k.copy(), "E0": E0, "R": R, "centre": centre}


def shadow(n, kappa_emit, R=0.125, emit_centre=(0.25, 0.5, 0.5),
           absorb_centre=(0.625, 0.5, 0.5), kappa_absorb=1e4):
    """Shadow-casting problem: an emitting sphere (eta = kappa_a = kappa_emit)
    in front of a black absorber (kappa_a = kappa_absorb, eta = 0)."""
    shape = (n, n, n)
    dx = 1.0 / n
    re = radius(shape, emit_centre, dx)
    ra = radius(shape, absorb_centre, dx)
    ka = np.zeros(shape)
    eta = np.zeros(shape)
    ka[re < R] = kappa_emit
    eta[re < R] = kappa_emit
    ka[ra < R] = kappa_absorb
    E0 = np.zeros(shape)
    return {"kappa_a": ka.astype(np.float32), "eta": eta.astype(np.float32),
            "E0": E0.astype(np.float32)}


def wave_ball(n, R_cells, centre=None):
    """Free-streaming wave (Sec. 4.1.2, radiation wave): E0 = 1 at cell centres
    closer than R_cells cells to the centre of an n^3 box, 0 elsewhere
    (isotropic populations I_i = w_i E0 are set by the caller).  Returns
    (E0 float32 [n, n, n], centre in cell units)."""
    c = (n / 2.0,) * 3 if centre is None else centre
    idx = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    return (r2 < R_cells ** 2).astype(np.float32), c


def random_fields(shape, seed, lo=0.5, hi=1.5):
    """Strictly positive seeded field, uniform in [lo, hi)."""
    g = np.random.default_rng(seed)
    return g.uniform(lo, hi, size=shape).astype(np.float32)


def random_populations(N, shape, seed, lo=0.0, hi=1.0):
    """Seeded populations I[i, z, y, x], uniform in [lo, hi) / N."""
    g = np.random.default_rng(seed)
    return (g.uniform(lo, hi, size=(N,) + tuple(shape)) / N).astype(np.float32)


def random_moments(shape, seed, flux_frac=0.2):
    """Seeded (E0, F0) with E0 in [0.5, 1.5) and |F0| <= flux_frac * E0 / 3, so
    that populations built as P1 states from them stay positive."""
    g = np.random.default_rng(seed)
    E = g.uniform(0.5, 1.5, size=shape)
    F = g.uniform(-1.0, 1.0, size=(3,) + tuple(shape))
    F *= (flux_frac * E / (3.0 * math.sqrt(3.0)))[None]
    return E.astype(np.float32), F.astype(np.float32)


def smooth_field(shape, seed, modes=8, amplitude=1.0):
    """Sum of `modes` seeded random Fourier modes on the periodic box, each
    of unit amplitude times `amplitude` / modes, wave numbers 1..3."""
    nz, ny, nx = shape
    dx = 1.0 / nx
    Z, Y, X = _centres(shape, dx)
    g = np.random.default_rng(seed)
    out = np.zeros(shape)
    for _ in range(modes):
        kx, ky, kz = g.integers(1, 4, size=3)
        ph = g.uniform(0, 2 * math.pi)
        out += np.sin(2 * math.pi * (kx * X + ky * Y * nx / max(ny, 1) + kz * Z * nx / max(nz, 1)) + ph)
    return amplitude * out / modes


def moving_fluid(n, seed=20200712, delta=0.02, vmax=0.6):
    """Relativistic moving background on an n^3 periodic box: a double tanh
    shear layer in v_x plus 8 seeded Fourier modes (amplitude 0.05) on every
    component, rescaled where |v| > vmax; a seeded smooth rho in [0, 1];
    kt_a = 0.1 * 1000^rho, kt_0 = 100 rho, eta_t = kt_a (E_eq = 1)."""
    shape = (n, n, n)
    dx = 1.0 / n
    Z, Y, X = _centres(shape, dx)
    vx = 0.5 * (np.tanh((Y - 0.25) / delta) - np.tanh((Y - 0.75) / delta) - 1.0)
    v = np.stack([vx, np.zeros(shape), np.zeros(shape)])
    for c in range(3):
        v[c] += smooth_field(shape, seed + c, modes=8, amplitude=0.05 * 8)
    speed = np.sqrt((v ** 2).sum(axis=0))
    scale = np.where(speed > vmax, vmax / np.maximum(speed, 1e-30), 1.0)
    v *= scale[None]
    rho = smooth_field(shape, seed + 7, modes=8, amplitude=8.0)
    rho = (rho - rho.min()) / max(rho.max() - rho.min(), 1e-30)
    kt_a = 0.1 * 1000.0 ** rho
    kt_0 = 100.0 * rho
    return {"v": v.astype(np.float32), "kt_a": kt_a.astype(np.float32),
            "kt_0": kt_0.astype(np.float32), "eta_t": kt_a.astype(np.float32)}


def serving_requests(count, seed=20200711, sizes=(32, 48, 64, 96, 128),
                     ndirs=(42, 162), steps=(200, 2000), rate=1.0):
    """Seeded request stream: Poisson arrival times at `rate` per second,
    kind in {sphere, shadow}, cubic size, direction count, log-uniform
    opacity in [1e-1, 1e4], step count uniform in [steps[0], steps[1]]."""
    g = np.random.default_rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    reqs = []
    for k in range(count):
        reqs.append({
            "id": k,
            "arrival": float(t[k]),
            "kind": "sphere" if g.random() < 0.5 else "shadow",
            "n": int(g.choice(sizes)),
            "ndir": int(g.choice(ndirs)),
            "kappa": float(10.0 ** g.uniform(-1.0, 4.0)),
            "steps": int(g.integers(steps[0], steps[1] + 1)),
        })
    return reqs
