"""Diffusion coefficient of the scheme under pure scattering (App. A), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With kappa_a = eta = 0 the scheme spreads an energy hill diffusively
(Sec. 4.2.3).  App. A derives the leading diffusion coefficient by a
Chapman-Enskog expansion (Eq. numerical-diff-coeff) and App. A.2 extends it
with three fitted coefficients (Eq. numerical-diff-coeff2):

    chi = kappa_0 (1 + alpha_1 lambda / d),
    D   = c / (d chi) [1 - (1/2 + alpha_2) dt c chi] + (dx^2 / dt) alpha_3,

where each alpha is fitted to the D that makes the analytic Gaussian hill
(Eq. gauss-hill-analytic) match the simulations at t / dt = 5 ... 200.

This module gives three routes to D, all written from that description:

1. `moment_recursion`: the exact evolution of the spatial moments of one
   lattice axis on an unbounded lattice.  Eq. (interp) pulls from the own
   and the upwind cell of each axis with weights 1 - a and a
   (a = cfl |n^x|, shift s = sgn(n^x) dx), which moves the direction's
   moments m_k = sum_r x^k I(r) as
       m0* = m0,  m1* = m1 + a s m0,  m2* = m2 + 2 a s m1 + a s^2 m0.
   The collision (Eq. rte_implicit, solved exactly) is one linear map per
   site with the same coefficients everywhere, so it maps each moment
   vector (m_k,i over i) like a vector of populations.  The variance
   V = m2/m0 - (m1/m0)^2 of a unit pulse then follows step by step, and
   D = lim [V(t + dt) - V(t)] / (2 dt).
2. `closed_form_D` (pure-scattering, isotropic table): the flux relaxes by
   p = 1 / (1 + dt chi), chi = kappa_0 (1 - lambda/d), per step, so a
   direction's velocity c n^x has autocorrelation p^k; the persistent walk
   gives dt c^2 <n_x^2> (1 + p) / (2 (1 - p)) = 1/(d chi) + dt/(2d) (c = 1),
   and the Bernoulli part of the pull adds <a (1 - a)>_w dx^2 / (2 dt)
   = (dx/2) <|n^x|>_w - dt/(2d).  Net D = 1/(d chi) + (dx/2) <|n^x|>_w.
   The explicit collision (p = 1 - dt chi) gives 1/(d chi) - dt/d + (dx/2) <|n^x|>_w;
   its walk part is Eq. (numerical-diff-coeff).  (Both tested against route 1.)
3. `fit_gaussian_D`: App. A.2's procedure on a simulated E: the D whose
   Gaussian hill (with the periodic images of the box) is closest to the
   snapshots, measured by the largest relative L2 error over the sample
   times (reading: the paper asks for that error to stay below 1 %).

`fit_alphas` fits Eq. (numerical-diff-coeff2) to a set of (kappa_0, dt, dx,
lambda, D) points: for fixed alpha_1 the model is linear in alpha_2 and
alpha_3 (the chi in front of the bracket cancels the one inside it), so
alpha_1 is scanned on a grid, refined by golden-section search, and
(alpha_2, alpha_3) come from weighted linear least squares.
"""
import math

import numpy as np

from . import lb


# ----------------------------------------------------------------------------
# 1. exact spatial-moment recursion
# ----------------------------------------------------------------------------

def moment_recursion(n, w, dims, cfl, dx, kappa_0, lam, steps, axis=0, collision="implicit"):
    """Variance V(t_k) (k = 0 .. steps) along `axis` of the energy of a unit
    isotropic pulse (I_i = w_i at one site) on an unbounded lattice, pure
    scattering, with the exact implicit (Eq. rte_implicit) or the explicit
    (Eq. collision-step) collision.  Returns an array of length steps + 1,
    in the units of dx squared."""
    collide = lb.collide_implicit if collision == "implicit" else lb.collide_explicit
    n = np.asarray(n, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    lat = lb.Lattice(dims, (1, 1, 3), n, w, cfl=cfl, dx=dx)
    co = lb.Static(kappa_0=kappa_0, lam=lam)
    a = cfl * np.abs(n[:, axis])
    s = np.where(n[:, axis] >= 0.0, 1.0, -1.0) * dx
    # moment vectors as three "sites" of a 1 x 1 x 3 lattice: m[:, 0, 0, k]
    m = np.zeros((len(w), 1, 1, 3))
    m[:, 0, 0, 0] = w
    V = np.empty(steps + 1)
    V[0] = 0.0
    for t in range(1, steps + 1):
        m0, m1, m2 = m[:, 0, 0, 0].copy(), m[:, 0, 0, 1].copy(), m[:, 0, 0, 2].copy()
        m[:, 0, 0, 1] = m1 + a * s * m0
        m[:, 0, 0, 2] = m2 + 2.0 * a * s * m1 + a * s * s * m0
        m = collide(m, lat, co)
        M0, M1, M2 = m[:, 0, 0, 0].sum(), m[:, 0, 0, 1].sum(), m[:, 0, 0, 2].sum()
        V[t] = M2 / M0 - (M1 / M0) ** 2
    return V


def recursion_D(n, w, dims, cfl, dx, kappa_0, lam, axis=0, collision="implicit", tol=1e-13,
                max_steps=200000):
    """Asymptotic D of route 1: iterate until the per-step variance
    increment stops changing (relative tol), then D = dV / (2 dt)."""
    dt = cfl * dx
    chi_dt = dt * kappa_0 * (1.0 - lam / dims)
    # flux retention per step; the transient decays like |p|^t
    p = 1.0 / (1.0 + chi_dt) if collision == "implicit" else 1.0 - chi_dt
    assert abs(p) < 1.0, "no diffusive limit"
    steps = int(min(max_steps, max(50, math.ceil(40.0 / max(1e-12, -math.log(max(abs(p), 1e-300)))))))
    V = moment_recursion(n, w, dims, cfl, dx, kappa_0, lam, steps, axis, collision)
    inc = np.diff(V)
    assert abs(inc[-1] - inc[-2]) <= tol * abs(inc[-1]) + 1e-300, "variance increment not settled"
    return inc[-1] / (2.0 * dt)


# ----------------------------------------------------------------------------
# 2. closed form
# ----------------------------------------------------------------------------

def closed_form_D(kappa_0, lam, dt, dx, dims, mean_abs_nx, collision="implicit"):
    """D = 1/(d chi) + (dx/2) <|n^x|>_w, chi = kappa_0 (1 - lambda/d), c = 1.
    The explicit collision retains p = 1 - dt chi of the flux per step, so
    its walk term is 1/(d chi) - dt/(2d) and D = 1/(d chi) - dt/d + (dx/2) <|n^x|>_w."""
    chi = kappa_0 * (1.0 - lam / dims)
    D = 1.0 / (dims * chi) + 0.5 * dx * mean_abs_nx
    return D if collision == "implicit" else D - dt / dims


# ----------------------------------------------------------------------------
# 3. App. A.2: D fitted to Gaussian snapshots
# ----------------------------------------------------------------------------

def gaussian_hill_periodic(x, y, centre, box, sigma0, D, t, dims=2, images=2):
    """Eq. (gauss-hill-analytic) in 2D with amplitude 1 on the grid of cell
    centres x (columns) and y (rows), summed over the periodic images of a
    box (Lx, Ly).  The sum over image pairs factorises,
    sum_jx sum_jy exp(-(dx_j^2 + dy_j^2) / 2s^2) = (sum_jx exp(-dx_j^2 / 2s^2)) (sum_jy ...),
    which is how it is evaluated."""
    s2 = sigma0 ** 2 + 2.0 * D * t
    amp = (sigma0 ** 2 / s2) ** (dims / 2.0)
    gx = np.zeros(len(x))
    gy = np.zeros(len(y))
    for j in range(-images, images + 1):
        gx += np.exp(-(np.asarray(x) - centre[0] + j * box[0]) ** 2 / (2.0 * s2))
        gy += np.exp(-(np.asarray(y) - centre[1] + j * box[1]) ** 2 / (2.0 * s2))
    return amp * np.outer(gy, gx)


def gaussian_errors(E_snaps, times, x, y, centre, box, sigma0, D):
    """Relative L2 error of each snapshot (rows y, columns x) against the
    periodic Gaussian hill."""
    errs = []
    for E, t in zip(E_snaps, times):
        G = gaussian_hill_periodic(x, y, centre, box, sigma0, D, t)
        errs.append(np.linalg.norm(E - G) / np.linalg.norm(G))
    return np.array(errs)


def fit_gaussian_D(E_snaps, times, x, y, centre, box, sigma0, D_lo=1e-4, D_hi=1e2,
                   iters=200):
    """D minimising the largest relative L2 error over the snapshots, by
    golden-section search in log D.  Returns (D, that largest error)."""
    def cost(logD):
        return gaussian_errors(E_snaps, times, x, y, centre, box, sigma0, math.exp(logD)).max()

    lo, hi = math.log(D_lo), math.log(D_hi)
    # coarse scan first: the cost is unimodal near its minimum but flat far away
    grid = np.linspace(lo, hi, 61)
    vals = [cost(g) for g in grid]
    k = int(np.argmin(vals))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = hi - g * (hi - lo), lo + g * (hi - lo)
    fc, fd = cost(c), cost(d)
    for _ in range(iters):
        if hi - lo < 1e-12:
            break
        if fc < fd:
            hi, d, fd = d, c, fc
            c = hi - g * (hi - lo)
            fc = cost(c)
        else:
            lo, c, fc = c, d, fd
            d = lo + g * (hi - lo)
            fd = cost(d)
    u = 0.5 * (lo + hi)
    return math.exp(u), cost(u)


# ----------------------------------------------------------------------------
# Eq. (numerical-diff-coeff2) fit
# ----------------------------------------------------------------------------

def model_D(alpha, kappa_0, lam, dt, dx, dims, c=1.0):
    """Eq. (numerical-diff-coeff2) with chi = kappa_0 (1 + alpha_1 lambda / d)."""
    a1, a2, a3 = alpha
    chi = kappa_0 * (1.0 + a1 * lam / dims)
    return c / (dims * chi) * (1.0 - (0.5 + a2) * dt * c * chi) + dx * dx / dt * a3


def _linear_part(a1, kappa_0, lam, dt, dx, dims, D):
    """Best (alpha_2, alpha_3) for fixed alpha_1 and the relative residual norm."""
    chi = kappa_0 * (1.0 + a1 * lam / dims)
    if np.any(chi <= 0.0):
        return None, np.inf
    # D = 1/(d chi) - dt/(2d) - alpha_2 dt/d + alpha_3 dx^2/dt, weighted by 1/D
    rhs = (D - 1.0 / (dims * chi) + dt / (2.0 * dims)) / D
    Amat = np.stack([-dt / dims / D, dx * dx / dt / D], axis=1)
    sol, *_ = np.linalg.lstsq(Amat, rhs, rcond=None)
    res = Amat @ sol - rhs
    return sol, float(np.sqrt(np.mean(res * res)))


def fit_alphas(kappa_0, lam, dt, dx, dims, D, a1_range=(-3.0, 3.0)):
    """(alpha_1, alpha_2, alpha_3) of Eq. (numerical-diff-coeff2) by least
    squares of the relative residual; returns (alphas, rms relative residual)."""
    kappa_0, lam, dt, dx, D = (np.asarray(x, dtype=np.float64) for x in (kappa_0, lam, dt, dx, D))
    grid = np.linspace(a1_range[0], a1_range[1], 601)
    vals = [_linear_part(a, kappa_0, lam, dt, dx, dims, D)[1] for a in grid]
    k = int(np.argmin(vals))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    f = lambda a: _linear_part(a, kappa_0, lam, dt, dx, dims, D)[1]
    c, d = hi - g * (hi - lo), lo + g * (hi - lo)
    fc, fd = f(c), f(d)
    for _ in range(200):
        if hi - lo < 1e-13:
            break
        if fc < fd:
            hi, d, fd = d, c, fc
            c = hi - g * (hi - lo)
            fc = f(c)
        else:
            lo, c, fc = c, d, fd
            d = lo + g * (hi - lo)
            fd = f(d)
    a1 = 0.5 * (lo + hi)
    sol, rms = _linear_part(a1, kappa_0, lam, dt, dx, dims, D)
    return (a1, float(sol[0]), float(sol[1])), rms
