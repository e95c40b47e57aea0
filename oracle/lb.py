"""One timestep of the grey radiative Lattice-Boltzmann scheme, FP64 (oracle).

Follows Sec. 3.3 ("Numerical procedure") step by step:

1. pull-streaming, I*_i(r) = I_i(r - n_i dt)  (Eq. rte-stream-collide), with the
   off-lattice value taken by the trilinear rule of Eq. (interp) (bilinear in
   2D): the eight (four) upwind corners r - sum_a b_a sgn(n_i^a) e_a, b in
   {0,1}^d, weighted by prod_a [b_a cfl|n_i^a| + (1 - b_a)(1 - cfl|n_i^a|)];
2. moments E = sum_i I_i, F = sum_i n_i I_i, P = sum_i n_i n_i I_i
   (Eqs. moments_discrete, higher_moments; the I_i carry the weights w_i);
3. the collision, in one of three forms:
   - explicit (Eq. collision-step) with I^eq_i = w_i (E + lambda n_i.F) and
     S_i = w_i eta - kappa_a I_i (Eq. source-and-equil);
   - implicit (Eq. rte_implicit), solved exactly.  The N x N system couples
     the directions only through (E, F), so it is solved as the equivalent
     (1+d) x (1+d) system for the new (E, F) built from the table sums
     T0 = sum w, T1 = sum w n, T2 = sum w n n (Eq. iso-tensors), then every
     I_i follows directly;
   - implicit by the literal Lambda iteration of Sec. 3.3 (initial guess:
     the moments of the streamed field; stop when |dE| <= tol |E| and
     |dF| <= tol |E| at every site), either to convergence or for a fixed
     number of cycles;
   - moving fluid (App. B, mixed-frame equation): per direction
     beta_i = 1 - v.n_i, lab-frame extinction W beta_i (kt_a + kt_0) and
     emission w_i (eta_t + kt_0 J) / (W beta_i)^3, with the fluid-frame energy
     density J = W^2 (E - 2 F.v + P:vv) = W^2 sum_i beta_i^2 I_i (Eq. J) taken
     at the new time level; exact solution by the scalar reduction in J, or
     by the literal Lambda iteration on J;
4. frozen cells: their populations are overwritten with prescribed values
   after the collision, so they act as sources for the next stream
   (Sec. 4.1.1, the injected and frozen beam regions).

Units: c = 1, dt = cfl * dx, interpolation weights a_{i,a} = cfl |n_i^a|.
Arrays: populations I[i, z, y, x] (direction-major, x fastest); per-site
coefficient fields are scalars or arrays of shape (nz, ny, nx).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from dataclasses import dataclass, field
import itertools

import numpy as np

from .directions import sgn

PERIODIC, VACUUM = "periodic", "vacuum"
_AXIS = {0: 2, 1: 1, 2: 0}  # lattice axis a (x, y, z) -> array axis of (nz, ny, nx)


@dataclass
class Lattice:
    dims: int                 # 2 or 3
    shape: tuple              # (nz, ny, nx); nz == 1 in 2D
    n: np.ndarray             # (N, 3) unit vectors (n_z = 0 in 2D)
    w: np.ndarray             # (N,) weights
    cfl: float                # c dt / dx, 0 < cfl <= 1
    dx: float = 1.0
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)   # per axis x, y, z

    @property
    def dt(self):
        return self.cfl * self.dx

    @property
    def N(self):
        return len(self.w)

    def table_sums(self):
        """T0 = sum w, T1 = sum w n, T2 = sum w n n^T restricted to d axes."""
        d = self.dims
        n = self.n[:, :d]
        return self.w.sum(), self.w @ n, np.einsum("i,ia,ib->ab", self.w, n, n)


@dataclass
class Static:
    """Static-fluid coefficients (Eq. rte_gray_bgkform): absorption kappa_a,
    scattering kappa_0, lambda = 3 kappa_1 / kappa_0, emissivity eta."""
    kappa_a: object = 0.0
    kappa_0: object = 0.0
    lam: object = 0.0
    eta: object = 0.0


@dataclass
class Moving:
    """Fluid-frame coefficients and velocity for the mixed-frame equation of
    App. B (kappa_1 = 0): v (3, ...), kt_a, kt_0, eta_t."""
    v: np.ndarray = None
    kt_a: object = 0.0
    kt_0: object = 0.0
    eta_t: object = 0.0


# ----------------------------------------------------------------------------
# 1. streaming
# ----------------------------------------------------------------------------

def _pull(f, k, axis, bc):
    """g(r) = f(r - k e_axis) for k in {-1, 0, 1}; outside the domain a
    periodic axis wraps and a vacuum axis reads zero."""
    if k == 0:
        return f
    g = np.roll(f, k, axis=axis)
    if bc == VACUUM:
        idx = [slice(None)] * f.ndim
        idx[axis] = slice(0, k) if k > 0 else slice(f.shape[axis] + k, None)
        g[tuple(idx)] = 0.0
    return g


def stream(I, lat):
    """I*_i(r) = sum over the 2^d upwind corners of Eq. (interp)."""
    d = lat.dims
    out = np.zeros_like(I)
    for i in range(lat.N):
        s = sgn(lat.n[i, :d])
        a = lat.cfl * np.abs(lat.n[i, :d])
        for b in itertools.product((0, 1), repeat=d):
            weight = 1.0
            g = I[i]
            for ax in range(d):
                weight *= a[ax] if b[ax] else 1.0 - a[ax]
                g = _pull(g, b[ax] * int(s[ax]), _AXIS[ax], lat.bc[ax])
            out[i] += weight * g
    return out


def stream_sites(value_at, sites, lat):
    """The same stencil evaluated at selected sites only.

    value_at(i, z, y, x) returns the populations of direction i at integer
    coordinates (arrays, already inside the domain); sites = (z, y, x) arrays.
    Returns I* of shape (N, S)."""
    d = lat.dims
    z0, y0, x0 = (np.asarray(c, dtype=np.int64) for c in sites)
    nz, ny, nx = lat.shape
    ext = (nx, ny, nz)
    out = np.zeros((lat.N, len(z0)))
    for i in range(lat.N):
        s = sgn(lat.n[i, :d])
        a = lat.cfl * np.abs(lat.n[i, :d])
        for b in itertools.product((0, 1), repeat=d):
            weight = 1.0
            c = [x0.copy(), y0.copy(), z0.copy()]
            for ax in range(d):
                weight *= a[ax] if b[ax] else 1.0 - a[ax]
                c[ax] = c[ax] - b[ax] * int(s[ax])
            inside = np.ones(len(z0), dtype=bool)
            for ax in range(3):
                if lat.bc[ax] == PERIODIC:
                    c[ax] = np.mod(c[ax], ext[ax])
                else:
                    inside &= (c[ax] >= 0) & (c[ax] < ext[ax])
                    c[ax] = np.clip(c[ax], 0, ext[ax] - 1)
            vals = value_at(i, c[2], c[1], c[0])
            out[i] += weight * np.where(inside, vals, 0.0)
    return out


# ----------------------------------------------------------------------------
# 2. moments
# ----------------------------------------------------------------------------

def moments(I, lat):
    """E = sum I_i, F^a = sum n^a I_i, P^ab = sum n^a n^b I_i over the first
    axis of I.  Returns E, F (d, ...), P (d, d, ...)."""
    d = lat.dims
    n = lat.n[:, :d]
    E = I.sum(axis=0)
    F = np.tensordot(n.T, I, axes=(1, 0))
    P = np.tensordot(np.einsum("ia,ib->abi", n, n), I, axes=(2, 0))
    return E, F, P


def _field(x, shape):
    return np.broadcast_to(np.asarray(x, dtype=np.float64), shape)


def _ndot(n, F):
    """n_i . F for every direction and site: shape (N, ...)."""
    return np.tensordot(n, F, axes=(1, 0))


def _wcol(w, ndim):
    return w.reshape((-1,) + (1,) * ndim)


# ----------------------------------------------------------------------------
# 3. collisions
# ----------------------------------------------------------------------------

def collide_explicit(Is, lat, co):
    """Eq. (collision-step): I = I* - kappa_0 dt (I* - I^eq) + dt S with the
    moments taken from I*."""
    site = Is.shape[1:]
    d, dt = lat.dims, lat.dt
    ka, k0, lam, eta = (_field(x, site) for x in (co.kappa_a, co.kappa_0, co.lam, co.eta))
    E, F, _ = moments(Is, lat)
    w = _wcol(lat.w, len(site))
    Ieq = w * (E + lam * _ndot(lat.n[:, :d], F))
    S = w * eta - ka * Is
    return Is - k0 * dt * (Is - Ieq) + dt * S


def implicit_moments(Is, lat, co):
    """New (E, F) of Eq. (rte_implicit), solved exactly.

    With A = 1 / (1 + dt (kappa_0 + kappa_a)) every direction obeys
        I_i = A [I*_i + dt w_i eta + dt kappa_0 w_i (E + lambda n_i.F)],
    and summing with weights 1 and n_i gives
        (Id - A dt kappa_0 M) [E; F] = A [E*; F*] + A dt eta [T0; T1],
    M = [[T0, lambda T1^T], [T1, lambda T2]]."""
    site = Is.shape[1:]
    d, dt = lat.dims, lat.dt
    ka, k0, lam, eta = (_field(x, site) for x in (co.kappa_a, co.kappa_0, co.lam, co.eta))
    T0, T1, T2 = lat.table_sums()
    Es, Fs, _ = moments(Is, lat)
    A = 1.0 / (1.0 + dt * (k0 + ka))
    S = int(np.prod(site)) if site else 1
    M = np.zeros((S, d + 1, d + 1))
    lam_f = lam.reshape(S)
    M[:, 0, 0] = T0
    M[:, 0, 1:] = lam_f[:, None] * T1[None, :]
    M[:, 1:, 0] = T1[None, :]
    M[:, 1:, 1:] = lam_f[:, None, None] * T2[None, :, :]
    c = (A * dt * k0).reshape(S)
    mat = np.eye(d + 1)[None] - c[:, None, None] * M
    rhs = np.empty((S, d + 1))
    rhs[:, 0] = (A * (Es + dt * eta * T0)).reshape(S)
    rhs[:, 1:] = (A[None] * (Fs + dt * eta[None] * T1.reshape((d,) + (1,) * len(site)))).reshape(d, S).T
    sol = np.linalg.solve(mat, rhs[..., None])[..., 0]
    E = sol[:, 0].reshape(site)
    F = sol[:, 1:].T.reshape((d,) + site)
    return E, F


def _implicit_populations(Is, lat, co, E, F):
    site = Is.shape[1:]
    d, dt = lat.dims, lat.dt
    ka, k0, lam, eta = (_field(x, site) for x in (co.kappa_a, co.kappa_0, co.lam, co.eta))
    A = 1.0 / (1.0 + dt * (k0 + ka))
    w = _wcol(lat.w, len(site))
    return A * (Is + dt * w * eta + dt * k0 * w * (E + lam * _ndot(lat.n[:, :d], F)))


def collide_implicit(Is, lat, co):
    """Exact solution of Eq. (rte_implicit)."""
    E, F = implicit_moments(Is, lat, co)
    return _implicit_populations(Is, lat, co, E, F)


def collide_lambda(Is, lat, co, tol=1e-14, max_iter=100000, cycles=None):
    """Literal Lambda iteration of Sec. 3.3.  Starts from the moments of I*,
    solves the decoupled per-direction equations, recomputes (E, F) and
    repeats.  With `cycles` set, runs exactly that many passes (the paper's
    timing runs fix five); otherwise stops at convergence.
    Returns (I, number of passes)."""
    E, F, _ = moments(Is, lat)
    it = 0
    while True:
        it += 1
        I = _implicit_populations(Is, lat, co, E, F)
        En, Fn, _ = moments(I, lat)
        dE = np.abs(En - E)
        dF = np.abs(Fn - F).max(axis=0)
        scale = np.abs(En)
        E, F = En, Fn
        if cycles is not None:
            if it >= cycles:
                return I, it
            continue
        if np.all((dE <= tol * scale) & (dF <= tol * scale)):
            return I, it
        if it >= max_iter:
            raise RuntimeError("Lambda iteration did not converge")


def _moving_terms(Is, lat, mo):
    """Per-site W and per-direction beta_i, A_i, D_i of the mixed-frame
    equation (App. B)."""
    site = Is.shape[1:]
    v = np.asarray(mo.v, dtype=np.float64).reshape((3,) + site)
    kt_a, kt_0, eta_t = (_field(x, site) for x in (mo.kt_a, mo.kt_0, mo.eta_t))
    W = 1.0 / np.sqrt(1.0 - (v ** 2).sum(axis=0))
    beta = 1.0 - _ndot(lat.n, v)                      # (N, ...)
    A = 1.0 / (1.0 + lat.dt * W * beta * (kt_a + kt_0))
    D = 1.0 / (W * beta) ** 3
    return W, beta, A, D, kt_a, kt_0, eta_t


def moving_J(Is, lat, mo):
    """Exact fluid-frame J at the new time level.  Each direction obeys
        I_i = A_i [I*_i + dt w_i D_i (eta_t + kt_0 J)],  J = W^2 sum beta_i^2 I_i,
    so J = X / (1 - Y) with X = W^2 sum beta_i^2 A_i (I*_i + dt w_i D_i eta_t)
    and Y = dt kt_0 W^2 sum beta_i^2 A_i w_i D_i."""
    W, beta, A, D, kt_a, kt_0, eta_t = _moving_terms(Is, lat, mo)
    w = _wcol(lat.w, Is.ndim - 1)
    dt = lat.dt
    X = W ** 2 * (beta ** 2 * A * (Is + dt * w * D * eta_t)).sum(axis=0)
    Y = dt * kt_0 * W ** 2 * (beta ** 2 * A * w * D).sum(axis=0)
    return X / (1.0 - Y)


def _moving_populations(Is, lat, mo, J):
    W, beta, A, D, kt_a, kt_0, eta_t = _moving_terms(Is, lat, mo)
    w = _wcol(lat.w, Is.ndim - 1)
    return A * (Is + lat.dt * w * D * (eta_t + kt_0 * J))


def collide_moving(Is, lat, mo):
    """Exact implicit solution of the mixed-frame equation (App. B)."""
    return _moving_populations(Is, lat, mo, moving_J(Is, lat, mo))


def collide_moving_lambda(Is, lat, mo, tol=1e-14, max_iter=100000):
    """Literal Lambda iteration on J for the mixed-frame equation; initial
    guess J from I*.  Returns (I, passes)."""
    W, beta, *_ = _moving_terms(Is, lat, mo)
    J = W ** 2 * (beta ** 2 * Is).sum(axis=0)
    it = 0
    while True:
        it += 1
        I = _moving_populations(Is, lat, mo, J)
        Jn = W ** 2 * (beta ** 2 * I).sum(axis=0)
        done = np.all(np.abs(Jn - J) <= tol * np.abs(Jn))
        J = Jn
        if done:
            return I, it
        if it >= max_iter:
            raise RuntimeError("Lambda iteration did not converge")


# ----------------------------------------------------------------------------
# 4. one full step
# ----------------------------------------------------------------------------

@dataclass
class Frozen:
    """Cells whose populations are prescribed after every collision."""
    cells: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), dtype=np.int64))  # (z, y, x)
    values: np.ndarray = field(default_factory=lambda: np.zeros((0, 0)))                  # (ncells, N)


def collide(Is, lat, co, collision="implicit", lambda_cycles=None):
    if isinstance(co, Moving):
        if collision != "implicit":
            raise ValueError("moving fluid: implicit collision only")
        return collide_moving(Is, lat, co)
    if collision == "implicit":
        return collide_implicit(Is, lat, co)
    if collision == "explicit":
        return collide_explicit(Is, lat, co)
    if collision == "lambda":
        return collide_lambda(Is, lat, co, cycles=lambda_cycles)[0]
    raise ValueError(collision)


def step(I, lat, co, collision="implicit", frozen=None, lambda_cycles=None, budget=None):
    """I^n -> I^{n+1}.  If `budget` is a dict, adds the FP64 energy terms of
    this step: outflow = sum E^n - sum E*, source = sum (E_coll - E*),
    injection = sum over frozen cells of (prescribed - collided) energy."""
    Is = stream(I, lat)
    Inew = collide(Is, lat, co, collision, lambda_cycles)
    if budget is not None:
        e_n, e_s, e_c = I.sum(), Is.sum(), Inew.sum()
        budget["outflow"] = budget.get("outflow", 0.0) + (e_n - e_s)
        budget["source"] = budget.get("source", 0.0) + (e_c - e_s)
    if frozen is not None and len(frozen.cells):
        z, y, x = frozen.cells.T
        if budget is not None:
            budget["injection"] = budget.get("injection", 0.0) + (
                frozen.values.sum() - Inew[:, z, y, x].sum())
        Inew[:, z, y, x] = frozen.values.T
    return Inew


def run(I, lat, co, nsteps, **kw):
    for _ in range(nsteps):
        I = step(I, lat, co, **kw)
    return I


# ----------------------------------------------------------------------------
# initial states
# ----------------------------------------------------------------------------

def isotropic(E0, lat):
    """I_i = w_i E0 (Sec. 4.2.2 and 4.2.3 initial data)."""
    return _wcol(lat.w, E0.ndim) * E0[None]


def p1_state(E0, F0, lat):
    """I_i = w_i (E0 + d n_i.F0): the populations whose moments are (E0, F0)
    for an isotropic table."""
    d = lat.dims
    return _wcol(lat.w, E0.ndim) * (E0[None] + d * _ndot(lat.n[:, :d], F0[:d]))
