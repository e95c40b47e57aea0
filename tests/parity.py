"""Helpers for the GPU-vs-oracle parity tests: one problem description runs
through the CUDA library (via the C ABI binding) and through the FP64 oracle
on the same seeded float32 inputs."""
import math
from dataclasses import dataclass, field

import numpy as np

from oracle import directions as OD
from oracle import lb as OL
from paper_2007_05718_gb300 import lbrt

BC = {"p": lbrt.LB_RT_PERIODIC, "v": lbrt.LB_RT_VACUUM}
OBC = {"p": OL.PERIODIC, "v": OL.VACUUM}
COLL = {"implicit": lbrt.LB_RT_IMPLICIT_EXACT, "explicit": lbrt.LB_RT_EXPLICIT,
        "lambda": lbrt.LB_RT_LAMBDA_K}


@dataclass
class Problem:
    dims: int
    shape: tuple                     # (nz, ny, nx)
    dirset: str = "ico"              # ico | ring | gl
    level: int = 1
    ndir: int = 16
    ring_offset: float = 0.0
    gl: tuple = (4, 8)
    cfl: float = 0.5
    bc: str = "ppp"                  # per axis x, y, z
    collision: str = "implicit"
    lambda_iters: int = 1
    storage: int = lbrt.LB_RT_F32
    coef: dict = field(default_factory=dict)    # kappa_a, kappa_0, lam, eta (scalar or array)
    moving: dict = None                         # v, kt_a, kt_0, eta_t
    state_kind: int = lbrt.LB_RT_STATE_POPULATIONS
    state: np.ndarray = None
    frozen: tuple = None                        # (cells [k] linear, values [k, N])
    budget: bool = False

    @property
    def dx(self):
        return 1.0 / self.shape[2]

    def oracle_dirs(self):
        if self.dirset == "ico":
            return OD.icosphere(self.level)
        if self.dirset == "ring":
            return OD.ring2d(self.ndir, self.ring_offset)
        return OD.gauss_legendre_product(*self.gl)

    def lattice(self):
        n, w = self.oracle_dirs()
        return OL.Lattice(self.dims, self.shape, n, w, self.cfl, self.dx,
                          tuple(OBC[c] for c in self.bc))


def make_handle(p, stream=None):
    nz, ny, nx = p.shape
    kw = dict(cfl=p.cfl, dx=p.dx, bc=tuple(BC[c] for c in p.bc), storage=p.storage,
              collision=COLL[p.collision], lambda_iters=p.lambda_iters,
              moving=p.moving is not None, budget=p.budget, stream=stream)
    if p.dirset == "ico":
        kw.update(dirset=lbrt.LB_RT_ICOSPHERE, level=p.level)
    elif p.dirset == "ring":
        kw.update(dirset=lbrt.LB_RT_RING2D, ndir=p.ndir, ring_offset=p.ring_offset)
    else:
        kw.update(dirset=lbrt.LB_RT_GAUSS_LEGENDRE, gl=p.gl)
    h = lbrt.lb_rt_create(p.dims, nx, ny, nz, **kw)
    if p.moving is not None:
        lbrt.lb_rt_set_fluid(h, **p.moving)
    else:
        c = dict(kappa_a=0.0, kappa_0=0.0, lam=0.0, eta=0.0)
        c.update(p.coef)
        lbrt.lb_rt_set_fluid(h, **c)
    lbrt.lb_rt_set_state(h, p.state, p.state_kind)
    if p.frozen is not None:
        lbrt.lb_rt_set_frozen(h, p.frozen[0], p.frozen[1])
    return h


def gpu_run(p, steps, keep_handle=False):
    """Returns (I [N, nz, ny, nx], E, F [3, ...], P [6, ...]) as float64 numpy."""
    h = make_handle(p)
    try:
        lbrt.lb_rt_step(h, steps)
        lbrt.lb_rt_sync(h)
        nz, ny, nx = p.shape
        S = nz * ny * nx
        N = lbrt.lb_rt_directions(h)[0].shape[0]
        I = np.zeros((N, S), dtype=np.float32)
        lbrt.lb_rt_get_populations(h, I)
        E = np.zeros(S, dtype=np.float32)
        F = np.zeros((3, S), dtype=np.float32)
        P = np.zeros((6, S), dtype=np.float32)
        budget = lbrt.lb_rt_moments(h, E, F, P, budget=True)
        out = (I.reshape((N,) + p.shape).astype(np.float64), E.reshape(p.shape).astype(np.float64),
               F.reshape((3,) + p.shape).astype(np.float64), P.reshape((6,) + p.shape).astype(np.float64))
        if keep_handle:
            return out + (budget, h)
        return out + (budget,)
    finally:
        if not keep_handle:
            lbrt.lb_rt_destroy(h)


def oracle_initial(p, lat):
    s = np.asarray(p.state, dtype=np.float64)
    if p.state_kind == lbrt.LB_RT_STATE_POPULATIONS:
        return s.reshape((lat.N,) + p.shape).copy()
    if p.state_kind == lbrt.LB_RT_STATE_ISOTROPIC:
        return OL.isotropic(s.reshape(p.shape), lat)
    s = s.reshape((4,) + p.shape)
    return OL.p1_state(s[0], s[1:], lat)


def oracle_coef(p):
    if p.moving is not None:
        m = {k: (np.asarray(v, dtype=np.float64) if not isinstance(v, (int, float)) else v)
             for k, v in p.moving.items() if v is not None}
        v = m.pop("v", None)
        if v is None:
            v = np.zeros((3,) + p.shape)
        return OL.Moving(v=v, kt_a=m.get("kt_a", 0.0), kt_0=m.get("kt_0", 0.0),
                         eta_t=m.get("eta_t", 0.0))
    c = {k: (np.asarray(v, dtype=np.float64) if not isinstance(v, (int, float)) else float(v))
         for k, v in p.coef.items()}
    return OL.Static(kappa_a=c.get("kappa_a", 0.0), kappa_0=c.get("kappa_0", 0.0),
                     lam=c.get("lam", 0.0), eta=c.get("eta", 0.0))


def oracle_run(p, steps):
    lat = p.lattice()
    I = oracle_initial(p, lat)
    co = oracle_coef(p)
    fz = None
    if p.frozen is not None:
        cells = np.asarray(p.frozen[0], dtype=np.int64)
        nz, ny, nx = p.shape
        zyx = np.stack([cells // (ny * nx), (cells // nx) % ny, cells % nx], axis=1)
        fz = OL.Frozen(cells=zyx, values=np.asarray(p.frozen[1], dtype=np.float64))
    budget = {}
    for _ in range(steps):
        I = OL.step(I, lat, co, collision=p.collision,
                    lambda_cycles=p.lambda_iters if p.collision == "lambda" else None,
                    frozen=fz, budget=budget)
    E, F, P = OL.moments(I, lat)
    return I, E, F, P, budget, lat


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def pad_F(F, dims):
    """Oracle F has d components; the library returns 3."""
    if F.shape[0] == 3:
        return F
    out = np.zeros((3,) + F.shape[1:])
    out[:dims] = F
    return out


def sym6(P, dims):
    """Oracle P (d, d, ...) -> library order xx, xy, xz, yy, yz, zz."""
    out = np.zeros((6,) + P.shape[2:])
    idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for k, (a, b) in enumerate(idx):
        if a < dims and b < dims:
            out[k] = P[a, b]
    return out


TOL_F32 = 1e-5   # relative L2 on E and F for float32 populations
