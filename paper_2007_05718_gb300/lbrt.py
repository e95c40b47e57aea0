"""Thin ctypes binding of liblbrt.so (include/lb_rt.h).

Every function here has the name of the C entry point it calls and does
argument marshalling only: all arithmetic of the LB step runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA); float32 and C-contiguous are required.  A failing call raises
LBRTError with the library's message.  If the library is not built the first
call raises: there is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbrt.so")

# constants of include/lb_rt.h
LB_RT_OK, LB_RT_EINVAL, LB_RT_ENOMEM, LB_RT_ECUDA, LB_RT_ETIMEDOUT, LB_RT_ESTATE = 0, -1, -2, -3, -4, -5
LB_RT_EBUSY = -6
LB_RT_BATCH_MAX = 256
LB_RT_RING2D, LB_RT_ICOSPHERE, LB_RT_GAUSS_LEGENDRE = 1, 2, 3
LB_RT_PERIODIC, LB_RT_VACUUM = 0, 1
LB_RT_F32, LB_RT_F16_DEV, LB_RT_BF16_DEV = 0, 1, 2
LB_RT_IMPLICIT_EXACT, LB_RT_EXPLICIT, LB_RT_LAMBDA_K = 0, 1, 2
LB_RT_HOST, LB_RT_DEVICE, LB_RT_HOST_MAPPED = 0, 1, 2
LB_RT_STATE_POPULATIONS, LB_RT_STATE_ISOTROPIC, LB_RT_STATE_P1 = 0, 1, 2
LB_RT_MAX_DIRS = 192

EXPORTED = [
    "lb_rt_create", "lb_rt_set_fluid", "lb_rt_set_state", "lb_rt_set_frozen", "lb_rt_step",
    "lb_rt_moments", "lb_rt_get_populations", "lb_rt_state_bytes", "lb_rt_save_state",
    "lb_rt_restore_state", "lb_rt_sync", "lb_rt_directions", "lb_rt_enable_timing",
    "lb_rt_last_step_ms", "lb_rt_last_error", "lb_rt_version", "lb_rt_destroy",
    "lb_rt_total_energy_noalloc", "lb_rt_coupling", "lb_rt_step_moments",
    "lb_rt_batch_create", "lb_rt_batch_destroy", "lb_rt_batch_problem_bytes", "lb_rt_batch_admit",
    "lb_rt_batch_tick", "lb_rt_batch_sync", "lb_rt_batch_poll", "lb_rt_batch_moments",
    "lb_rt_batch_steps", "lb_rt_batch_release", "lb_rt_batch_tuning", "lb_rt_batch_last_error",
    "lb_rt_batch_plan",
]


class lb_rt_config(C.Structure):
    _fields_ = [
        ("dims", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ndir", C.c_int), ("dirs", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double)),
        ("dirset", C.c_int), ("dirset_param", C.c_int * 2), ("ring_offset", C.c_double),
        ("cfl", C.c_double), ("dx", C.c_double), ("bc", C.c_int * 3), ("storage", C.c_int),
        ("collision", C.c_int), ("lambda_iters", C.c_int), ("moving", C.c_int),
        ("budget", C.c_int), ("stream", C.c_void_p),
    ]


class lb_rt_fluid(C.Structure):
    _fields_ = [
        ("kappa_a", C.c_void_p), ("kappa_a_s", C.c_float),
        ("kappa_0", C.c_void_p), ("kappa_0_s", C.c_float),
        ("lambda_", C.c_void_p), ("lambda_s", C.c_float),
        ("eta", C.c_void_p), ("eta_s", C.c_float),
        ("v", C.c_void_p),
        ("kt_a", C.c_void_p), ("kt_a_s", C.c_float),
        ("kt_0", C.c_void_p), ("kt_0_s", C.c_float),
        ("eta_t", C.c_void_p), ("eta_t_s", C.c_float),
    ]


class lb_rt_batch_config(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_problems", C.c_int), ("storage", C.c_int),
                ("steps_per_tick", C.c_int), ("use_graph", C.c_int), ("autotune", C.c_int),
                ("stream", C.c_void_p), ("pair_groups", C.c_int)]


class lb_rt_budget(C.Structure):
    _fields_ = [("total", C.c_double), ("initial", C.c_double), ("outflow", C.c_double),
                ("source", C.c_double), ("injection", C.c_double), ("steps", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LBRTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lb_rt status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load(path=LIB_PATH):
    """Load liblbrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbrt.so is not built (%s); run paper_2007_05718_gb300.build.build()" % path)
    lib = C.CDLL(path)
    H = C.c_void_p
    sig = {
        "lb_rt_create": (C.c_int, [C.POINTER(lb_rt_config), C.POINTER(C.c_void_p)]),
        "lb_rt_set_fluid": (C.c_int, [H, C.POINTER(lb_rt_fluid), C.c_int]),
        "lb_rt_set_state": (C.c_int, [H, C.c_void_p, C.c_int, C.c_int]),
        "lb_rt_set_frozen": (C.c_int, [H, C.c_void_p, C.c_int, C.c_void_p]),
        "lb_rt_step": (C.c_int, [H, C.c_int]),
        "lb_rt_step_moments": (C.c_int, [H, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
        "lb_rt_moments": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(lb_rt_budget), C.c_int]),
        "lb_rt_get_populations": (C.c_int, [H, C.c_void_p, C.c_int]),
        "lb_rt_state_bytes": (C.c_size_t, [H]),
        "lb_rt_save_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "lb_rt_restore_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "lb_rt_sync": (C.c_int, [H]),
        "lb_rt_directions": (C.c_int, [H, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]),
        "lb_rt_enable_timing": (C.c_int, [H, C.c_int]),
        "lb_rt_last_step_ms": (C.c_int, [H, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
        "lb_rt_last_error": (C.c_char_p, [H]),
        "lb_rt_version": (C.c_char_p, []),
        "lb_rt_destroy": (None, [H]),
        "lb_rt_total_energy_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_void_p,
                                                 C.c_int, C.c_void_p]),
        "lb_rt_coupling": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
        "lb_rt_batch_create": (C.c_int, [C.POINTER(lb_rt_batch_config), C.POINTER(C.c_void_p)]),
        "lb_rt_batch_destroy": (None, [H]),
        "lb_rt_batch_problem_bytes": (C.c_size_t, [H, C.POINTER(lb_rt_config)]),
        "lb_rt_batch_admit": (C.c_int, [H, C.POINTER(lb_rt_config), C.POINTER(lb_rt_fluid), C.c_int,
                                        C.c_void_p, C.c_int, C.c_int, C.c_longlong,
                                        C.POINTER(C.c_int)]),
        "lb_rt_batch_tick": (C.c_int, [H, C.POINTER(C.c_int)]),
        "lb_rt_batch_sync": (C.c_int, [H]),
        "lb_rt_batch_poll": (C.c_int, [H, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
        "lb_rt_batch_moments": (C.c_int, [H, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
        "lb_rt_batch_steps": (C.c_int, [H, C.c_int, C.POINTER(C.c_longlong)]),
        "lb_rt_batch_release": (C.c_int, [H, C.c_int]),
        "lb_rt_batch_tuning": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lb_rt_batch_plan": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]),
        "lb_rt_batch_last_error": (C.c_char_p, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(h, st):
    if st != LB_RT_OK:
        msg = load().lb_rt_last_error(h)
        raise LBRTError(st, msg.decode() if msg else "")


def _ptr(x):
    """(pointer, ptr_kind) of a float32 contiguous numpy array or torch tensor."""
    if x is None:
        return None, LB_RT_HOST
    mod = type(x).__module__
    if mod.startswith("torch"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (LB_RT_DEVICE if x.is_cuda else LB_RT_HOST)
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be a C-contiguous numpy array")
    return x.ctypes.data, LB_RT_HOST


def _f32(x):
    if x is None:
        return None
    mod = type(x).__module__
    if mod.startswith("torch"):
        import torch
        if x.dtype != torch.float32:
            raise ValueError("float32 tensor required")
        return x
    import numpy as np
    return np.ascontiguousarray(x, dtype=np.float32)


def _kind_of(objs):
    kinds = {_ptr(o)[1] for o in objs if o is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else LB_RT_HOST


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def _make_config(dims, nx, ny, nz=1, *, dirset=LB_RT_ICOSPHERE, ndir=0, level=1, gl=(0, 0),
                 dirs=None, weights=None, ring_offset=0.0, cfl=0.5, dx=None,
                 bc=(LB_RT_PERIODIC,) * 3, storage=LB_RT_F32, collision=LB_RT_IMPLICIT_EXACT,
                 lambda_iters=1, moving=False, budget=False, stream=None):
    """lb_rt_config from keyword arguments; returns (config, arrays to keep alive)."""
    cfg = lb_rt_config()
    cfg.dims, cfg.nx, cfg.ny, cfg.nz = dims, nx, ny, nz
    keep = []
    if dirs is not None:
        import numpy as np
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        keep.append(d)
        cfg.ndir = len(d)
        cfg.dirs = d.ctypes.data_as(C.POINTER(C.c_double))
        if weights is not None:
            wv = np.ascontiguousarray(weights, dtype=np.float64)
            keep.append(wv)
            cfg.weights = wv.ctypes.data_as(C.POINTER(C.c_double))
    else:
        cfg.ndir = ndir
        cfg.dirset = dirset
        if dirset == LB_RT_ICOSPHERE:
            cfg.dirset_param[0] = level
        elif dirset == LB_RT_GAUSS_LEGENDRE:
            cfg.dirset_param[0], cfg.dirset_param[1] = gl
    cfg.ring_offset = ring_offset
    cfg.cfl = cfl
    cfg.dx = (1.0 / max(nx, 1)) if dx is None else dx
    for a in range(3):
        cfg.bc[a] = bc[a]
    cfg.storage, cfg.collision, cfg.lambda_iters = storage, collision, lambda_iters
    cfg.moving, cfg.budget = int(bool(moving)), int(bool(budget))
    cfg.stream = stream or None
    return cfg, keep


def lb_rt_create(dims, nx, ny, nz=1, **kw):
    """Create a handle (lb_rt_create); keywords as _make_config.  `stream` is
    a cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream)
    or None."""
    lib = load()
    cfg, keep = _make_config(dims, nx, ny, nz, **kw)
    h = C.c_void_p()
    _check(None, lib.lb_rt_create(C.byref(cfg), C.byref(h)))
    return h


def lb_rt_destroy(h):
    load().lb_rt_destroy(h)


def _make_fluid(kappa_a=0.0, kappa_0=0.0, lam=0.0, eta=0.0, v=None, kt_a=None, kt_0=None,
                eta_t=None):
    """lb_rt_fluid from scalars or float32 site fields; returns (fluid,
    pointer kind, arrays to keep alive)."""
    f = lb_rt_fluid()
    arrays = []

    def put(name, val):
        if val is None:
            return
        if isinstance(val, (int, float)):
            setattr(f, name + "_s", float(val))
            return
        a = _f32(val)
        arrays.append(a)
        setattr(f, name, _ptr(a)[0])

    for name, val in (("kappa_a", kappa_a), ("kappa_0", kappa_0), ("lambda", lam), ("eta", eta)):
        if name == "lambda":
            if isinstance(val, (int, float)):
                f.lambda_s = float(val)
            elif val is not None:
                a = _f32(val)
                arrays.append(a)
                f.lambda_ = _ptr(a)[0]
            continue
        put(name, val)
    if v is not None:
        a = _f32(v)
        arrays.append(a)
        f.v = _ptr(a)[0]
    put("kt_a", kt_a)
    put("kt_0", kt_0)
    put("eta_t", eta_t)
    return f, _kind_of(arrays), arrays


def lb_rt_set_fluid(h, kappa_a=0.0, kappa_0=0.0, lam=0.0, eta=0.0, v=None, kt_a=None,
                    kt_0=None, eta_t=None, mapped=False):
    """Scalars or float32 site fields [nz, ny, nx] (v: [3, nz, ny, nx]).
    mapped=True: the fields are page-locked host tensors that the kernels
    read in place (LB_RT_HOST_MAPPED); the caller keeps them alive and
    unchanged until the steps that use them have completed."""
    f, kind, keep = _make_fluid(kappa_a, kappa_0, lam, eta, v, kt_a, kt_0, eta_t)
    if mapped:
        if kind != LB_RT_HOST:
            raise ValueError("mapped fields must be host memory")
        kind = LB_RT_HOST_MAPPED
    _check(h, load().lb_rt_set_fluid(h, C.byref(f), kind))


def lb_rt_set_state(h, data, kind=LB_RT_STATE_POPULATIONS):
    a = _f32(data)
    p, pk = _ptr(a)
    _check(h, load().lb_rt_set_state(h, p, kind, pk))


def lb_rt_set_frozen(h, cells, values):
    import numpy as np
    c = np.ascontiguousarray(cells, dtype=np.int64)
    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(h, load().lb_rt_set_frozen(h, c.ctypes.data if len(c) else None, len(c),
                                      v.ctypes.data if len(c) else None))


def lb_rt_step(h, nsteps=1):
    _check(h, load().lb_rt_step(h, nsteps))


def lb_rt_moments(h, E=None, F=None, P=None, budget=False):
    """Fill the given outputs (E [sites], F [3, sites], P [6, sites]); returns
    the budget dict when budget=True."""
    kind = _kind_of([E, F, P])
    b = lb_rt_budget()
    _check(h, load().lb_rt_moments(h, _ptr(E)[0], _ptr(F)[0], _ptr(P)[0],
                                   C.byref(b) if budget else None, kind))
    return b.as_dict() if budget else None


def lb_rt_step_moments(h, nsteps, E=None, F=None):
    """Advance nsteps and fill E [sites], F [3, sites] of the new state from
    the last step's collision (lb_rt_step_moments)."""
    kind = _kind_of([E, F])
    _check(h, load().lb_rt_step_moments(h, int(nsteps), _ptr(E)[0], _ptr(F)[0], kind))


def lb_rt_coupling(h, J=None, H=None, S=None):
    """Comoving J [sites], H [3, sites] and the four-force S [4, sites]."""
    kind = _kind_of([J, H, S])
    _check(h, load().lb_rt_coupling(h, _ptr(J)[0], _ptr(H)[0], _ptr(S)[0], kind))


def lb_rt_get_populations(h, out):
    p, pk = _ptr(out)
    _check(h, load().lb_rt_get_populations(h, p, pk))


def lb_rt_state_bytes(h):
    return int(load().lb_rt_state_bytes(h))


def lb_rt_save_state(h):
    n = lb_rt_state_bytes(h)
    buf = C.create_string_buffer(n)
    _check(h, load().lb_rt_save_state(h, buf, n))
    return buf.raw


def lb_rt_restore_state(h, raw):
    buf = C.create_string_buffer(raw, len(raw))
    _check(h, load().lb_rt_restore_state(h, buf, len(raw)))


def lb_rt_sync(h):
    _check(h, load().lb_rt_sync(h))


def lb_rt_directions(h):
    """(dirs [N, 3] float64, weights [N], signs [N, 3] int8) in library order."""
    import numpy as np
    n = C.c_int()
    _check(h, load().lb_rt_directions(h, C.byref(n), None, None, None))
    d = np.zeros((n.value, 3))
    w = np.zeros(n.value)
    s = np.zeros((n.value, 3), dtype=np.int8)
    _check(h, load().lb_rt_directions(h, C.byref(n), d.ctypes.data, w.ctypes.data, s.ctypes.data))
    return d, w, s


def lb_rt_enable_timing(h, on=True):
    _check(h, load().lb_rt_enable_timing(h, int(bool(on))))


def lb_rt_last_step_ms(h):
    ms, n = C.c_float(), C.c_int()
    _check(h, load().lb_rt_last_step_ms(h, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def lb_rt_last_error(h):
    m = load().lb_rt_last_error(h)
    return m.decode() if m else ""


def lb_rt_version():
    return load().lb_rt_version().decode()


def lb_rt_total_energy_noalloc(pop, ndir, sites, out=None, stream=None):
    """FP64 total energy of a dense device population array [ndir][sites]
    without any allocation inside the library.  With out=None the result is
    returned as a Python float (host output); otherwise `out` is a float64
    CUDA tensor of one element that receives it on the device."""
    # every check comes before the C call: a wrong dtype or a short tensor
    # would make the reduction kernel read or write past the allocation
    if not type(pop).__module__.startswith("torch"):
        raise ValueError("populations must be a CUDA tensor")
    import torch
    if pop.dtype != torch.float32:
        raise ValueError("populations must be float32")
    if not pop.is_contiguous():
        raise ValueError("populations must be contiguous")
    if int(ndir) < 1 or int(sites) < 1:
        raise ValueError("ndir and sites must be >= 1")
    if pop.numel() < int(ndir) * int(sites):
        raise ValueError("populations hold %d values, fewer than ndir x sites = %d"
                         % (pop.numel(), int(ndir) * int(sites)))
    if out is not None:
        if not type(out).__module__.startswith("torch"):
            raise ValueError("out must be a CUDA tensor")
        if out.dtype != torch.float64 or out.numel() < 1 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of at least one element")
        if not out.is_cuda:
            raise ValueError("out must be a CUDA tensor")
    p, pk = _ptr(pop)
    if pk != LB_RT_DEVICE:
        raise ValueError("populations must be a CUDA tensor")
    lib = load()
    if out is None:
        res = C.c_double()
        _check(None, lib.lb_rt_total_energy_noalloc(p, ndir, sites, C.byref(res), LB_RT_HOST,
                                                    stream or None))
        return res.value
    op, ok = _ptr(out)
    if ok != LB_RT_DEVICE:
        raise ValueError("out must be a CUDA tensor")
    _check(None, lib.lb_rt_total_energy_noalloc(p, ndir, sites, op, LB_RT_DEVICE, stream or None))
    return out


# ---- batch (many resident problems, one persistent launch per group) ----

def _bcheck(b, st):
    if st != LB_RT_OK:
        msg = load().lb_rt_batch_last_error(b)
        raise LBRTError(st, msg.decode() if msg else "")


def lb_rt_batch_create(*, max_problems=64, storage=LB_RT_F16_DEV, steps_per_tick=10,
                       mem_budget=0, use_graph=True, autotune=True, stream=None, pair_groups=0):
    """pair_groups: 0 one launch per group and step, 1 two groups of different
    direction counts share one launch per step where a paired kernel exists,
    2 the autotuner chooses."""
    cfg = lb_rt_batch_config()
    cfg.mem_budget, cfg.max_problems, cfg.storage = mem_budget, max_problems, storage
    cfg.steps_per_tick, cfg.use_graph, cfg.autotune = steps_per_tick, int(use_graph), int(autotune)
    cfg.stream = stream or None
    cfg.pair_groups = int(pair_groups)
    b = C.c_void_p()
    st = load().lb_rt_batch_create(C.byref(cfg), C.byref(b))
    if st != LB_RT_OK:
        raise LBRTError(st, "lb_rt_batch_create failed")
    return b


def lb_rt_batch_destroy(b):
    load().lb_rt_batch_destroy(b)


def lb_rt_batch_problem_bytes(b, dims, nx, ny, nz=1, **kw):
    cfg, keep = _make_config(dims, nx, ny, nz, **kw)
    return int(load().lb_rt_batch_problem_bytes(b, C.byref(cfg)))


def lb_rt_batch_admit(b, problem, fluid, state, state_kind, nsteps):
    """problem: keyword dict for _make_config (dims, nx, ny, nz, ...);
    fluid: keyword dict for _make_fluid.  Returns the slot, or None when the
    problem does not fit now (LB_RT_EBUSY)."""
    p = dict(problem)
    cfg, keep = _make_config(p.pop("dims"), p.pop("nx"), p.pop("ny"), p.pop("nz", 1), **p)
    f, fkind, fkeep = _make_fluid(**fluid)
    a = _f32(state)
    sp, skind = _ptr(a)
    slot = C.c_int(-1)
    st = load().lb_rt_batch_admit(b, C.byref(cfg), C.byref(f), fkind, sp, state_kind, skind,
                                  int(nsteps), C.byref(slot))
    if st == LB_RT_EBUSY:
        return None
    _bcheck(b, st)
    return slot.value


def lb_rt_batch_tick(b):
    n = C.c_int(0)
    _bcheck(b, load().lb_rt_batch_tick(b, C.byref(n)))
    return n.value


def lb_rt_batch_sync(b):
    _bcheck(b, load().lb_rt_batch_sync(b))


def lb_rt_batch_poll(b, max_slots=LB_RT_BATCH_MAX):
    arr = (C.c_int * max_slots)()
    n = C.c_int(0)
    _bcheck(b, load().lb_rt_batch_poll(b, arr, max_slots, C.byref(n)))
    return [arr[i] for i in range(n.value)]


def lb_rt_batch_moments(b, slot, E=None, F=None, P=None):
    kind = _kind_of([E, F, P])
    _bcheck(b, load().lb_rt_batch_moments(b, slot, _ptr(E)[0], _ptr(F)[0], _ptr(P)[0], kind))


def lb_rt_batch_steps(b, slot):
    n = C.c_longlong(0)
    _bcheck(b, load().lb_rt_batch_steps(b, slot, C.byref(n)))
    return n.value


def lb_rt_batch_release(b, slot):
    _bcheck(b, load().lb_rt_batch_release(b, slot))


def lb_rt_batch_tuning(b, slot):
    z = C.c_int(0)
    c = C.c_int(0)
    _bcheck(b, load().lb_rt_batch_tuning(b, slot, C.byref(z), C.byref(c)))
    return z.value, c.value


def lb_rt_batch_plan(b, slot):
    """(directions per warp, planes per batch, paired) of the group of `slot`."""
    d, z, p = C.c_int(0), C.c_int(0), C.c_int(0)
    _bcheck(b, load().lb_rt_batch_plan(b, slot, C.byref(d), C.byref(z), C.byref(p)))
    return d.value, z.value, p.value


def lb_rt_batch_last_error(b):
    m = load().lb_rt_batch_last_error(b)
    return m.decode() if m else ""

