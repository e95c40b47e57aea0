"""Batched problems (lb_rt_batch_*): many independent static problems of
uneven size and direction count advanced by one persistent launch per
direction group and step, or one launch per step for a 42- and a
162-direction group together (pair_groups), with the tile shape chosen by
the autotuner.  Each result must equal the problem run alone (bit for bit:
its tiles depend only on its own data), the single-problem library path,
and the FP64 oracle within the storage's tolerance."""
import numpy as np
import pytest

from paper_2007_05718_gb300 import lbrt
from paper_2007_05718_gb300 import workloads as W
from parity import TOL_F32, Problem, oracle_run, pad_F, rel_l2

pytestmark = pytest.mark.gpu

TOL = {lbrt.LB_RT_F32: TOL_F32, lbrt.LB_RT_F16_DEV: 2e-3}
STORAGES = [pytest.param(lbrt.LB_RT_F32, id="fp32"), pytest.param(lbrt.LB_RT_F16_DEV, id="fp16")]


def _sphere(n, level, kappa_r, nsteps, shape=None):
    """A radiating sphere on n^3, or (with `shape`) a ragged box with smooth
    E and random absorption/emission; vacuum faces."""
    shape = shape or (n, n, n)
    if shape == (n, n, n):
        sp = W.radiating_sphere(n, kappa_r)
        E0, ka, eta = sp["E0"], sp["kappa_a"], sp["eta"]
    else:
        E0 = (0.5 + 0.5 * W.smooth_field(shape, 3)).astype(np.float32)
        ka = W.random_fields(shape, 4, 0.0, 20.0)
        eta = W.random_fields(shape, 5, 0.0, 20.0)
    nz, ny, nx = shape
    return dict(problem=dict(dims=3, nx=nx, ny=ny, nz=nz, dirset=lbrt.LB_RT_ICOSPHERE, level=level,
                             cfl=0.5, bc=(lbrt.LB_RT_VACUUM,) * 3),
                fluid=dict(kappa_a=ka, eta=eta), state=E0, nsteps=nsteps, shape=shape)


def _run_batch(reqs, storage, steps_per_tick=4, use_graph=True, autotune=True, mem_budget=0,
               pair_groups=0, plans=None):
    """Run `reqs` to completion in one batch; `plans` (a list) receives, per
    tick, each slot's (directions per warp, planes per batch, paired)."""
    b = lbrt.lb_rt_batch_create(max_problems=16, storage=storage, steps_per_tick=steps_per_tick,
                                use_graph=use_graph, autotune=autotune, mem_budget=mem_budget,
                                pair_groups=pair_groups)
    out = []
    try:
        slots = [lbrt.lb_rt_batch_admit(b, r["problem"], r["fluid"], r["state"],
                                        lbrt.LB_RT_STATE_ISOTROPIC, r["nsteps"]) for r in reqs]
        assert all(s is not None for s in slots)
        for _ in range(10000):
            if lbrt.lb_rt_batch_tick(b) == 0:
                break
            if plans is not None:
                plans.append([lbrt.lb_rt_batch_plan(b, s) for s in slots])
        lbrt.lb_rt_batch_sync(b)
        assert sorted(lbrt.lb_rt_batch_poll(b)) == sorted(slots)
        for r, s in zip(reqs, slots):
            S = int(np.prod(r["shape"]))
            E = np.zeros(S, dtype=np.float32)
            F = np.zeros((3, S), dtype=np.float32)
            lbrt.lb_rt_batch_moments(b, s, E, F)
            assert lbrt.lb_rt_batch_steps(b, s) == r["nsteps"]
            z, c = lbrt.lb_rt_batch_tuning(b, s)
            assert z in (8, 16, 32, 64) and c >= 1
            out.append((E, F))
    finally:
        lbrt.lb_rt_batch_destroy(b)
    return out


def _single(r, storage):
    p = r["problem"]
    h = lbrt.lb_rt_create(p["dims"], p["nx"], p["ny"], p["nz"], dirset=p["dirset"], level=p["level"],
                          cfl=p["cfl"], bc=p["bc"], storage=storage)
    try:
        lbrt.lb_rt_set_fluid(h, **r["fluid"])
        lbrt.lb_rt_set_state(h, r["state"], lbrt.LB_RT_STATE_ISOTROPIC)
        lbrt.lb_rt_step(h, r["nsteps"])
        S = int(np.prod(r["shape"]))
        E = np.zeros(S, dtype=np.float32)
        F = np.zeros((3, S), dtype=np.float32)
        lbrt.lb_rt_moments(h, E, F)
        return E, F
    finally:
        lbrt.lb_rt_destroy(h)


def _mix():
    """Uneven sizes, both direction sets, step counts that are and are not
    multiples of the tick."""
    return [_sphere(32, 1, 10.0, 23), _sphere(48, 2, 1.0, 9), _sphere(0, 1, 0.0, 14, shape=(9, 20, 70)),
            _sphere(24, 2, 100.0, 17), _sphere(32, 1, 1.0, 4), _sphere(0, 2, 0.0, 11, shape=(6, 13, 33))]


@pytest.mark.parametrize("storage", STORAGES)
def test_batch_matches_alone_and_single_path(cuda, storage):
    reqs = _mix()
    mixed = _run_batch(reqs, storage)
    for r, (E, F) in zip(reqs, mixed):
        Ea, Fa = _run_batch([r], storage)[0]
        assert np.array_equal(E, Ea) and np.array_equal(F, Fa)   # alone == in the mix
        Es, Fs = _single(r, storage)
        assert np.array_equal(E, Es) and np.array_equal(F, Fs)   # batched == single-problem kernel


@pytest.mark.parametrize("storage", STORAGES)
def test_batch_against_oracle(cuda, storage):
    reqs = [_sphere(24, 1, 10.0, 30), _sphere(0, 2, 0.0, 8, shape=(7, 10, 19))]
    res = _run_batch(reqs, storage, steps_per_tick=7)
    for r, (E, F) in zip(reqs, res):
        p = r["problem"]
        prob = Problem(3, r["shape"], "ico", level=p["level"], bc="vvv", coef=dict(r["fluid"]),
                       state_kind=lbrt.LB_RT_STATE_ISOTROPIC, state=r["state"])
        Io, Eo, Fo, Po, bo, lat = oracle_run(prob, r["nsteps"])
        assert rel_l2(E.reshape(r["shape"]), Eo) <= TOL[storage]
        assert rel_l2(F.reshape((3,) + r["shape"]), pad_F(Fo, 3)) <= TOL[storage]


def test_graph_replay_equals_direct_launches(cuda):
    """Ticks replayed from captured graphs (the launch plan changes as
    problems run out of steps) give the direct launches' results."""
    reqs = _mix()[:4]
    a = _run_batch(reqs, lbrt.LB_RT_F16_DEV, use_graph=True, autotune=False)
    b = _run_batch(reqs, lbrt.LB_RT_F16_DEV, use_graph=False, autotune=False)
    for (Ea, Fa), (Eb, Fb) in zip(a, b):
        assert np.array_equal(Ea, Eb) and np.array_equal(Fa, Fb)


def test_admission_by_memory_and_release(cuda):
    r1 = _sphere(48, 2, 10.0, 5)
    r2 = _sphere(48, 2, 10.0, 5)
    b = lbrt.lb_rt_batch_create(max_problems=4, storage=lbrt.LB_RT_F16_DEV, steps_per_tick=5)
    try:
        need = lbrt.lb_rt_batch_problem_bytes(b, **r1["problem"])
        assert need > 0
    finally:
        lbrt.lb_rt_batch_destroy(b)
    # a budget for one problem and a half: the second waits for the first
    b = lbrt.lb_rt_batch_create(max_problems=4, storage=lbrt.LB_RT_F16_DEV, steps_per_tick=5,
                                mem_budget=int(need * 1.5))
    try:
        s1 = lbrt.lb_rt_batch_admit(b, r1["problem"], r1["fluid"], r1["state"],
                                    lbrt.LB_RT_STATE_ISOTROPIC, r1["nsteps"])
        assert s1 is not None
        assert lbrt.lb_rt_batch_admit(b, r2["problem"], r2["fluid"], r2["state"],
                                      lbrt.LB_RT_STATE_ISOTROPIC, r2["nsteps"]) is None
        lbrt.lb_rt_batch_tick(b)
        lbrt.lb_rt_batch_sync(b)
        assert lbrt.lb_rt_batch_poll(b) == [s1]
        lbrt.lb_rt_batch_release(b, s1)
        s2 = lbrt.lb_rt_batch_admit(b, r2["problem"], r2["fluid"], r2["state"],
                                    lbrt.LB_RT_STATE_ISOTROPIC, r2["nsteps"])
        assert s2 is not None
    finally:
        lbrt.lb_rt_batch_destroy(b)


def test_batch_rejects_unsupported_problems(cuda):
    b = lbrt.lb_rt_batch_create(max_problems=2, storage=lbrt.LB_RT_F32)
    try:
        r = _sphere(16, 1, 10.0, 3)
        p = dict(r["problem"], budget=True)
        with pytest.raises(lbrt.LBRTError):
            lbrt.lb_rt_batch_admit(b, p, r["fluid"], r["state"], lbrt.LB_RT_STATE_ISOTROPIC, 3)
        with pytest.raises(lbrt.LBRTError):
            lbrt.lb_rt_batch_moments(b, 1, np.zeros(8, dtype=np.float32))
    finally:
        lbrt.lb_rt_batch_destroy(b)


PAIR_STORAGES = [pytest.param(lbrt.LB_RT_F32, id="fp32"), pytest.param(lbrt.LB_RT_F16_DEV, id="fp16"),
                 pytest.param(lbrt.LB_RT_BF16_DEV, id="bf16")]


@pytest.mark.parametrize("storage", PAIR_STORAGES)
@pytest.mark.parametrize("pair_groups", [1, 2])
def test_paired_launch_equals_separate_launches(cuda, storage, pair_groups):
    """42- and 162-direction problems stepped in ONE launch per step (each CTA
    runs its own group's tile plan) give the bits of the separate launches;
    with pair_groups = 1 every tick with both groups active is paired."""
    reqs = _mix()
    plans = []
    # without the z-chunk tuner the first tick already pairs (the tuner
    # times groups one launch each, and retunes a group whose sites shrink)
    paired = _run_batch(reqs, storage, pair_groups=pair_groups, plans=plans, autotune=False)
    sep = _run_batch(reqs, storage, pair_groups=0)
    for (Ea, Fa), (Eb, Fb) in zip(paired, sep):
        assert np.array_equal(Ea, Eb) and np.array_equal(Fa, Fb)
    dpts = {p[0] for tick in plans for p in tick}
    assert len(dpts) == 2                                   # two tile plans in the batch
    if pair_groups == 1:
        assert all(p[2] == 1 for p in plans[0])



@pytest.mark.parametrize("storage", STORAGES)
def test_tuned_planes_per_batch_give_the_same_bits(cuda, storage):
    """The autotuner times the alternative batched kernel of the 42-direction
    plan (another number of planes per batch, same layout) after the z
    chunks; the tick that runs it, and whatever it keeps, give the bits of
    the single-problem path."""
    reqs = [_sphere(24, 1, 10.0, 40), _sphere(0, 1, 0.0, 40, shape=(11, 17, 40)),
            _sphere(20, 1, 1.0, 40)]
    plans = []
    res = _run_batch(reqs, storage, plans=plans)
    zcs = {p[1] for tick in plans for p in tick}
    assert len(zcs) == 2                        # both kernels ran (tick 4 times the other one)
    for r, (E, F) in zip(reqs, res):
        Es, Fs = _single(r, storage)
        assert np.array_equal(E, Es) and np.array_equal(F, Fs)
