"""Pins for the oracle's pull-streaming (Eqs. rte-stream-collide, interp)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import directions as D
from oracle import lb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def _binom_pmf(n, a):
    return np.array([math.comb(n, j) * a ** j * (1 - a) ** (n - j) for j in range(n + 1)])


def test_pulse_binomial_closed_form_2d():
    """2D, 64^2 periodic, ring-16 rotated by 30 degrees, cfl 0.5, vacuum
    coefficients: a pulse I_0 = 1 at cell (x=0, y=32) after n steps is the
    product of two binomial distributions Binom(n, cfl cos 30) in x and
    Binom(n, cfl sin 30) in y, wrapped mod 64; every other direction stays 0."""
    n_steps, L = 200, 64
    n, w = D.ring2d(16, math.pi / 6)
    lat = lb.Lattice(2, (1, L, L), n, w, cfl=0.5, dx=1.0 / L)
    I = np.zeros((16, 1, L, L))
    I[0, 0, 32, 0] = 1.0
    I = lb.run(I, lat, lb.Static(), n_steps)
    ax, ay = 0.5 * math.cos(math.pi / 6), 0.5 * math.sin(math.pi / 6)
    px, py = _binom_pmf(n_steps, ax), _binom_pmf(n_steps, ay)
    expect = np.zeros((L, L))
    jy, jx = np.meshgrid(np.arange(n_steps + 1), np.arange(n_steps + 1), indexing="ij")
    np.add.at(expect, ((32 + jy) % L, jx % L), np.outer(py, px))
    assert np.abs(I[0, 0] - expect).max() < 1e-13
    assert np.abs(I[1:]).max() == 0.0
    assert abs(I.sum() - 1.0) < 1e-13
    # centroid (circular mean) moves by n cfl n_hat = (86.603, 50.000) cells
    E = I[0, 0]
    ang = 2 * math.pi * np.arange(L) / L
    cx = np.angle(np.sum(E.sum(0) * np.exp(1j * ang))) * L / (2 * math.pi) % L
    # binomial mean is exactly n a; its circular mean differs by O(variance/L^2)
    assert abs(cx - (n_steps * ax) % L) < 0.05


def test_cfl1_axis_shift_is_exact():
    facts = json.load(open(GOLDEN))["cfl1_axis_shift"]
    L = 32
    n, w = D.ring2d(8, 0.0)
    lat = lb.Lattice(2, (1, L, L), n, w, cfl=facts["cfl"], dx=1.0 / L,
                     bc=(lb.VACUUM, lb.PERIODIC, lb.PERIODIC))
    rng = np.random.default_rng(1)
    I = np.zeros((8, 1, L, L))
    I[0, 0] = rng.random((L, L))          # direction 0 = +x
    I[2, 0] = rng.random((L, L))          # direction 2 = +y
    I0 = I.copy()
    k = 5
    I = lb.run(I, lat, lb.Static(), k)
    assert np.array_equal(I[0, 0, :, k:], I0[0, 0, :, :-k])
    assert np.all(I[0, 0, :, :k] == 0.0)          # vacuum inflow
    assert np.array_equal(I[2, 0], np.roll(I0[2, 0], k, axis=0))


def test_single_corner_weights_3d():
    """A unit value streamed one step along a 3D direction lands on the
    eight downwind cells with weights prod_a (a_a or 1 - a_a), each axis
    handled separately (guards against a transposed or sign-flipped axis)."""
    nvec = np.array([[0.48, -0.6, 0.64]])   # unit: 0.2304 + 0.36 + 0.4096 = 1
    lat = lb.Lattice(3, (6, 6, 6), nvec, np.array([1.0]), cfl=0.5)
    I = np.zeros((1, 6, 6, 6))
    I[0, 2, 3, 1] = 1.0                      # (z, y, x)
    out = lb.stream(I, lat)[0]
    a = 0.5 * np.abs(nvec[0])
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                wgt = (a[0] if bx else 1 - a[0]) * (a[1] if by else 1 - a[1]) * (a[2] if bz else 1 - a[2])
                assert abs(out[2 + bz, 3 - by, 1 + bx] - wgt) < 1e-15
    assert abs(out.sum() - 1.0) < 1e-15
    assert np.count_nonzero(out) == 8


def test_crossing_beams_superpose():
    L = 48
    n, w = D.ring2d(16, 0.0)
    lat = lb.Lattice(2, (1, L, L), n, w, cfl=0.2, dx=1.0 / L,
                     bc=(lb.VACUUM, lb.VACUUM, lb.PERIODIC))
    A = np.zeros((16, 1, L, L))
    B = np.zeros((16, 1, L, L))
    A[2, 0, 10:14, 5] = 1.0    # 45 degrees
    B[6, 0, 10:14, 40] = 1.0   # 135 degrees
    ra = lb.run(A, lat, lb.Static(), 60)
    rb = lb.run(B, lat, lb.Static(), 60)
    rab = lb.run(A + B, lat, lb.Static(), 60)
    assert np.abs(rab - (ra + rb)).max() < 1e-14


@pytest.mark.parametrize("bc", [lb.PERIODIC, lb.VACUUM])
def test_stream_sites_matches_full_stream(bc):
    n, w = D.icosphere(1)
    shape = (5, 6, 7)
    lat = lb.Lattice(3, shape, n, w, cfl=0.7, dx=1.0 / 7, bc=(bc, bc, bc))
    I = np.random.default_rng(3).random((len(w),) + shape)
    full = lb.stream(I, lat)
    zz, yy, xx = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    sites = (zz.ravel(), yy.ravel(), xx.ravel())
    part = lb.stream_sites(lambda i, z, y, x: I[i, z, y, x], sites, lat)
    assert np.abs(part - full.reshape(len(w), -1)).max() < 1e-15


def test_vacuum_outflow_budget():
    n, w = D.icosphere(1)
    shape = (8, 8, 8)
    lat = lb.Lattice(3, shape, n, w, cfl=0.5, dx=1 / 8, bc=(lb.VACUUM,) * 3)
    I = np.random.default_rng(4).random((len(w),) + shape)
    b = {}
    I1 = lb.step(I, lat, lb.Static(), budget=b)
    assert b["outflow"] > 0
    assert abs(I.sum() - b["outflow"] - I1.sum()) < 1e-12
