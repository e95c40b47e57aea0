"""Pins for the oracle's direction tables (Sec. 3.2.1, Eqs. iso-tensors,
isotropy-cond, sph-quad-cond-2d)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import directions as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def _delta_product(k, dims=3):
    """Sum over the distinct pairings of delta products, rank k (k even)."""
    out = np.zeros((dims,) * k)
    for idx in itertools.product(range(dims), repeat=k):
        # count pairings (a1 a2)(a3 a4)... over all perfect matchings
        def matchings(items):
            if not items:
                yield []
                return
            a = items[0]
            for j in range(1, len(items)):
                rest = items[1:j] + items[j + 1:]
                for m in matchings(rest):
                    yield [(a, items[j])] + m
        tot = 0
        for m in matchings(list(range(k))):
            tot += all(idx[p] == idx[q] for p, q in m)
        out[idx] = tot
    return out


@pytest.mark.parametrize("level,N", [(1, 42), (2, 162)])
def test_icosphere_counts_and_norms(level, N):
    n, w = D.icosphere(level)
    assert n.shape == (N, 3)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    # distinct points
    d2 = ((n[:, None] - n[None]) ** 2).sum(-1) + np.eye(N)
    assert d2.min() > 1e-3


@pytest.mark.parametrize("level", [1, 2])
def test_icosphere_isotropy_to_rank5(level):
    n, w = D.icosphere(level)
    for k in (1, 3, 5):
        assert np.abs(D.isotropy_tensor(n, w, k)).max() < 1e-15
    assert np.allclose(D.isotropy_tensor(n, w, 2), np.eye(3) / 3.0, atol=1e-15, rtol=0)
    T4 = D.isotropy_tensor(n, w, 4)
    assert np.allclose(T4, _delta_product(4) / 15.0, atol=1e-15, rtol=0)
    # rank 6 is NOT isotropic (first invariant harmonic has degree 6): the
    # set has order exactly p = 5
    T6 = D.isotropy_tensor(n, w, 6)
    assert np.abs(T6 - _delta_product(6) / 105.0).max() > 1e-6


def test_icosphere_level1_contains_axes():
    n, _ = D.icosphere(1)
    for ax in range(3):
        for s in (-1.0, 1.0):
            e = np.zeros(3)
            e[ax] = s
            assert any(np.array_equal(row, e) for row in n)


def test_ring_order():
    facts = json.load(open(GOLDEN))["ring_order"]
    N, p = facts["N"], facts["p"]
    for phi0 in (0.0, math.pi / 6):
        n, w = D.ring2d(N, phi0)
        phi = np.arctan2(n[:, 1], n[:, 0])
        for m in range(1, p + 1):
            assert abs(np.sum(w * np.exp(1j * m * phi))) < 1e-14
        # degree p + 1 is not integrated exactly
        assert abs(np.sum(w * np.exp(1j * (p + 1) * phi))) > 0.5
        assert np.allclose(D.isotropy_tensor(n, w, 2, dims=2), np.eye(2) / 2, atol=1e-15)


def test_ring_rotation_puts_beam_on_direction_zero():
    n, _ = D.ring2d(16, math.pi / 6)
    assert np.allclose(n[0], [math.sqrt(3) / 2, 0.5, 0.0], atol=1e-16)


def test_ring_snaps_zero_components():
    n, _ = D.ring2d(16, 0.0)
    assert n[4, 0] == 0.0 and not math.copysign(1.0, n[4, 0]) < 0
    assert n[12, 0] == 0.0 and not math.copysign(1.0, n[12, 0]) < 0
    assert list(D.sgn(np.array([0.0, -0.0, -1e-3, 2.0]))) == [1, 1, -1, 1]


def test_gauss_legendre_product_order():
    n, w = D.gauss_legendre_product(4, 8)
    assert len(w) == 32 and abs(w.sum() - 1) < 1e-15
    # GL with 4 nodes integrates mu^k exactly for k <= 7; trapezoid with 8
    # points integrates e^{i m phi} for |m| < 8: all ranks <= 7 isotropic
    for k in (1, 3, 5, 7):
        assert np.abs(D.isotropy_tensor(n, w, k)).max() < 1e-15
    assert np.allclose(D.isotropy_tensor(n, w, 2), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(D.isotropy_tensor(n, w, 4), _delta_product(4) / 15, atol=1e-15)
    assert np.allclose(D.isotropy_tensor(n, w, 6), _delta_product(6) / 105, atol=1e-15)


def test_canonical_order_is_sorted_by_integer_key():
    n, _ = D.icosphere(2)
    keys = [tuple(np.rint(row[::-1] * 1e9).astype(np.int64)) for row in n]
    assert keys == sorted(keys)
