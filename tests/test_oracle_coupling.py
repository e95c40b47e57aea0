"""Pins of the coupling outputs (oracle/coupling.py): a radiation field
built from a known comoving state must transform back to it."""
import numpy as np

from oracle import coupling as CP


def _lab_moments(J, H, v):
    """Lab E = T^00, F^i = T^0i, P^ij = T^ij of the radiation stress tensor
    with comoving energy density J, comoving flux H and isotropic comoving
    pressure J/3: T^mn = (4/3) J u^m u^n + (1/3) J eta^mn + H^m u^n + H^n u^m,
    eta = diag(-1, 1, 1, 1), u = W (1, v), H^0 = H.v so that H.u = 0."""
    W = 1.0 / np.sqrt(1.0 - v @ v)
    u = W * np.concatenate([[1.0], v])
    Hm = np.concatenate([[H @ v], H])
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    T = (4.0 / 3.0) * J * np.outer(u, u) + (J / 3.0) * eta + np.outer(Hm, u) + np.outer(u, Hm)
    return T[0, 0], T[0, 1:], T[1:, 1:]


def test_boosted_field_returns_comoving_state():
    g = np.random.default_rng(7)
    for _ in range(50):
        v = g.normal(size=3)
        v *= g.uniform(0.0, 0.9) / np.linalg.norm(v)
        J = g.uniform(0.1, 5.0)
        H = g.normal(size=3) * 0.3 * J
        E, F, P = _lab_moments(J, H, v)
        Jc, Hc = CP.comoving(np.array(E), F[:, None], P[:, :, None], v[:, None])
        assert abs(Jc[0] - J) < 1e-12 * J
        assert np.allclose(Hc[:, 0], H, rtol=0, atol=1e-12 * J)


def test_rest_frame_reduces_to_lab_moments():
    g = np.random.default_rng(8)
    E = g.uniform(1, 2, size=5)
    F = g.normal(size=(3, 5))
    P = g.normal(size=(3, 3, 5))
    P = P + P.transpose(1, 0, 2)
    v = np.zeros((3, 5))
    S0, S, J, H, H0 = CP.four_force(E, F, P, v, kt_a=2.0, kt_0=3.0, eta_t=0.5)
    assert np.allclose(J, E) and np.allclose(H, F) and np.allclose(H0, 0.0)
    assert np.allclose(S0, 2.0 * E - 0.5)
    assert np.allclose(S, 5.0 * F)


def test_H0_makes_H_orthogonal_to_u_and_sources_in_equilibrium_vanish():
    # comoving isotropic field in equilibrium: J = eta_t / kt_a, H = 0
    v = np.array([0.3, -0.4, 0.2])
    J = 2.5
    E, F, P = _lab_moments(J, np.zeros(3), v)
    S0, S, Jc, Hc, H0 = CP.four_force(np.array([E]), F[:, None], P[:, :, None], v[:, None],
                                      kt_a=4.0, kt_0=1.5, eta_t=4.0 * J)
    assert abs(S0[0]) < 1e-12 and np.allclose(S[:, 0], 0.0, atol=1e-12)
    # a comoving flux: H_mu u^mu = 0 with H_0 = -v.H
    H = np.array([0.1, 0.2, -0.3])
    E, F, P = _lab_moments(J, H, v)
    S0, S, Jc, Hc, H0 = CP.four_force(np.array([E]), F[:, None], P[:, :, None], v[:, None],
                                      kt_a=1.0, kt_0=0.0, eta_t=0.0)
    # H^mu u_mu = -W H^0 + W v.H = 0
    W = 1.0 / np.sqrt(1.0 - v @ v)
    assert abs(-W * H0[0] + W * (v @ Hc[:, 0])) < 1e-12


def _boost(v):
    """Lorentz boost Lambda(v): rest-frame components of a four-vector ->
    components in the lab frame in which the rest frame moves with v."""
    W = 1.0 / np.sqrt(1.0 - v @ v)
    L = np.eye(4)
    L[0, 0] = W
    L[0, 1:] = L[1:, 0] = W * v
    L[1:, 1:] += (W - 1.0) * np.outer(v, v) / (v @ v)
    return L


def test_four_force_is_the_boosted_rest_frame_source():
    """In the fluid rest frame the source four-vector is (kt_a J - eta_t,
    kt H): the energy exchange and the momentum drag of Sec. 5.  Boosted to
    the lab frame it must equal (S_0, S_j) of the oracle, out of equilibrium
    (kt_a J != eta_t), with a comoving flux H != 0 and v != 0, so that the
    W (kt_a J - eta_t) v_j term and the kt H_0 term both carry weight: a sign
    slip in either fails here."""
    g = np.random.default_rng(9)
    for _ in range(50):
        v = g.normal(size=3)
        v *= g.uniform(0.05, 0.9) / np.linalg.norm(v)
        J = g.uniform(0.1, 5.0)
        Hr = g.normal(size=3) * 0.3 * J             # rest-frame comoving flux
        kt_a, kt_0 = g.uniform(0.1, 10.0), g.uniform(0.0, 10.0)
        eta_t = kt_a * J * g.uniform(0.2, 3.0)      # away from equilibrium
        L = _boost(v)
        Hlab = L @ np.concatenate([[0.0], Hr])      # comoving flux four-vector in the lab
        E, F, P = _lab_moments(J, Hlab[1:], v)
        G = L @ np.concatenate([[kt_a * J - eta_t], (kt_a + kt_0) * Hr])
        S0, S, Jc, Hc, H0 = CP.four_force(np.array([E]), F[:, None], P[:, :, None], v[:, None],
                                          kt_a=kt_a, kt_0=kt_0, eta_t=eta_t)
        scale = abs(kt_a * J - eta_t) + (kt_a + kt_0) * np.linalg.norm(Hr)
        assert abs(S0[0] - G[0]) < 1e-11 * scale
        assert np.allclose(S[:, 0], G[1:], rtol=0, atol=1e-11 * scale)
        assert abs(H0[0] - Hlab[0]) < 1e-11 * J
