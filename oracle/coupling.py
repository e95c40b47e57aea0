"""Coupling outputs of the radiation field for a fluid code, FP64 (oracle).

Sec. 5 (coupling with a relativistic fluid code, step 4) gives, from the
lab-frame moments E, F^i, P^ij and the fluid three-velocity v (c = 1):

  J   = W^2 (E - 2 F.v + P:vv)                          (Eq. J, comoving energy density)
  H_j = W^3 (F.v - E) v_j + W h_ji F^i - W h_ji v_k P^ik (comoving momentum density)
  h_ij = W^2 v_i v_j + delta_ij,  W = (1 - v^2)^(-1/2)

and the radiative four-force source terms

  S_0 = W (kt_a J - eta_t) + kt H_0,
  S_j = W (kt_a J - eta_t) v_j + kt H_j,   kt = kt_a + kt_s,  kt_s = kt_0 - kt_1 / 3.

Reading of the index placement: (S_0, S_j) are the lab-frame components of
ONE four-vector, G^mu = (kt_a J - eta_t) u^mu + kt H^mu, with u^mu = W (1, v)
and H^mu the comoving flux four-vector (H^mu u_mu = 0, signature (-, +, +, +)).
Its spatial part is the printed S_j; its time part is W (kt_a J - eta_t) +
kt H^0 with H^0 = v^j H_j, the time component fixed by the orthogonality the
paper names.  (Taking H_0 as the covariant component -v^j H_j would make S_0
and S_j parts of no single four-vector.)  In the fluid rest frame G reduces
to (kt_a J - eta_t, kt H): the tests boost that vector to the lab frame and
compare.  This scheme keeps kt_1 = 0.

Test infrastructure only: tests, smoke() and the bench's CPU baseline may use
this module; the library never does.
"""
import numpy as np


def lorentz(v):
    """W = (1 - v^2)^(-1/2) for v [3, ...]."""
    return 1.0 / np.sqrt(1.0 - np.einsum("i...,i...->...", v, v))


def comoving(E, F, P, v):
    """(J, H [3, ...]) from lab moments E [...], F [3, ...], P [3, 3, ...]."""
    W = lorentz(v)
    Fv = np.einsum("i...,i...->...", F, v)
    Pvv = np.einsum("ij...,i...,j...->...", P, v, v)
    J = W ** 2 * (E - 2.0 * Fv + Pvv)
    d = len(v)
    h = W ** 2 * np.einsum("i...,j...->ij...", v, v) + np.eye(d).reshape((d, d) + (1,) * (v.ndim - 1))
    Pv = np.einsum("ik...,k...->i...", P, v)          # v_k P^ik
    H = (W ** 3 * (Fv - E))[None] * v + W * np.einsum("ji...,i...->j...", h, F) \
        - W * np.einsum("ji...,i...->j...", h, Pv)
    return J, H


def four_force(E, F, P, v, kt_a, kt_0, eta_t, kt_1=0.0):
    """(S_0, S [3, ...]) of step 4 of the coupling (and J, H, H^0)."""
    J, H = comoving(E, F, P, v)
    W = lorentz(v)
    kt = kt_a + (kt_0 - kt_1 / 3.0)
    H0 = np.einsum("i...,i...->...", v, H)  # time component of H^mu (H^mu u_mu = 0)
    emit = W * (kt_a * J - eta_t)
    S0 = emit + kt * H0
    S = emit[None] * v + kt * H
    return S0, S, J, H, H0


def sym_P(P6, d=3):
    """[3, 3, ...] tensor from the 6 unique components (xx, xy, xz, yy, yz, zz)."""
    xx, xy, xz, yy, yz, zz = P6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
