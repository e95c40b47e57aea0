"""Coupling outputs of the radiation field for a fluid code, FP64 (oracle).

Sec. 5 (coupling with a relativistic fluid code, step 4) gives, from the
lab-frame moments E, F^i, P^ij and the fluid three-velocity v (c = 1):

  J   = W^2 (E - 2 F.v + P:vv)                          (Eq. J, comoving energy density)
  H_j = W^3 (F.v - E) v_j + W h_ji F^i - W h_ji v_k P^ik (comoving momentum density)
  h_ij = W^2 v_i v_j + delta_ij,  W = (1 - v^2)^(-1/2)

and the radiative four-force source terms

  S_0 = W (kt_a J - eta_t) + kt H_0,
  S_j = W (kt_a J - eta_t) v_j + kt H_j,   kt = kt_a + kt_s,  kt_s = kt_0 - kt_1 / 3.

H_0 follows from H_mu u^mu = 0 (reading: metric signature (-, +, +, +),
u^mu = W (1, v), so H_0 = -v^j H_j).  This scheme keeps kt_1 = 0.

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
    """(S_0, S [3, ...]) of step 4 of the coupling (and J, H, H_0)."""
    J, H = comoving(E, F, P, v)
    W = lorentz(v)
    kt = kt_a + (kt_0 - kt_1 / 3.0)
    H0 = -np.einsum("i...,i...->...", v, H)
    emit = W * (kt_a * J - eta_t)
    S0 = emit + kt * H0
    S = emit[None] * v + kt * H
    return S0, S, J, H, H0


def sym_P(P6, d=3):
    """[3, 3, ...] tensor from the 6 unique components (xx, xy, xz, yy, yz, zz)."""
    xx, xy, xz, yy, yz, zz = P6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
