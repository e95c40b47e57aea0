"""Diffusion-coefficient study (App. A.2) on the GPU through the batch C ABI.

Reduced size: every sweep point's E at each sample time equals the FP64
oracle's lattice run (1e-5 relative L2).  Full size (80 points, 512^2
periodic, 120-direction ring, 200 steps): the variance growth of every run
equals the oracle's exact spatial-moment recursion, the variance D equals
the recursion's, the Gaussian-hill fit of App. A.2 agrees with the oracle's
own fit, and the Eq. (numerical-diff-coeff2) coefficients are reported."""
import math

import numpy as np
import pytest

from oracle import diffusion as Df
from oracle import directions as OD
from oracle import lb
from paper_2007_05718_gb300 import diffusion_study as S
from paper_2007_05718_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def test_study_reduced_parity(cuda):
    n, sigma0, steps = 64, 6.0, (5, 10, 20)
    pts = [dict(kappa_0=1.0, cfl=0.5, lam=0.5), dict(kappa_0=5.0, cfl=1.0, lam=0.75),
           dict(kappa_0=0.5, cfl=0.1, lam=0.0)]
    out = S.run_sweep(pts, n=n, sigma0=sigma0, sample_steps=steps)
    nn, w = OD.ring2d(120, 0.0)
    E0 = W.gaussian_E0((1, n, n), sigma0).astype(np.float64)
    for p, snaps in zip(pts, out["E"]):
        lat = lb.Lattice(2, (1, n, n), nn, w, cfl=p["cfl"], dx=1.0)
        co = lb.Static(kappa_0=p["kappa_0"], lam=p["lam"])
        I = lb.isotropic(E0, lat)
        done = 0
        for k, t in enumerate(steps):
            I = lb.run(I, lat, co, t - done)
            done = t
            Eo = I.sum(0)[0]
            err = np.linalg.norm(snaps[k] - Eo) / np.linalg.norm(Eo)
            assert err <= TOL_F32, (p, t, err)


def test_study_full_sweep(cuda):
    n, sigma0 = 512, 10.0
    pts = S.sweep_points()
    out = S.run_sweep(pts, n=n, sigma0=sigma0)
    steps = out["steps"]
    E0 = W.gaussian_E0((1, n, n), sigma0)[0]
    V0 = S.variance(E0, 0)
    nn, w = OD.ring2d(120, 0.0)
    mabs = float(np.sum(w * np.abs(nn[:, 0])))
    rows = []
    for j, (p, snaps) in enumerate(zip(pts, out["E"])):
        Vp = Df.moment_recursion(nn, w, 2, p["cfl"], 1.0, p["kappa_0"], p["lam"], steps[-1])
        for k, t in enumerate(steps):
            dv = S.variance(snaps[k], 0) - V0
            assert abs(dv - Vp[t]) <= 1e-4 * Vp[t] + 2e-4, (p, t, dv, Vp[t])
        Dv = S.variance_D(snaps, steps, p["cfl"])
        Dx = (Vp[steps[-1]] - Vp[steps[-2]]) / (2.0 * (steps[-1] - steps[-2]) * p["cfl"])
        assert abs(Dv / Dx - 1.0) < 1e-3, (p, Dv, Dx)
        Dc = Df.closed_form_D(p["kappa_0"], p["lam"], p["cfl"], 1.0, 2, mabs)
        Dg, eg = S.fit_gaussian_D(snaps, steps, p["cfl"], sigma0, Dv)
        rows.append(dict(p, D_var=Dv, D_closed=Dc, D_gauss=Dg, err=eg))
        if j % 10 == 0:   # the oracle's own App. A.2 fit on a subset
            x = np.arange(n) + 0.5 - 0.5 * n
            Do, eo = Df.fit_gaussian_D([s.astype(np.float64) for s in snaps],
                                       [t * p["cfl"] for t in steps], x, x, (0.0, 0.0), (n, n),
                                       sigma0)
            assert abs(Dg / Do - 1.0) < 1e-4 and abs(eg - eo) < 1e-6, (p, Dg, Do, eg, eo)
    k0, lam, dt = (np.array([r[key] for r in rows]) for key in ("kappa_0", "lam", "cfl"))
    a_var, rms_var = S.fit_alphas(k0, lam, dt, [r["D_var"] for r in rows])
    a_cl, rms_cl = Df.fit_alphas(k0, lam, dt, 1.0, 2, [r["D_closed"] for r in rows])
    dif = [r for r in rows if r["err"] <= 0.01]
    a_g, rms_g = S.fit_alphas([r["kappa_0"] for r in dif], [r["lam"] for r in dif],
                              [r["cfl"] for r in dif], [r["D_gauss"] for r in dif])
    print("diffusion study 512^2 ring-120: %d points, %d within 1%% of a Gaussian hill"
          % (len(rows), len(dif)))
    worst = max(abs(r["D_var"] / r["D_closed"] - 1.0) for r in rows)
    print("variance D vs closed form: worst relative difference %.2e" % worst)
    print("alpha fit (variance D): %s rms %.3f" % (["%.4f" % a for a in a_var], rms_var))
    print("alpha fit (closed form): %s rms %.3f" % (["%.4f" % a for a in a_cl], rms_cl))
    print("alpha fit (Gaussian fit, diffusive points): %s rms %.3f"
          % (["%.4f" % a for a in a_g], rms_g))
    for r in rows[::4]:
        print("  k0dx=%-5g cfl=%-5g lam=%-5g D_var=%.5f D_closed=%.5f D_gauss=%.5f err=%.4f"
              % (r["kappa_0"], r["cfl"], r["lam"], r["D_var"], r["D_closed"], r["D_gauss"],
                 r["err"]))
    np.testing.assert_allclose(a_var, a_cl, rtol=2e-2, atol=2e-3)
