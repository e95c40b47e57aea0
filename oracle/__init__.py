"""FP64 CPU oracle for the grey radiative Lattice-Boltzmann step (Weih et al. 2020).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (``paper_2007_05718_gb300``): it builds its own direction tables,
its own streaming stencil and its own collision, in plain numpy FP64, written
so that each function can be checked against the paper by eye.

Modules
-------
directions  discrete direction sets (Sec. 3.2.1): 2D ring, icosahedral
            geodesic sets, Gauss-Legendre x trapezoid product sets, and the
            isotropy tensors of Eq. (iso-tensors).
lb          one timestep (Sec. 3.3): pull-streaming with the trilinear /
            bilinear rule of Eq. (interp), moments (Eqs. moments_discrete,
            higher_moments), the explicit collision (Eq. collision-step), the
            implicit collision (Eq. rte_implicit) solved exactly and by the
            literal Lambda iteration, the mixed-frame moving-fluid collision
            (App. B), frozen cells, and the energy budget.
analytic    closed-form references: radiating sphere (Sec. 4.2.2), Gaussian
            diffusion (Eq. gauss-hill-analytic with the diffusion coefficient
            of App. A), the free-streaming radiation wave (Sec. 4.1.2), and
            the dense N x N brute-force collision solve.
coupling    comoving J, H and the radiative four-force (S_0, S_j) of the
            coupling with a fluid code (Sec. 5, Eq. J).
diffusion   the diffusion coefficient of the scheme (App. A): exact
            spatial-moment recursion, closed form, the Gaussian-hill fit of
            App. A.2 and the fit of Eq. (numerical-diff-coeff2).

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: isotropy identities, the binomial closed form of free streaming,
the exact CFL = 1 shift, linearity, brute-force dense solves, conservation
under pure scattering, the radiating-sphere and Gaussian-diffusion analytic
solutions, the paper's statement that the Lambda iteration converges in
at most three cycles for kappa_a = 1e7, Lorentz boosts of known comoving
states, the exact energy and second-moment identities of the free-streaming
wave, and brute-force lattice runs for the moment recursion.
"""
