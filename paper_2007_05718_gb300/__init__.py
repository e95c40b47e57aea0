"""GB300-native grey radiative Lattice-Boltzmann (Weih et al. 2020).

Importing the package is cheap: the CUDA library is loaded on first use
through :mod:`paper_2007_05718_gb300.lbrt`.
"""
__all__ = ["lbrt", "workloads"]
