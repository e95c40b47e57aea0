"""Argument checks of the allocation-free energy reduction's binding.

A float16 or short population tensor would make the reduction kernel read
past the allocation, and a float32 `out` would take an 8-byte store into a
4-byte buffer: the binding must reject all of these before it reaches the C
entry point.  No GPU is needed: the library is replaced by a stub that fails
the test if it is ever called."""
import pytest
import torch

from paper_2007_05718_gb300 import lbrt


@pytest.fixture
def no_c_call(monkeypatch):
    def forbidden(*a, **k):
        raise AssertionError("the C entry point must not be reached")
    monkeypatch.setattr(lbrt, "load", forbidden)


@pytest.mark.parametrize("pop,ndir,sites,frag", [
    (torch.zeros(42 * 8, dtype=torch.float16), 42, 8, "float32"),
    (torch.zeros(42 * 8, dtype=torch.bfloat16), 42, 8, "float32"),
    (torch.zeros(42 * 8, dtype=torch.float64), 42, 8, "float32"),
    (torch.zeros(42 * 8 - 1, dtype=torch.float32), 42, 8, "fewer"),
    (torch.zeros((8, 84), dtype=torch.float32).t(), 42, 8, "contiguous"),
    (torch.zeros(8, dtype=torch.float32), 0, 8, ">= 1"),
    (torch.zeros(8, dtype=torch.float32), 1, 0, ">= 1"),
])
def test_bad_populations_rejected_before_the_c_call(no_c_call, pop, ndir, sites, frag):
    with pytest.raises(ValueError, match=frag):
        lbrt.lb_rt_total_energy_noalloc(pop, ndir, sites)


@pytest.mark.parametrize("out", [
    torch.zeros(1, dtype=torch.float32),
    torch.zeros(0, dtype=torch.float64),
    torch.zeros(1, dtype=torch.float64),  # host tensor: the device output must be on the GPU
])
def test_bad_output_rejected_before_the_c_call(no_c_call, out):
    pop = torch.zeros(42 * 8, dtype=torch.float32)
    with pytest.raises(ValueError):
        lbrt.lb_rt_total_energy_noalloc(pop, 42, 8, out=out)


def test_numpy_populations_rejected(no_c_call):
    import numpy as np
    with pytest.raises(ValueError, match="CUDA tensor"):
        lbrt.lb_rt_total_energy_noalloc(np.zeros(42 * 8, dtype=np.float32), 42, 8)
