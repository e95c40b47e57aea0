"""The C ABI library loads and exports every entry point of include/lb_rt.h;
configuration errors are reported before any CUDA call (CPU-only tests)."""
import os
import re
import subprocess

import pytest

from paper_2007_05718_gb300 import lbrt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lb_rt_\w+)\s*\(", text))
    return names


def test_header_declares_the_five_core_calls():
    d = _declared()
    for n in ("lb_rt_create", "lb_rt_set_fluid", "lb_rt_step", "lb_rt_moments", "lb_rt_destroy"):
        assert n in d


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lbrt.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lb_rt_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing
    for name in _declared():
        assert hasattr(lib, name)


def test_binding_covers_the_header():
    assert set(lbrt.EXPORTED) == _declared()
    for name in lbrt.EXPORTED:
        assert callable(getattr(lbrt, name))


@pytest.mark.parametrize("kw,frag", [
    (dict(dims=4, nx=8, ny=8, nz=8), "dims"),
    (dict(dims=2, nx=8, ny=8, nz=2), "nz == 1"),
    (dict(dims=3, nx=8, ny=8, nz=8, cfl=1.5), "cfl"),
    (dict(dims=3, nx=0, ny=8, nz=8), "grid"),
    (dict(dims=3, nx=8, ny=8, nz=8, level=5), "level"),
    (dict(dims=2, nx=8, ny=8, nz=1, dirset=lbrt.LB_RT_RING2D, ndir=2), "ring"),
    (dict(dims=2, nx=8, ny=8, nz=1, dirset=lbrt.LB_RT_ICOSPHERE, level=1), "n_z"),
    (dict(dims=3, nx=8, ny=8, nz=8, collision=lbrt.LB_RT_LAMBDA_K, lambda_iters=0), "lambda_iters"),
    (dict(dims=3, nx=8, ny=8, nz=8, dirs=[[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]), "isotropic"),
    (dict(dims=3, nx=8, ny=8, nz=8, dirs=[[2.0, 0, 0]]), "unit"),
    (dict(dims=3, nx=8, ny=8, nz=8, moving=True, collision=lbrt.LB_RT_EXPLICIT), "moving"),
    (dict(dims=3, nx=2048, ny=2048, nz=1024), "2^31"),
])
def test_invalid_configs_rejected_before_cuda(lib, kw, frag):
    with pytest.raises(lbrt.LBRTError) as ei:
        lbrt.lb_rt_create(**kw)
    assert ei.value.status == lbrt.LB_RT_EINVAL
    assert frag in str(ei.value)


def test_null_handle_calls_are_safe(lib):
    assert lib.lb_rt_step(None, 1) == lbrt.LB_RT_EINVAL
    assert lib.lb_rt_step_moments(None, 1, None, None, lbrt.LB_RT_HOST) == lbrt.LB_RT_EINVAL
    assert lib.lb_rt_coupling(None, None, None, None, lbrt.LB_RT_HOST) == lbrt.LB_RT_EINVAL
    assert lib.lb_rt_sync(None) == lbrt.LB_RT_EINVAL
    lib.lb_rt_destroy(None)
    assert lib.lb_rt_state_bytes(None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without liblbrt.so every call raises."""
    monkeypatch.setattr(lbrt, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        lbrt.load(str(tmp_path / "liblbrt.so"))
