"""The public header is plain C: a C11 translation unit that uses every
entry point compiles warning-free with gcc, and links against liblbrt.so
(no call is executed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stddef.h>
#include <stdint.h>
#include "lb_rt.h"

int use_every_call(void) {
  lb_rt_config cfg = {0};
  cfg.dims = 3; cfg.nx = cfg.ny = cfg.nz = 16; cfg.dirset = LB_RT_ICOSPHERE;
  cfg.cfl = 0.5; cfg.dx = 1.0 / 16;
  lb_rt* h = NULL;
  if (lb_rt_create(&cfg, &h) != LB_RT_OK) return 1;
  lb_rt_fluid f = {0};
  f.kappa_a_s = 1.0f;
  float E[16 * 16 * 16], F[3 * 16 * 16 * 16], J[16 * 16 * 16], H[3 * 16 * 16 * 16],
      S[4 * 16 * 16 * 16];
  lb_rt_budget b;
  int n = 0;
  float ms = 0.f;
  int launches = 0;
  int st = lb_rt_set_fluid(h, &f, LB_RT_HOST) | lb_rt_set_state(h, E, LB_RT_STATE_ISOTROPIC, LB_RT_HOST) |
           lb_rt_step(h, 1) | lb_rt_step_moments(h, 1, E, F, LB_RT_HOST) |
           lb_rt_moments(h, E, F, NULL, &b, LB_RT_HOST) | lb_rt_coupling(h, J, H, S, LB_RT_HOST) |
           lb_rt_get_populations(h, NULL, LB_RT_HOST) | lb_rt_sync(h) |
           lb_rt_directions(h, &n, NULL, NULL, NULL) | lb_rt_enable_timing(h, 1) |
           lb_rt_last_step_ms(h, &ms, &launches) | lb_rt_set_frozen(h, NULL, 0, NULL);
  size_t bytes = lb_rt_state_bytes(h);
  (void)bytes;
  st |= lb_rt_save_state(h, NULL, 0) | lb_rt_restore_state(h, NULL, 0);
  double tot = 0.0;
  st |= lb_rt_total_energy_noalloc(NULL, 0, 0, &tot, LB_RT_HOST, NULL);
  (void)lb_rt_last_error(h);
  (void)lb_rt_version();
  lb_rt_destroy(h);
  lb_rt_batch_config bc = {0};
  lb_rt_batch* bt = NULL;
  st |= lb_rt_batch_create(&bc, &bt);
  int slot = -1, slots[4];
  st |= lb_rt_batch_admit(bt, &cfg, &f, LB_RT_HOST, E, LB_RT_STATE_ISOTROPIC, LB_RT_HOST, 10, &slot);
  st |= lb_rt_batch_tick(bt, &n) | lb_rt_batch_sync(bt) | lb_rt_batch_poll(bt, slots, 4, &n);
  long long steps = 0;
  int zc = 0, ctas = 0;
  st |= lb_rt_batch_moments(bt, slot, E, F, NULL, LB_RT_HOST) | lb_rt_batch_steps(bt, slot, &steps) |
        lb_rt_batch_tuning(bt, slot, &zc, &ctas) | lb_rt_batch_plan(bt, slot, &zc, &ctas, &n) |
        lb_rt_batch_release(bt, slot);
  (void)lb_rt_batch_problem_bytes(bt, &cfg);
  (void)lb_rt_batch_last_error(bt);
  lb_rt_batch_destroy(bt);
  return st;
}

int main(int argc, char** argv) {
  (void)argv;
  return argc > 100 ? use_every_call() : 0;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2007_05718_gb300 import build as B
    B.build()
    src = tmp_path / "use.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "use"
    lib_dir = os.path.dirname(B.LIB)
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", lib_dir, "-llbrt",
                        "-Wl,-rpath," + lib_dir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
