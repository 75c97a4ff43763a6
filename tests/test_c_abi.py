"""The C ABI from plain C (no Python, no torch): a C99 program compiled against include/fdfd.h
and linked to libfdfd.so runs the host-side calls on the CPU: default options, context
creation with its argument checks, the symbolic phase and its statistics, the mode solver,
and the error codes of calls made in the wrong order."""
import os
import shutil
import subprocess

import pytest

fd = pytest.importorskip("paper_2307_05388_gb300.fdfd")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "fdfd.h"

int main(void) {
  fdfd_options opt;
  fdfd_default_options(&opt);
  if (opt.mode != FDFD_MODE_MIXED || opt.gmres_restart != 8) return 10;
  double k0 = 2.0 * 3.141592653589793 / 1.55;
  fdfd_grid grid = {60, 50};
  fdfd_pml pml = {8, 8, log(1e-8), 3.0};
  fdfd_box box = {15, 12, 30, 26};
  fdfd_ctx* ctx = NULL;
  if (fdfd_create(&ctx, grid, 0.04, &k0, 1, pml, box, &opt, NULL) != FDFD_OK || !ctx) return 11;
  fdfd_box bad = {50, 40, 30, 26};
  fdfd_ctx* c2 = NULL;
  if (fdfd_create(&c2, grid, 0.04, &k0, 1, pml, bad, &opt, NULL) != FDFD_ERR_ARG || c2) return 12;
  if (fdfd_solve(ctx, (const double*)&k0, (double*)&opt, 1, 0) != FDFD_ERR_STATE) return 13;
  if (fdfd_analyze(ctx) != FDFD_OK) return 14;
  fdfd_stats st;
  if (fdfd_stats_get(ctx, &st) != FDFD_OK || st.sf != 1 || st.n_fronts < 2 || st.max_front < 1) return 15;
  printf("fronts %d levels %d max_front %d\n", st.n_fronts, st.n_levels, st.max_front);
  fdfd_destroy(ctx);
  double eps[40], mu[2], th[2], phi[80];
  for (int j = 0; j < 40; ++j) eps[j] = (j >= 16 && j < 24) ? 12.11 : 2.085;
  if (fdfd_slab_modes(40, 0.16, eps, 2, mu, th, phi) != FDFD_OK) return 16;
  if (!(mu[0] > mu[1]) || !(mu[1] > 0.16 * 0.16 * 2.085)) return 17;
  if (fdfd_slab_modes(40, 0.16, eps, 41, mu, th, phi) != FDFD_ERR_ARG) return 18;
  printf("mu %.12f %.12f\n", mu[0], mu[1]);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_against_the_header_and_library(tmp_path):
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(fd.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lfdfd", f"-Wl,-rpath,{libdir}", "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    mu = [float(v) for v in r.stdout.split("mu ")[1].split()]
    import numpy as np
    from oracle import fdfd_oracle as O
    eps = np.where((np.arange(40) >= 16) & (np.arange(40) < 24), 12.11, 2.085)
    mu_o, _, _ = O.slab_modes(eps, 0.16, 2)
    np.testing.assert_allclose(mu, mu_o, rtol=0, atol=1e-11)
