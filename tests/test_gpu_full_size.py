"""Element-wise oracle parity at the benchmarked sizes (C2 to C4).

* C2 (340 x 340) with the library's default options, the configuration the benchmark
  times: tensor-core update matrices in the BF16 three-way split form with the contraction
  split over several CTAs on its small levels.  Forward and transpose fields against
  SuperLU, element by element, at 1e-8; the raw complex FP32-factor error is printed.
  Also with L21 and U12 formed on the tensor cores (option tensor_offdiag), at C2 and C3.
* C3 (540 x 540, TE0 and TE1 sources of its input guide) and C4 (1040 x 1040), each
  restricted to its first wavelength: the same comparison on 292k and 1.08M unknowns.  Each
  side builds the mode sources with its own mode solver.
* C4's gradient (four wavelengths) on 32 seeded design pixels against central differences
  of the oracle's objective with step 1e-4 in rho (Eq. 3), every perturbed F evaluated
  exactly by a rank-one update of the oracle's factorisation.

The oracle runs in spawned worker processes, started before the GPU work."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import fdfd_oracle as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402
from tests import _gpu_util as U  # noqa: E402
from tests import _oracle_jobs as J  # noqa: E402

FIELD_TOL = 1e-8
GRAD_TOL = 1e-6
DEV = "cuda"


@pytest.fixture(scope="module")
def pool():
    ex = cf.ProcessPoolExecutor(max_workers=max(1, min(4, (os.cpu_count() or 1) - 1)),
                                mp_context=mp.get_context("spawn"))
    yield ex
    ex.shutdown(wait=True, cancel_futures=True)


def _fields_on_gpu(s, b):
    """Refined and raw (unrefined complex FP32 factors) solutions, forward and transpose."""
    out = {}
    for tr in (False, True):
        out[tr] = s.solve(b, transpose=tr).cpu().numpy()
    s.set_options(ir_max_iter=0)
    raw = {tr: s.solve(b, transpose=tr).cpu().numpy() for tr in (False, True)}
    s.set_options(ir_max_iter=40)
    return out, raw


def _compare(name, x, raw, ref_f, ref_t):
    for tr, ref in ((False, ref_f), (True, ref_t)):
        for r in range(ref.shape[0]):
            err = O.rel_err(x[tr][0, r], ref[r])
            rerr = O.rel_err(raw[tr][0, r], ref[r])
            print(f"{name} transpose={tr} rhs {r}: field error {err:.2e} (raw FP32 factors {rerr:.2e})")
            assert err <= FIELD_TOL
            assert rerr < 1e-1


def _gpu_rhs(name, random_seed=None):
    """The same right-hand sides as the oracle job's, sources built with the library's mode solver."""
    wl = W.with_modes(W.make(name), FD.slab_modes).select_wavelengths([0])
    rows = [wl.source_dense(s, 0) for s in range(wl.n_src)]
    if random_seed is not None:
        rows.append(W.random_complex(wl.n, random_seed))
    return wl, np.stack(rows)


@pytest.mark.parametrize("offdiag", [0, 1])
def test_c2_default_options_fields_match_the_oracle(pool, offdiag):
    """offdiag 1: L21 and U12 of the tensor-core fronts as products with the triangular inverses
    on the tensor cores, the panel steps over the pivot blocks only."""
    job = pool.submit(J.fields, "c2", 0, 41)
    wl, rhs = _gpu_rhs("c2", 41)
    s = U.make_solver(wl, tensor_offdiag=offdiag)
    s.profile(True)
    s.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    prof = s.profile_get()
    s.profile(False)
    # the benchmarked path: update matrices on the tensor cores with split contractions
    assert prof["lu_schur_tc"]["launches"] > 0 and prof["lu_schur_sum"]["launches"] > 0
    assert (prof.get("lu_trsm_tc", {}).get("launches", 0) > 0) == bool(offdiag)
    x, raw = _fields_on_gpu(s, torch.from_numpy(rhs[None].copy()).to(DEV))
    ref_f, ref_t = job.result()
    _compare(f"c2 (offdiag {offdiag})", x, raw, ref_f, ref_t)
    s.close()


@pytest.mark.parametrize("name,offdiag", [("c3", 0), ("c3", 1), ("c4", 0)])
def test_first_wavelength_fields_match_the_oracle(pool, name, offdiag):
    job = pool.submit(J.fields, name, 0)
    wl, rhs = _gpu_rhs(name)
    s = U.make_solver(wl, tensor_offdiag=offdiag)
    s.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    x, raw = _fields_on_gpu(s, torch.from_numpy(rhs[None].copy()).to(DEV))
    ref_f, ref_t = job.result()
    _compare(f"{name} (first wavelength, offdiag {offdiag})", x, raw, ref_f, ref_t)
    s.close()


def test_c4_gradient_matches_central_differences_on_32_pixels(pool):
    """dF/drho of one C4 design iteration (four wavelengths, adjoint solves on the cached factors,
    Eq. 3) at 32 seeded pixels against (F(rho + h e_p) - F(rho - h e_p)) / 2h of the oracle, h = 1e-4."""
    wl = W.make("c4")
    bw, bh = wl.box[2], wl.box[3]
    pixels = np.random.default_rng(2307).choice(bw * bh, 32, replace=False)
    jobs = [pool.submit(J.pixel_differences, "c4", w, pixels, 1e-4) for w in range(wl.n_omega)]
    prob = U.problem(wl)
    F, g = prob.iteration(U.eps_design_tensor(wl, wl.rho))
    lib = g.cpu().numpy()[pixels] * W.DELTA_EPS
    prob.solver.close()
    fd = sum(j.result() for j in jobs)
    err = O.rel_err(lib, fd)
    print(f"c4 gradient at 32 pixels: relative error {err:.2e} against central differences")
    assert err <= GRAD_TOL
