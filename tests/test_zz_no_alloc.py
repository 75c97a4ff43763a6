"""fdfd_solve_raw_noalloc: the cached-factor solve that allocates no device memory.

It is meant for callers that cannot call cudaMalloc at solve time (no
allocator-induced device synchronisation in a latency-critical loop, budgeted
or foreign-owned device memory, embedding applications that forbid allocation
after set-up).  Its temporary storage is one fixed device array inside the
library.  These tests call it through the C ABI twice in a row and compare
with the existing entry point, fdfd_solve without refinement (ir_max_iter = 0),
which runs the same sweeps on context-allocated scratch.  This file is named
so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402

TOL = 1e-12    # same kernels, same inputs: the two paths agree to rounding (in practice bit for bit)


def _solver(wl, mode):
    s = FD.Solver(wl.nx, wl.ny, wl.dx, 2 * np.pi / wl.wavelengths, wl.npml, box=wl.box,
                  options=FD.default_options(mode=mode, ir_max_iter=0))
    s.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).cuda())
    return s


def _noalloc(s, b, transpose):
    x = torch.empty_like(b)
    nrhs = b.numel() // (s.n_omega * s.n)
    st = FD._lib.fdfd_solve_raw_noalloc(s._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), nrhs,
                                        int(transpose))
    return st, x


@pytest.mark.parametrize("mode", [FD.MODE_MIXED, FD.MODE_F64])
@pytest.mark.parametrize("transpose", [False, True])
def test_noalloc_matches_existing_solve_twice(mode, transpose):
    wl = W.make_small(48, 41, 6, (12, 10, 20, 18), n_omega=2, n_src=1, seed=21)
    s = _solver(wl, mode)
    for call in range(2):
        b = torch.from_numpy(W.random_complex((wl.n_omega, 2, wl.n), 100 + call)).cuda()
        st, x = _noalloc(s, b, transpose)
        assert st == FD.FDFD_OK, FD._lib.fdfd_last_error(s._h).decode()
        ref = s.solve(b, transpose=transpose)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= TOL, (call, err)
    s.close()


def test_noalloc_c1_workload():
    wl = W.make("c1")
    s = _solver(wl, FD.MODE_MIXED)
    b = torch.from_numpy(wl.source_dense(0).reshape(1, 1, -1).copy()).cuda()
    for _ in range(2):
        st, x = _noalloc(s, b, False)
        assert st == FD.FDFD_OK
        ref = s.solve(b)
        assert (torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)).item() <= TOL
    s.close()


def test_noalloc_rejects_oversized_solve():
    wl = W.make("c1")
    s = _solver(wl, FD.MODE_MIXED)
    limit = FD._lib.fdfd_noalloc_scratch_bytes()
    # the scratch holds one front vector per system: the summed front sizes in complex64
    # (8 bytes) each, plus the sweep counters; this many systems need more than the array
    k, m, *_ = s.plan_fronts()
    vec_total = int((k + m).sum())
    nrhs = 1 + limit // (8 * vec_total)
    b = torch.zeros((1, nrhs, wl.n), dtype=torch.complex128, device="cuda")
    st, _ = _noalloc(s, b, False)
    assert st == 1                               # FDFD_ERR_ARG
    assert "scratch" in FD._lib.fdfd_last_error(s._h).decode()
    s.close()


def test_noalloc_before_factor_is_state_error():
    wl = W.make_small(12, 12, 2, (3, 3, 4, 4), seed=2)
    s = FD.Solver(wl.nx, wl.ny, wl.dx, 2 * np.pi / wl.wavelengths, wl.npml, box=wl.box)
    b = torch.zeros((1, 1, wl.n), dtype=torch.complex128, device="cuda")
    st, _ = _noalloc(s, b, False)
    assert st == 2                               # FDFD_ERR_STATE
    s.close()


def test_noalloc_f64_matches_the_oracle():
    """On complex128 factors the raw sweeps are a direct solve: the no-allocation call reaches the
    oracle's SuperLU solution (forward and transpose) to 1e-10, twice in a row."""
    from oracle import fdfd_oracle as O
    wl = W.make_small(48, 41, 6, (12, 10, 20, 18), n_omega=2, n_src=1, seed=21)
    s = _solver(wl, FD.MODE_F64)
    eps = wl.eps_full()
    facs = [O.Factor(O.assemble(wl.nx, wl.ny, eps, k0dx, wl.npml), (wl.nx, wl.ny)) for k0dx in wl.k0dx()]
    for call, transpose in enumerate((False, True, False)):
        b = W.random_complex((wl.n_omega, 2, wl.n), 200 + call)
        st, x = _noalloc(s, torch.from_numpy(b).cuda(), transpose)
        assert st == FD.FDFD_OK, FD._lib.fdfd_last_error(s._h).decode()
        x = x.cpu().numpy()
        for w, fac in enumerate(facs):
            for r in range(2):
                ref = fac.solve_T(b[w, r]) if transpose else fac.solve(b[w, r])
                assert O.rel_err(x[w, r], ref) <= 1e-10, (call, w, r)
    s.close()


def test_noalloc_reports_a_wait_that_gave_up():
    """A bounded device wait that gave up before the call (the deferred self-test leaves the
    context's error word set, as a sweep that timed out would) is reported by the no-allocation
    call as FDFD_ERR_TIMEOUT; the word is then cleared and the next call solves normally."""
    wl = W.make("c1")
    s = _solver(wl, FD.MODE_MIXED)
    b = torch.from_numpy(wl.source_dense(0).reshape(1, 1, -1).copy()).cuda()
    st, _ = _noalloc(s, b, False)                # growth checked once, nothing pending
    assert st == FD.FDFD_OK
    assert s.selftest_wait_async() == FD.FDFD_OK
    torch.cuda.synchronize()
    st, _ = _noalloc(s, b, False)
    assert st == 7, FD._lib.fdfd_last_error(s._h).decode()     # FDFD_ERR_TIMEOUT
    st, x = _noalloc(s, b, False)
    assert st == FD.FDFD_OK
    ref = s.solve(b)
    assert (torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)).item() <= TOL
    s.close()
