"""Launch-parameter tuning and eigenmode sources on the GPU.

Autotuner: it measures real design iterations, its choice is the fastest admissible
candidate, the solver built with the chosen options still meets the field tolerance against
the oracle, and a second call reads the cache.

Eigenmode sources: a straight Si guide through the design box, fed by its TE0 and TE1 modes
and monitored by the same modes downstream; each side takes the modes from its own mode
solver.  Objective within 1e-8 and gradient within 1e-6 of the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fdfd_oracle as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import autograd as AG  # noqa: E402
from paper_2307_05388_gb300 import autotune as AT  # noqa: E402
from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402
from tests import _gpu_util as U  # noqa: E402


def test_autotune_c1(tmp_path):
    wl = W.make("c1")
    eps_bg = torch.from_numpy(wl.eps_bg.reshape(-1).copy()).cuda()
    cols, g = U.monitor_tensors(wl)
    b = U.rhs_tensor(wl)

    def make(opts):
        s = FD.Solver(wl.nx, wl.ny, wl.dx, U.k0_of(wl), wl.npml, box=wl.box, options=opts)
        return AG.DesignProblem(s, eps_bg, b, cols, g)

    path = str(tmp_path / "tune.json")
    search = (("tensor_form", (3, 2)), ("tensor_min_m", (128, 256)))   # 256: C1's fronts all SIMT
    res = AT.tune(make, U.eps_design_tensor(wl, wl.rho), search=search, steps=2, warmup=1, cache_path=path)
    ok = [t for t in res.trials if t.ok]
    print("autotune c1:", [(t.params, t.ms, t.status) for t in res.trials])
    assert ok and res.params in [t.params for t in ok]
    assert min(t.ms for t in ok) == [t.ms for t in ok if t.params == res.params][0]
    assert all(t.ms is not None and t.ms > 0 for t in ok)

    # the chosen options meet the field tolerance, forward and transpose
    s = FD.Solver(wl.nx, wl.ny, wl.dx, U.k0_of(wl), wl.npml, box=wl.box, options=res.options)
    eps = wl.eps_full()
    s.factor(torch.from_numpy(eps.reshape(-1).copy()).cuda())
    rhs = W.random_complex((wl.n_omega, 1, wl.n), 11)
    fac = O.Factor(O.assemble(wl.nx, wl.ny, eps, wl.k0dx()[0], wl.npml))
    for tr in (False, True):
        x = s.solve(torch.from_numpy(rhs).cuda(), transpose=tr).cpu().numpy()
        ref = fac.solve_T(rhs[0, 0]) if tr else fac.solve(rhs[0, 0])
        assert O.rel_err(x.reshape(-1), ref) <= 1e-8
    s.close()

    again = AT.tune(make, U.eps_design_tensor(wl, wl.rho), search=search, cache_path=path, key=res.key)
    assert again.cached and again.params == res.params
    np.testing.assert_equal(AT.options_dict(again.options), AT.options_dict(res.options))


def test_eigenmode_sources_and_mode_monitors():
    nx, ny, npml, dx, lam = 120, 70, 10, 0.04, 1.55
    k0dx = 2 * np.pi * dx / lam
    eps_line = np.full(ny, W.EPS_SIO2)
    eps_line[ny // 2 - 6:ny // 2 + 6] = W.EPS_SI          # 480 nm Si core
    eps = np.tile(eps_line, (nx, 1))
    box = (45, 20, 30, 30)
    rng = np.random.default_rng(31)
    rho = rng.uniform(0, 1, (box[2], box[3]))
    eps[box[0]:box[0] + box[2], box[1]:box[1] + box[3]] = W.EPS_SIO2 + W.DELTA_EPS * rho
    i_src, i_mon = 20, 98

    # CUDA path: modes from the library's solver, objective and gradient through the C ABI
    _, _, phi = FD.slab_modes(eps_line, k0dx, 2)
    n = nx * ny
    b = np.zeros((1, 2, nx, ny), complex)
    for m in range(2):
        b[0, m, i_src, :] = phi[m]
    s = FD.Solver(nx, ny, dx, [2 * np.pi / lam], npml, box=box, options=FD.default_options())
    eps_bg = torch.from_numpy(np.tile(eps_line, (nx, 1)).reshape(-1).copy()).cuda()
    cols = torch.full((2,), i_mon, dtype=torch.int32, device="cuda")
    g = torch.from_numpy(phi.astype(np.complex128)).cuda()
    prob = AG.DesignProblem(s, eps_bg, torch.from_numpy(b.reshape(1, 2, n)).cuda(), cols, g)
    eps_d = torch.from_numpy(np.ascontiguousarray(eps[box[0]:box[0] + box[2], box[1]:box[1] + box[3]]).reshape(-1)).cuda()
    F, grad = prob.iteration(eps_d)
    torch.cuda.synchronize()

    # oracle: its own modes, plain solves and Eq. 3-4
    _, _, phi_o = O.slab_modes(eps_line, k0dx, 2)
    fac = O.Factor(O.assemble(nx, ny, eps, k0dx, npml))
    F_ref, g_ref = 0.0, np.zeros((box[2], box[3]))
    for m in range(2):
        bm = np.zeros((nx, ny), complex)
        bm[i_src, :] = phi_o[m]
        gm = np.zeros((nx, ny), complex)
        gm[i_mon, :] = phi_o[m]
        E = fac.solve(bm.ravel())
        F_ref += abs(O.overlap(E, gm.ravel())) ** 2
        Ea = fac.solve_T(O.adjoint_source(E, gm.ravel()))
        g_ref += O.design_box_of(O.grad_eps(E, Ea, k0dx), nx, ny, box)
    print(f"mode transmission F {float(F):.6e} (oracle {F_ref:.6e})")
    assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
    assert O.rel_err(grad.cpu().numpy().reshape(box[2], box[3]), g_ref) <= 1e-6
    s.close()
