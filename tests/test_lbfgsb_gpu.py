"""The multi-mode design loop on the GPU (Sec. III-IV: TE0/TE1 inputs at several wavelengths,
the squared difference between port transmissions and their targets minimised by L-BFGS-B over
the filtered and projected density).

A C3-sized problem (540 x 540 grid, 400 x 400 design box) restricted to two of its wavelengths,
fed by the TE0 and TE1 eigenmodes of its 1.2 um input guide (library mode solver on the GPU side,
the oracle's on the oracle side), each mode monitored at its own output port.  At the initial
density the objective and dF/drho through the smoothing filter, the projection and the solver
Function match the oracle (1e-8 / 1e-6); three L-BFGS-B iterations then lower the objective and
keep the density inside [0, 1]."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import autograd as AG  # noqa: E402
from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402
from paper_2307_05388_gb300 import optimize as OPT  # noqa: E402

RADIUS, BETA, ETA = 5.0, 8.0, 0.5       # 200 nm filter at dx = 40 nm
LO, HI = W.EPS_SIO2, W.EPS_SI


def _workload():
    return W.make("c3").select_wavelengths([0, 7])


def _targets(powers):
    # ask for half the TE0 power and one and a half times the TE1 power at every wavelength
    return [[powers[w][s] * (0.5 if s == 0 else 1.5) for s in range(2)] for w in range(len(powers))]


def _oracle_start(rho):
    """Oracle side: powers at the initial design, then F and dF/drho with the targets."""
    from oracle import fdfd_oracle as O
    wl = W.with_modes(_workload(), O.slab_modes)
    eps_d = O.filter_project(rho, RADIUS, BETA, ETA, LO, HI)
    rho_eps = (eps_d - LO) / W.DELTA_EPS
    _, _, fields = O.design_iteration(wl, rho_eps, wl.eps_full, W.DELTA_EPS)
    powers = [[abs(O.overlap(fields[(w, s)][0], wl.monitor_dense(w, s))) ** 2 for s in range(2)] for w in range(2)]
    F, g_rho_eps, _ = O.design_iteration(wl, rho_eps, wl.eps_full, W.DELTA_EPS, targets=_targets(powers))
    g = O.filter_project_grad(rho, g_rho_eps / W.DELTA_EPS, RADIUS, BETA, ETA, LO, HI)
    return F, g, powers


def test_lbfgsb_on_mode_transmission_targets_c3():
    from oracle import fdfd_oracle as O
    wl = W.with_modes(_workload(), FD.slab_modes)
    with cf.ProcessPoolExecutor(1, mp_context=mp.get_context("spawn")) as ex:
        job = ex.submit(_oracle_start, wl.rho.copy())
        dev = "cuda"
        k0 = 2 * np.pi / np.asarray(wl.wavelengths)
        s = FD.Solver(wl.nx, wl.ny, wl.dx, k0, wl.npml, box=wl.box)
        b = np.stack([np.stack([wl.source_dense(i, w) for i in range(2)]) for w in range(2)])
        cols = np.array([wl.monitors[w][i].col for w in range(2) for i in range(2)], np.int32)
        g = np.stack([wl.monitors[w][i].values for w in range(2) for i in range(2)]).astype(np.complex128)
        prob = AG.DesignProblem(s, torch.from_numpy(wl.eps_bg.reshape(-1).copy()).to(dev), torch.from_numpy(b).to(dev),
                                torch.from_numpy(cols).to(dev), torch.from_numpy(g).to(dev))
        # the powers at the initial design set the targets (the same rule on both sides)
        rho0 = torch.from_numpy(wl.rho.reshape(-1).copy()).to(dev)
        eps0 = AG.FilterProject.apply(rho0, s, RADIUS, BETA, ETA, LO, HI)
        prob.iteration(eps0.reshape(-1))
        _, o, _ = s.objective(prob.x, prob.cols, prob.g)
        p = (o.abs() ** 2).cpu().numpy().reshape(2, 2)
        prob.target = torch.tensor(_targets(p), dtype=torch.float64, device=dev).reshape(-1)
        f = OPT.density_objective(prob, RADIUS, BETA, ETA, LO, HI)
        F0, g0 = f(rho0)
        F_ref, g_ref, powers_ref = job.result()
    assert np.allclose(p, np.asarray(powers_ref), rtol=1e-8, atol=0)
    assert abs(float(F0) - F_ref) <= 1e-8 * abs(F_ref)
    assert O.rel_err(g0.cpu().numpy().reshape(wl.rho.shape), g_ref) <= 1e-6
    history = []
    rho, F, res = OPT.lbfgsb(f, rho0, maxiter=3, maximize=False, callback=lambda k, fv, x: history.append(fv))
    print(f"L-BFGS-B on C3 (2 wavelengths x TE0/TE1): F {float(F0):.4e} -> {F:.4e} in {res.nit} iterations, "
          f"{res.nfev} evaluations")
    assert F < 0.9 * float(F0)
    assert float(rho.min()) >= 0.0 and float(rho.max()) <= 1.0
    s.close()
