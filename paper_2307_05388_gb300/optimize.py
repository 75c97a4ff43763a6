"""Host optimisation loop over the design density: L-BFGS-B with box bounds (Sec. III runs its
multi-mode devices with a quasi-Newton optimiser under 0 <= rho <= 1).

The objective and its gradient are evaluated on the device by the caller's chain, for example
``density_objective`` below: filter + projection, design refactor, forward solves, objective,
transpose solves, pixel gradient, chain rule back to the density.  Each evaluation moves the
density to the device and F and dF/drho back (8 bytes per pixel each way).  L-BFGS-B itself
(SciPy's implementation) runs on the host; its work per step is O(pixels x memory), small next
to the solves.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import torch


def density_objective(prob, radius: float, beta: float, eta: float, eps_lo: float, eps_hi: float):
    """F(rho) and dF/drho through FilterProject and FdfdObjective (both in libfdfd's kernels).

    prob: an autograd.DesignProblem; rho is the design-box density [w*h] (float64, device)."""
    from .autograd import FilterProject

    def f(rho: torch.Tensor):
        rho = rho.detach().clone().requires_grad_(True)
        eps = FilterProject.apply(rho, prob.solver, radius, beta, eta, eps_lo, eps_hi)
        F = prob(eps)
        F.backward()
        return F.detach(), rho.grad.detach()
    return f


def lbfgsb(objective: Callable[[torch.Tensor], tuple], rho0: torch.Tensor, maxiter: int = 20,
           bounds: tuple = (0.0, 1.0), maximize: bool = True, memory: int = 10,
           callback: Callable[[int, float, np.ndarray], None] | None = None):
    """Runs L-BFGS-B on objective(rho) -> (F, dF/drho) from rho0 (a device tensor).

    maximize: ascend F (the mode-transmission objectives); else descend.
    Returns (rho as a device tensor shaped like rho0, best F, SciPy's result object)."""
    from scipy.optimize import minimize

    shape, dev = rho0.shape, rho0.device
    sign = -1.0 if maximize else 1.0
    history = []

    def fun(x: np.ndarray):
        rho = torch.from_numpy(x.reshape(shape)).to(dev)
        F, g = objective(rho)
        Fv = float(F)
        gv = g.detach().to("cpu", torch.float64).numpy().reshape(-1)
        history.append(Fv)
        return sign * Fv, sign * gv

    def cb(xk):
        if callback is not None:
            callback(len(history), history[-1], xk)

    x0 = rho0.detach().to("cpu", torch.float64).numpy().reshape(-1).copy()
    res = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=[bounds] * x0.size, callback=cb,
                   options={"maxiter": maxiter, "maxcor": memory})
    rho = torch.from_numpy(res.x.reshape(shape)).to(dev)
    return rho, sign * float(res.fun), res
