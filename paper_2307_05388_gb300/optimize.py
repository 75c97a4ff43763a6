"""Optimisation loops over the design density.

* L-BFGS-B with box bounds (Sec. III runs its multi-mode devices with a quasi-Newton optimiser
  under 0 <= rho <= 1), on the host.
* The per-step updates of the seeded workloads' loops, on the density's own device: a sign step,
  and Adam with the box clip (the differentiable 1040^2, four-wavelength loop).

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


class SignStep:
    """Ascent by a fixed step along the sign of the gradient, clipped to the box:
    rho <- clip(rho + step sign(dF/drho), lo, hi), sign(0) = 0.  The loop of the workloads that
    name no optimiser of their own."""

    def __init__(self, step: float, bounds: tuple = (0.0, 1.0)):
        self.step_size = float(step)
        self.bounds = bounds

    def step(self, rho: torch.Tensor, grad: torch.Tensor) -> torch.Tensor:
        """The next density, a new tensor on rho's device (rho is not modified)."""
        return torch.clamp(rho + self.step_size * torch.sign(grad), *self.bounds)

    def state_dict(self) -> dict:
        return {}

    def load_state_dict(self, state: dict) -> None:
        pass


class Adam:
    """Adam (Kingma and Ba, 2015) on the design density, clipped to the box after every step.

    With t counting the steps taken:
        m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
        rho <- clip(rho + lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), lo, hi),
    g = dF/drho when maximising (the design objectives here), -dF/drho otherwise.  The moments
    live on rho's device, so a device loop moves nothing to the host.  The first step moves every
    pixel by lr sign(g) (for |g| >> eps); at a constant gradient every step moves lr until the
    bound."""

    def __init__(self, lr: float, betas: tuple = (0.9, 0.999), eps: float = 1e-8,
                 maximize: bool = True, bounds: tuple = (0.0, 1.0)):
        self.lr = float(lr)
        self.b1, self.b2 = (float(b) for b in betas)
        self.eps = float(eps)
        self.maximize = maximize
        self.bounds = bounds
        self.t = 0
        self.m = self.v = None

    def step(self, rho: torch.Tensor, grad: torch.Tensor) -> torch.Tensor:
        """The next density, a new tensor on rho's device (rho is not modified)."""
        g = grad if self.maximize else -grad
        if self.m is None:
            self.m = torch.zeros_like(rho)
            self.v = torch.zeros_like(rho)
        self.t += 1
        self.m.mul_(self.b1).add_(g, alpha=1.0 - self.b1)
        self.v.mul_(self.b2).addcmul_(g, g, value=1.0 - self.b2)
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return torch.clamp(rho + self.lr * mh / (torch.sqrt(vh) + self.eps), *self.bounds)

    def state_dict(self) -> dict:
        """Step count and moments, for a checkpoint of the design loop."""
        return {"t": self.t, "m": self.m, "v": self.v}

    def load_state_dict(self, state: dict) -> None:
        self.t = int(state["t"])
        self.m = None if state["m"] is None else state["m"].clone()
        self.v = None if state["v"] is None else state["v"].clone()


def design_optimizer(kind: str, step: float):
    """The design loop's update by name: 'sign' (SignStep(step)) or 'adam' (Adam(lr=step))."""
    if kind == "sign":
        return SignStep(step)
    if kind == "adam":
        return Adam(step)
    raise ValueError(f"unknown optimiser {kind!r}")
