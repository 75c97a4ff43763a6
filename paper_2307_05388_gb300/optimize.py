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

import json
import os
import time
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


def linear_density_objective(prob, eps_lo: float, eps_hi: float):
    """F(rho) and dF/drho for the unfiltered design map eps = eps_lo + rho (eps_hi - eps_lo):
    the library's density map (fdfd_density_eps), one design iteration (refactor, forward solves,
    objective, adjoint solves, gradient) and the chain rule dF/drho = (eps_hi - eps_lo) dF/deps.

    prob: an autograd.DesignProblem; rho is the design-box density [w*h] (float64, device)."""
    scale = float(eps_hi) - float(eps_lo)

    def f(rho: torch.Tensor):
        eps = prob.solver.density_eps(rho, eps_lo, eps_hi)
        F, g = prob.iteration(eps)
        return F, g * scale
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


def _state_to(state, device):
    if isinstance(state, torch.Tensor):
        return state.to(device)
    if isinstance(state, dict):
        return {k: _state_to(v, device) for k, v in state.items()}
    return state


class DesignLoop:
    """The design loop rho <- optimizer.step(rho, dF/drho(rho)), with checkpoint / resume and one
    JSON record per iteration.

    objective(rho) -> (F, dF/drho) on rho's device (density_objective, linear_density_objective);
    optimizer: SignStep, Adam, or any object with step(rho, g), state_dict() and load_state_dict().

    checkpoint: a path.  Every `every` iterations the loop writes the iteration count, rho, the
    optimizer's state and the history of F there (torch.save to a temporary file, then an atomic
    rename, so that an interrupted write leaves the previous checkpoint).  The loop draws no random
    numbers, so that is all its state.  Factor caches are not saved: the first iteration after a
    resume factors from scratch (one analysis and one full factorisation in a new solver), after
    which the loop follows the same trajectory.  On the GPU, FGMRES sizes its first cycle from the
    previous solve, so a resumed loop agrees with an unbroken one to rounding, not bit for bit.

    log: a path.  One JSON object per iteration is appended to it: the iteration, F, the 2-norm of
    dF/drho, the wall time, and whatever stats() returns (for a solver: refinement iterations, the
    final residual, pivot growth, repivots, FP64 fallbacks).  After a resume the iterations since the
    last checkpoint appear twice, the second time as recomputed."""

    def __init__(self, objective: Callable[[torch.Tensor], tuple], optimizer, rho0: torch.Tensor,
                 checkpoint: str | None = None, every: int = 1, log: str | None = None,
                 stats: Callable[[], dict] | None = None):
        if every < 1:
            raise ValueError("every must be at least 1")
        self.objective = objective
        self.optimizer = optimizer
        self.rho = rho0.detach().clone()
        self.iteration = 0
        self.history: list = []
        self.checkpoint = checkpoint
        self.every = int(every)
        self.log = log
        self.stats = stats

    def run(self, iterations: int) -> torch.Tensor:
        """Runs that many more iterations; returns the current density."""
        for _ in range(int(iterations)):
            t0 = time.perf_counter()
            F, g = self.objective(self.rho)
            Fv = float(F)
            rec = {"iteration": self.iteration, "F": Fv, "grad_norm": float(torch.linalg.vector_norm(g))}
            self.rho = self.optimizer.step(self.rho, g)
            self.iteration += 1
            self.history.append(Fv)
            rec["seconds"] = time.perf_counter() - t0
            if self.log is not None:
                if self.stats is not None:
                    rec.update(self.stats())
                with open(self.log, "a") as fh:
                    fh.write(json.dumps(rec, default=float) + "\n")
            if self.checkpoint is not None and self.iteration % self.every == 0:
                self.save(self.checkpoint)
        return self.rho

    def save(self, path: str) -> None:
        state = {"iteration": self.iteration, "rho": self.rho.detach().cpu(),
                 "optimizer": _state_to(self.optimizer.state_dict(), "cpu"), "history": list(self.history)}
        tmp = f"{path}.tmp"
        torch.save(state, tmp)
        os.replace(tmp, path)

    @classmethod
    def resume(cls, path: str, objective: Callable[[torch.Tensor], tuple], optimizer,
               device: str | torch.device = "cpu", **kw) -> "DesignLoop":
        """A loop restored from a checkpoint: rho and the optimizer's state on `device`; kw as for
        the constructor (checkpoint, every, log, stats)."""
        state = torch.load(path, map_location="cpu")
        optimizer.load_state_dict(_state_to(state["optimizer"], device))
        loop = cls(objective, optimizer, state["rho"].to(device), **kw)
        loop.iteration = int(state["iteration"])
        loop.history = [float(v) for v in state["history"]]
        return loop
