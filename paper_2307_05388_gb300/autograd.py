"""torch.autograd.Functions over the cached solver (Sec. II, Eq. 3-6) and the
design parametrisation before it (Sec. III: smoothing filter and projection).

forward(eps_design): design refactor (or a full factorisation on the first
call), forward solves for all wavelengths and sources, mode-overlap objective
F and its adjoint source.  backward(dL/dF): transpose solves on the same
cached factors (no new factorisation, the paper's first caching idea) and the
pixel gradient kernel.  Every numerical step runs in libfdfd's kernels.
"""
from __future__ import annotations

import torch

from . import fdfd


class DesignProblem:
    """One adjoint design problem: solver, background permittivity, sources, monitors.

    eps_bg: float64 [nx*ny] (device); b: complex128 [n_omega, nrhs, nx*ny];
    cols: int32 [n_omega*nrhs] monitor columns; g: complex128 [n_omega*nrhs, ny]
    monitor profiles; weight: float64 [n_omega*nrhs] or None; target: float64
    [n_omega*nrhs] transmission targets or None.  Without targets F = sum w |o|^2;
    with them F = sum w (|o|^2 - target)^2, the squared transmission error that
    the paper's devices minimise (Sec. III-IV).
    """

    def __init__(self, solver: fdfd.Solver, eps_bg: torch.Tensor, b: torch.Tensor, cols: torch.Tensor,
                 g: torch.Tensor, weight: torch.Tensor | None = None, target: torch.Tensor | None = None):
        self.solver = solver
        self.eps_bg = eps_bg.reshape(-1).contiguous()
        self.b = b.contiguous()
        self.cols = cols.contiguous()
        self.g = g.contiguous()
        self.weight = weight
        self.target = target
        self.factored = False
        self.version = 0          # factorisations loaded so far (the backward pass checks it)
        x0, y0, w, h = solver.box
        self._box = (x0, y0, w, h)
        self.x = torch.empty_like(self.b)
        self.xa = torch.empty_like(self.b)

    def _load(self, eps_design: torch.Tensor):
        if not self.factored:
            x0, y0, w, h = self._box
            eps = self.eps_bg.clone().reshape(self.solver.nx, self.solver.ny)
            eps[x0:x0 + w, y0:y0 + h] = eps_design.reshape(w, h)
            self.solver.factor(eps.reshape(-1))
            self.factored = True
        else:
            self.solver.refactor_design(eps_design.reshape(-1).contiguous())
        self.version += 1

    def iteration(self, eps_design: torch.Tensor, grad_out: torch.Tensor | None = None,
                  accumulate: bool = False):
        """One forward + adjoint design iteration; returns (F, dF/deps_design [w*h]).  With
        accumulate the gradient is added to grad_out instead of overwriting it."""
        s = self.solver
        self._load(eps_design)
        s.solve(self.b, out=self.x)
        F, o, badj = s.objective(self.x, self.cols, self.g, self.weight, target=self.target)
        s.solve(badj, transpose=True, out=self.xa)
        # the adjoint source already carries the per-system weights
        g = s.grad(self.x, self.xa, None, out=grad_out, accumulate=accumulate)
        return F, g

    def __call__(self, eps_design: torch.Tensor) -> torch.Tensor:
        return FdfdObjective.apply(eps_design, self)


class FdfdObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_design: torch.Tensor, prob: DesignProblem):
        s = prob.solver
        prob._load(eps_design.detach())
        x = s.solve(prob.b)
        F, o, badj = s.objective(x, prob.cols, prob.g, prob.weight, target=prob.target)
        ctx.prob = prob
        ctx.version = prob.version
        ctx.save_for_backward(x, badj)
        ctx.shape = eps_design.shape
        return F

    @staticmethod
    def backward(ctx, gF: torch.Tensor):
        prob = ctx.prob
        if prob.version != ctx.version:
            # the adjoint solve needs the factors of this forward pass's permittivity
            raise RuntimeError("the solver was refactored after this forward pass; call backward before "
                               "evaluating the problem again")
        x, badj = ctx.saved_tensors
        s = prob.solver
        xa = s.solve(badj, transpose=True)
        nsys = prob.cols.numel()
        # the adjoint source already carries the per-system weights; only dL/dF scales here
        w = gF.reshape(1).to(torch.float64).expand(nsys).contiguous()
        g = s.grad(x, xa, w)
        return g.reshape(ctx.shape), None


class FilterProject(torch.autograd.Function):
    """Design density -> design-box permittivity through the conic smoothing filter and
    the tanh projection (Sec. III), with the chain rule back to the density; both
    directions run in libfdfd's kernels.  Use as eps = FilterProject.apply(rho, solver,
    radius, beta, eta, eps_lo, eps_hi), then F = problem(eps)."""

    @staticmethod
    def forward(ctx, rho: torch.Tensor, solver: fdfd.Solver, radius: float, beta: float, eta: float,
                eps_lo: float, eps_hi: float):
        eps, work = solver.filter_project(rho.detach(), radius, beta, eta, eps_lo, eps_hi)
        ctx.solver = solver
        ctx.radius = radius
        ctx.shape = rho.shape
        ctx.save_for_backward(work)
        return eps.reshape(rho.shape)

    @staticmethod
    def backward(ctx, g_eps: torch.Tensor):
        (work,) = ctx.saved_tensors
        g = ctx.solver.filter_project_adjoint(g_eps.to(torch.float64), work, ctx.radius)
        return g.reshape(ctx.shape), None, None, None, None, None, None
