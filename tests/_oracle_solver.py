"""A stand-in for fdfd.Solver backed by the CPU oracle, for host-logic tests without a GPU.

It answers the binding's calls (factor, refactor_design, solve, objective, grad,
filter_project, filter_project_adjoint, stats, close) with the oracle's plain definitions on
CPU tensors, so that the Python layers above the C ABI (autograd Functions, the L-BFGS-B loop)
can be exercised on the CPU.  Test infrastructure only."""
import numpy as np
import torch

from oracle import fdfd_oracle as O


class OracleSolver:
    def __init__(self, nx, ny, dx, k0, npml, box, options=None):
        self.nx, self.ny, self.dx, self.npml, self.box = nx, ny, dx, npml, tuple(box)
        self.k0 = np.atleast_1d(np.asarray(k0, float))
        self.n_omega = len(self.k0)
        self.options = options

    @property
    def n(self):
        return self.nx * self.ny

    def factor(self, eps):
        self.eps = eps.detach().reshape(self.nx, self.ny).numpy().copy()
        self.facs = [O.Factor(O.assemble(self.nx, self.ny, self.eps, k * self.dx, self.npml), (self.nx, self.ny))
                     for k in self.k0]

    def refactor_design(self, eps_design):
        x0, y0, w, h = self.box
        self.eps[x0:x0 + w, y0:y0 + h] = eps_design.detach().reshape(w, h).numpy()
        self.factor(torch.from_numpy(self.eps))

    def solve(self, b, transpose=False, out=None, allow_not_converged=False):
        bb = b.numpy().reshape(self.n_omega, -1, self.n)
        x = np.stack([np.stack([(f.solve_T if transpose else f.solve)(bb[w, r]) for r in range(bb.shape[1])])
                      for w, f in enumerate(self.facs)]).reshape(b.shape)
        t = torch.from_numpy(x)
        if out is not None:
            out.copy_(t)
            return out
        return t

    def objective(self, x, cols, g, weight=None, with_adjoint=True, target=None):
        xx = x.numpy().reshape(self.n_omega, -1, self.nx, self.ny)
        nrhs = xx.shape[1]
        F, badj, o = 0.0, np.zeros_like(xx), []
        for s in range(self.n_omega * nrhs):
            w, r = divmod(s, nrhs)
            c, gs = int(cols[s]), g[s].numpy()
            ov = np.sum(gs * xx[w, r, c])
            wt = 1.0 if weight is None else float(weight[s])
            if target is None:
                F += wt * abs(ov) ** 2
                badj[w, r, c] = wt * np.conj(ov) * gs
            else:
                F += O.target_objective(ov, float(target[s]), wt)
                badj[w, r, c] = 2.0 * wt * (abs(ov) ** 2 - float(target[s])) * np.conj(ov) * gs
            o.append(ov)
        return torch.tensor(F, dtype=torch.float64), torch.tensor(np.array(o)), torch.from_numpy(badj.reshape(x.shape))

    def grad(self, x_fwd, x_adj, weight=None, out=None, accumulate=False):
        a = x_fwd.numpy().reshape(self.n_omega, -1, self.n)
        b = x_adj.numpy().reshape(a.shape)
        nrhs = a.shape[1]
        g = np.zeros((self.box[2], self.box[3]))
        for w in range(self.n_omega):
            for r in range(nrhs):
                wt = 1.0 if weight is None else float(weight[w * nrhs + r])
                g += wt * O.design_box_of(O.grad_eps(a[w, r], b[w, r], self.k0[w] * self.dx), self.nx, self.ny, self.box)
        t = torch.from_numpy(g.reshape(-1).copy())
        if out is not None:
            if accumulate:
                out.add_(t)
            else:
                out.copy_(t)
            return out
        return t

    def density_eps(self, rho, eps_lo, eps_hi, out=None):
        eps = eps_lo + rho.reshape(-1) * (eps_hi - eps_lo)
        if out is not None:
            out.copy_(eps)
            return out
        return eps

    def filter_project(self, rho, radius, beta, eta, eps_lo, eps_hi):
        w, h = self.box[2], self.box[3]
        r = rho.detach().reshape(w, h).numpy()
        self._fp = (r.copy(), beta, eta, eps_lo, eps_hi)
        eps = O.filter_project(r, radius, beta, eta, eps_lo, eps_hi)
        return torch.from_numpy(eps.reshape(-1).copy()), torch.zeros(2 * w * h, dtype=torch.float64)

    def filter_project_adjoint(self, g_eps, work, radius):
        r, beta, eta, lo, hi = self._fp
        g = O.filter_project_grad(r, g_eps.detach().reshape(r.shape).numpy(), radius, beta, eta, lo, hi)
        return torch.from_numpy(g.reshape(-1).copy())

    def stats(self):
        return dict(fallbacks=0, ir_resid=0.0, ir_iters=0, growth=1.0)

    def close(self):
        pass
