"""Helpers for the GPU tests: build device tensors and a DesignProblem from a Workload."""
import numpy as np
import torch

import workloads as W

from paper_2307_05388_gb300 import autograd as AG
from paper_2307_05388_gb300 import fdfd as FD


def k0_of(wl):
    return 2 * np.pi / np.asarray(wl.wavelengths, dtype=np.float64)


def make_solver(wl, **opts):
    return FD.Solver(wl.nx, wl.ny, wl.dx, k0_of(wl), wl.npml, box=wl.box, options=FD.default_options(**opts))


def rhs_tensor(wl, dev="cuda"):
    """[n_omega, n_src, N] complex128: every source at every wavelength (mode sources resolved per
    wavelength by the library's mode solver)."""
    if any(isinstance(src, W.ModeLine) for src in wl.sources) and "mode_profiles" not in wl.extra:
        wl = W.with_modes(wl, FD.slab_modes)
    b = np.stack([np.stack([wl.source_dense(s, w) for s in range(wl.n_src)]) for w in range(wl.n_omega)])
    return torch.from_numpy(b).to(dev)


def monitor_tensors(wl, dev="cuda"):
    cols = np.array([wl.monitors[w][s].col for w in range(wl.n_omega) for s in range(wl.n_src)], np.int32)
    g = np.stack([wl.monitors[w][s].values for w in range(wl.n_omega) for s in range(wl.n_src)])
    return torch.from_numpy(cols).to(dev), torch.from_numpy(g.astype(np.complex128)).to(dev)


def problem(wl, dev="cuda", **opts):
    s = make_solver(wl, **opts)
    eps_bg = torch.from_numpy(wl.eps_bg.reshape(-1).copy()).to(dev)
    cols, g = monitor_tensors(wl, dev)
    return AG.DesignProblem(s, eps_bg, rhs_tensor(wl, dev), cols, g)


def eps_design_tensor(wl, rho, dev="cuda"):
    return torch.from_numpy(np.ascontiguousarray(wl.eps_design(rho)).reshape(-1)).to(dev)
