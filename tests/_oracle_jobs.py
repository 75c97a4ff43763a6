"""Oracle work for the full-size GPU tests, run in spawned worker processes.

Each job rebuilds its seeded workload from the name, keeps one wavelength and
returns plain NumPy arrays, so a test can start the CPU oracle before its GPU
work and collect the results afterwards.  Imports only the workload generators
and the oracle (no torch, no CUDA)."""
from __future__ import annotations

import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import fdfd_oracle as O  # noqa: E402


def one_wavelength(name: str, w: int, seed: int = 0):
    wl = W.make(name, seed=seed)
    wl.wavelengths = wl.wavelengths[w:w + 1]
    wl.monitors = wl.monitors[w:w + 1]
    return wl


def fields(name: str, w: int, rhs: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Forward and transpose SuperLU solutions A x = b, A^T x = b at wavelength w of the workload's
    initial design, for every row of rhs ([k, N])."""
    wl = one_wavelength(name, w)
    fac = O.Factor(O.assemble(wl.nx, wl.ny, wl.eps_full(), wl.k0dx()[0], wl.npml))
    return (np.stack([fac.solve(b) for b in rhs]), np.stack([fac.solve_T(b) for b in rhs]))


def pixel_differences(name: str, w: int, pixels: np.ndarray, h: float) -> np.ndarray:
    """Wavelength w's share of the central differences of F at the listed design pixels (F sums
    over wavelengths, so the shares add up to the workload's differences)."""
    wl = one_wavelength(name, w)
    return O.objective_pixel_differences(wl, wl.rho, pixels, h, W.DELTA_EPS)
