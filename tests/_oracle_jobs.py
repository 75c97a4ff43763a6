"""Oracle work for the full-size GPU tests, run in spawned worker processes.

Each job rebuilds its seeded workload from the name, keeps one wavelength and
returns plain NumPy arrays, so a test can start the CPU oracle before its GPU
work and collect the results afterwards.  Imports only the workload generators
and the oracle (no torch, no CUDA)."""
from __future__ import annotations

import os

# up to four jobs run at once: each takes a quarter of the host cores for its BLAS
os.environ.setdefault("OPENBLAS_NUM_THREADS", str(max(1, (os.cpu_count() or 4) // 4)))
os.environ.setdefault("OMP_NUM_THREADS", os.environ["OPENBLAS_NUM_THREADS"])

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import fdfd_oracle as O  # noqa: E402


def one_wavelength(name: str, w: int, seed: int = 0):
    """The workload at wavelength w only, mode sources resolved by the oracle's mode solver."""
    return W.with_modes(W.make(name, seed=seed), O.slab_modes).select_wavelengths([w])


def rhs_of(wl, random_seed: int | None) -> np.ndarray:
    """[k, N]: the workload's sources at its (single) wavelength, then one seeded random vector."""
    rows = [wl.source_dense(s, 0) for s in range(wl.n_src)]
    if random_seed is not None:
        rows.append(W.random_complex(wl.n, random_seed))
    return np.stack(rows)


def fields(name: str, w: int, random_seed: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Forward and transpose SuperLU solutions A x = b, A^T x = b at wavelength w of the workload's
    initial design, for every row of rhs_of (sources built with the oracle's own mode solver)."""
    wl = one_wavelength(name, w)
    fac = O.Factor(O.assemble(wl.nx, wl.ny, wl.eps_full(), wl.k0dx()[0], wl.npml), (wl.nx, wl.ny))
    rhs = rhs_of(wl, random_seed)
    return (np.stack([fac.solve(b) for b in rhs]), np.stack([fac.solve_T(b) for b in rhs]))


def pixel_differences(name: str, w: int, pixels: np.ndarray, h: float) -> np.ndarray:
    """Wavelength w's share of the central differences of F at the listed design pixels (F sums
    over wavelengths, so the shares add up to the workload's differences)."""
    wl = one_wavelength(name, w)
    return O.objective_pixel_differences(wl, wl.rho, pixels, h, W.DELTA_EPS)
