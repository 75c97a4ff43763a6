"""Seeded synthetic inputs for the 2D TM (Ez) FDFD inverse-design workloads.

This module only generates inputs: grids, wavelengths, design boxes, design
densities rho, background permittivity maps, source lines and monitor lines.
It holds none of the solver's arithmetic (no PML, no stencil, no solve, no
objective), so that both the CPU oracle and the CUDA path can consume the same
seeded inputs without sharing any computation.

Physical setting (Sec. III-V of the paper): silicon-on-oxide photonics,
wavelengths 1.50-1.60 um (1.31 um for one large case), footprints from 16 um^2
to over 7000 um^2.  The paper's own device geometries and target spectra are
not published, so seeded random design densities stand in for them.

Units: lengths in micrometres.  Cell (i, j) has its centre at
((i + 0.5) dx, (j + 0.5) dx); the flat unknown index is n = i * ny + j.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EPS_SIO2 = 2.085   # relative permittivity of the oxide cladding (background)
EPS_SI = 12.11     # relative permittivity of silicon
DELTA_EPS = EPS_SI - EPS_SIO2


@dataclass
class Line:
    """A vector supported on one grid column: values[j] at cell (col, j)."""
    col: int
    values: np.ndarray          # complex128 [ny]


@dataclass
class ModeLine:
    """A guided-mode source on one grid column: amplitude * phi_mode[j] at cell (col, j), where
    phi_mode is the mode-th guided mode (0 = TE0, 1 = TE1, ...) of the cross-section eps_line at
    each wavelength.  The profile is not computed here: each consumer resolves it with its own
    mode solver (with_modes)."""
    col: int
    eps_line: np.ndarray        # float64 [ny]
    mode: int
    amplitude: complex = -1j


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float                   # um
    npml: int                   # PML cells on every side, counted inside nx, ny
    wavelengths: np.ndarray     # float64 [n_omega], um
    box: tuple                  # design box (x0, y0, w, h) in cells
    eps_bg: np.ndarray          # float64 [nx, ny], permittivity outside the design box
    rho: np.ndarray             # float64 [w, h] initial design density in [0, 1]
    sources: list               # [n_src] Line (same at every wavelength) or ModeLine (resolved per wavelength)
    monitors: list              # [n_omega][n_src] Line: overlap weights g
    iterations: int
    optimizer: str              # "sign" or "adam"
    step: float
    seed: int
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def n_omega(self) -> int:
        return len(self.wavelengths)

    @property
    def n_src(self) -> int:
        return len(self.sources)

    def k0dx(self) -> np.ndarray:
        """Free-space wavenumber times the cell size, per wavelength."""
        return 2.0 * np.pi * self.dx / np.asarray(self.wavelengths, dtype=np.float64)

    def eps_design(self, rho: np.ndarray | None = None) -> np.ndarray:
        """Permittivity of the design pixels: eps_SiO2 + rho * (eps_Si - eps_SiO2)."""
        r = self.rho if rho is None else rho
        return EPS_SIO2 + np.asarray(r, dtype=np.float64) * DELTA_EPS

    def eps_full(self, rho: np.ndarray | None = None) -> np.ndarray:
        """Full permittivity map [nx, ny]: background with the design box filled in."""
        x0, y0, w, h = self.box
        eps = self.eps_bg.copy()
        eps[x0:x0 + w, y0:y0 + h] = self.eps_design(rho)
        return eps

    def source_line(self, s: int, w: int = 0) -> Line:
        src = self.sources[s]
        if isinstance(src, ModeLine):
            prof = self.extra.get("mode_profiles")
            if prof is None:
                raise ValueError("mode sources not resolved: call with_modes(workload, mode_solver) first")
            return Line(src.col, src.amplitude * prof[(s, w)])
        return src

    def source_dense(self, s: int, w: int = 0) -> np.ndarray:
        """Source s at wavelength w as a dense complex128 vector of length nx*ny (flat n = i*ny + j)."""
        return line_dense(self.source_line(s, w), self.nx, self.ny)

    def select_wavelengths(self, ws) -> "Workload":
        """A copy restricted to the listed wavelengths (resolved mode profiles follow)."""
        import copy
        out = copy.copy(self)
        ws = list(ws)
        out.wavelengths = np.asarray(self.wavelengths)[ws]
        out.monitors = [self.monitors[w] for w in ws]
        out.extra = dict(self.extra)
        prof = self.extra.get("mode_profiles")
        if prof is not None:
            out.extra["mode_profiles"] = {(s, i): prof[(s, w)] for i, w in enumerate(ws)
                                          for s in range(self.n_src) if (s, w) in prof}
        return out

    def monitor_dense(self, w: int, s: int) -> np.ndarray:
        return line_dense(self.monitors[w][s], self.nx, self.ny)


def line_dense(line: Line, nx: int, ny: int) -> np.ndarray:
    v = np.zeros((nx, ny), dtype=np.complex128)
    v[line.col, :] = line.values
    return v.reshape(-1)


def box_blur(a: np.ndarray, k: int) -> np.ndarray:
    """k x k box mean with edge replication; window offsets [-(k//2), k - k//2 - 1]."""
    lo = k // 2
    hi = k - lo - 1
    p = np.pad(a, ((lo, hi + 1), (lo, hi + 1)), mode="edge")
    c = np.cumsum(np.cumsum(p, axis=0), axis=1)
    c = np.pad(c, ((1, 0), (1, 0)))
    w, h = a.shape
    s = c[k:k + w, k:k + h] - c[0:w, k:k + h] - c[k:k + w, 0:h] + c[0:w, 0:h]
    return s / float(k * k)


def gaussian_profile(ny: int, dx: float, center: float, w0: float, lo: int, hi: int) -> np.ndarray:
    """exp(-((y - center)/w0)^2) on rows [lo, hi), zero elsewhere; y = (j + 0.5) dx."""
    y = (np.arange(ny) + 0.5) * dx
    g = np.exp(-((y - center) / w0) ** 2)
    g[:lo] = 0.0
    g[hi:] = 0.0
    return g


def with_modes(wl: Workload, mode_solver) -> Workload:
    """A copy of wl whose ModeLine sources are resolved at every wavelength by
    mode_solver(eps_line, k0dx, n_modes) -> (mu, theta, phi) (the library's slab_modes or the
    oracle's: each side brings its own).  phi[mode] becomes the source profile."""
    import copy
    out = copy.copy(wl)
    out.extra = dict(wl.extra)
    prof = {}
    for s, src in enumerate(wl.sources):
        if not isinstance(src, ModeLine):
            continue
        for w, k0dx in enumerate(wl.k0dx()):
            _, _, phi = mode_solver(src.eps_line, float(k0dx), src.mode + 1)
            prof[(s, w)] = np.asarray(phi[src.mode], dtype=np.float64).copy()
    out.extra["mode_profiles"] = prof
    return out


def _centred_box(nx: int, ny: int, w: int, h: int) -> tuple:
    return ((nx - w) // 2, (ny - h) // 2, w, h)


def _blurred_rho(rng: np.random.Generator, w: int, h: int) -> np.ndarray:
    return np.clip(box_blur(rng.uniform(0.0, 1.0, size=(w, h)), 8), 0.0, 1.0)


def _stub_eps(nx: int, ny: int, npml: int, box: tuple, dx: float, width_um: float) -> np.ndarray:
    """Background with Si waveguide stubs from the PML edges to the design box, centred in y."""
    eps = np.full((nx, ny), EPS_SIO2)
    x0, y0, w, h = box
    wc = int(round(width_um / dx / 2.0)) * 2          # even number of cells
    jc = ny // 2
    eps[npml:x0, jc - wc // 2:jc + wc // 2] = EPS_SI
    eps[x0 + w:nx - npml, jc - wc // 2:jc + wc // 2] = EPS_SI
    return eps


def make(name: str, seed: int = 0, grid: int | None = None, design: int | None = None) -> Workload:
    """The five seeded workloads, by name: 'c1' .. 'c5' (sizes in each docstring line).

    For c2 .. c5, grid and design (cells) replace the square grid's and the centred design box's
    sizes while dx, the PML, the wavelengths, sources, monitors and optimiser stay those of the
    workload: the same recipe at a size a test's oracle finishes in seconds."""
    rng = np.random.default_rng(seed)
    name = name.lower()
    if name == "c1":
        # 4x4 um + 10-cell PML at dx = 50 nm (100x100), lambda 1.55 um, 40x40 centred design.
        nx = ny = 100
        dx, npml = 0.05, 10
        box = _centred_box(nx, ny, 40, 40)
        rho = rng.uniform(0.0, 1.0, size=(40, 40))
        eps_bg = np.full((nx, ny), EPS_SIO2)
        src = Line(npml, np.where((np.arange(ny) >= npml) & (np.arange(ny) < ny - npml), -1j, 0j))
        g = gaussian_profile(ny, dx, ny * dx / 2, 0.5, npml, ny - npml).astype(np.complex128)
        mons = [[Line(nx - npml - 1, g)]]
        return Workload("c1", nx, ny, dx, npml, np.array([1.55]), box, eps_bg, rho, [src], mons,
                        iterations=5, optimizer="sign", step=0.05, seed=seed,
                        notes="line source on the first non-PML column; Gaussian monitor (w0 0.5 um)")
    if name in ("c2", "c3", "c4", "c5"):
        if name == "c2":
            nx, dx, npml, dsz = 340, 0.04, 20, 250
            wls = np.array([1.55])
            modes, iters, opt, step = 1, 50, "sign", 0.05
        elif name == "c3":
            nx, dx, npml, dsz = 540, 0.04, 20, 400
            wls = np.linspace(1.50, 1.60, 8)
            modes, iters, opt, step = 2, 30, "sign", 0.05
        elif name == "c4":
            nx, dx, npml, dsz = 1040, 0.04, 20, 900
            wls = np.linspace(1.53, 1.57, 4)
            modes, iters, opt, step = 1, 200, "adam", 0.01
        else:
            nx, dx, npml, dsz = 1760, 0.05, 20, 1680
            wls = np.array([1.31, 1.55])
            modes, iters, opt, step = 2, 20, "sign", 0.05
        if grid is not None or design is not None:
            nx, dsz = grid or nx, design or dsz
            if not 0 < dsz <= nx - 2 * npml - 4:
                raise ValueError(f"design {dsz} does not fit a {nx}-cell grid with {npml} PML cells")
            name = f"{name}@{nx}"
        ny = nx
        box = _centred_box(nx, ny, dsz, dsz)
        rho = _blurred_rho(rng, dsz, dsz)
        eps_bg = _stub_eps(nx, ny, npml, box, dx, 0.5 if modes == 1 else 1.2)
        yc = ny * dx / 2
        lo, hi = npml, ny - npml
        if modes == 1:
            srcs = [Line(npml, -1j * gaussian_profile(ny, dx, yc, 0.5, lo, hi))]
        else:
            # TE0 / TE1 of the 1.2 um input guide, launched on the first non-PML column
            srcs = [ModeLine(npml, eps_bg[npml].copy(), m) for m in range(modes)]
        nw = len(wls)
        if name.startswith("c3"):
            # 8 Gaussian ports evenly on the right monitor column; port 2*(l//2) + m.
            span = (hi - lo) * dx
            centres = lo * dx + span * (np.arange(8) + 0.5) / 8.0
            mons = [[Line(nx - npml - 1, gaussian_profile(ny, dx, centres[2 * (l // 2) + m], 0.5,
                                                          lo, hi).astype(np.complex128))
                     for m in range(modes)] for l in range(nw)]
        else:
            g = gaussian_profile(ny, dx, yc, 0.5, lo, hi).astype(np.complex128)
            mons = [[Line(nx - npml - 1, g) for _ in range(modes)] for _ in range(nw)]
        return Workload(name, nx, ny, dx, npml, wls, box, eps_bg, rho, srcs, mons,
                        iterations=iters, optimizer=opt, step=step, seed=seed)
    raise ValueError(f"unknown workload {name!r}")


def make_small(nx: int, ny: int, npml: int, box: tuple, n_omega: int = 1, n_src: int = 1,
               seed: int = 0, dx: float = 0.05, wl: float = 1.55) -> Workload:
    """A small seeded workload of arbitrary shape for parity tests (ragged, non-square)."""
    rng = np.random.default_rng(seed)
    x0, y0, w, h = box
    rho = rng.uniform(0.0, 1.0, size=(w, h))
    eps_bg = np.full((nx, ny), EPS_SIO2)
    eps_bg += 0.5 * rng.uniform(0.0, 1.0, size=(nx, ny))
    wls = wl + 0.05 * np.arange(n_omega)
    srcs = []
    for s in range(n_src):
        v = rng.standard_normal(ny) + 1j * rng.standard_normal(ny)
        srcs.append(Line(min(npml + s, nx - 1), v))
    mons = [[Line(max(nx - npml - 1 - s, 0), rng.standard_normal(ny) + 0j) for s in range(n_src)]
            for _ in range(n_omega)]
    return Workload(f"small{nx}x{ny}", nx, ny, dx, npml, wls, box, eps_bg, rho, srcs, mons,
                    iterations=1, optimizer="sign", step=0.05, seed=seed)


def random_complex(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
