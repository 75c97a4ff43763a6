"""CPU oracle for the FDFD design-iteration hot path (complex128, SciPy SuperLU).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
definition that the CUDA path is checked against.  Only the test suite, the
smoke check of the package entry file and the CPU-baseline leg of the
benchmark may import it.  The product path never calls it and shares no code
with it: it is written from the paper's equations, not from the CUDA sources.

What it computes (paper, Sec. II):
  * Eq. 1-2: the 2D TM (Ez) frequency-domain operator
        (-omega^2 eps0 eps_r + mu0^-1 curl curl) E = -i omega J
    discretised on a Yee grid with stretched-coordinate PML.  Multiplying by
    mu0 dx^2 gives the dimensionless operator used throughout:
        A = -dx^2 Lap_s - (k0 dx)^2 diag(eps_r),  k0 = omega / c,
    where Lap_s is the PML-stretched 5-point Laplacian with a zero (PEC)
    field one cell beyond the grid on every side.
  * Eq. 5: E = A^-1 b by a direct sparse LU (SuperLU is the library step).
  * Eq. 4 and 6: the adjoint solve A^T E_adj = (dF/dE)^T on the same factor.
  * Eq. 3: dF/dtheta_i = -2 Re{E_adj^T (dA/dtheta_i) E}; with
    dA/deps_p = -(k0 dx)^2 e_p e_p^T this is 2 (k0 dx)^2 Re(E_adj[p] E[p]).
  * Objective: mode overlap o = g^T E on a monitor line, F = sum |o|^2, whose
    Wirtinger derivative (E* held fixed) gives dF/dE = conj(o) g^T.

Readings where the paper is silent (it gives no discretisation): Yee 5-point
stencil, eps sampled at Ez nodes, PEC behind the PML, polynomial grading m = 3
with target reflection R = 1e-8, PML cells counted inside the grid, e^{+i w t}
time convention (from the -i omega J right-hand side of Eq. 1), so that
s = 1 - i sigma / (omega eps0) absorbs outgoing waves.

Design parametrisation before the hot path (Sec. III: a smoothing filter of
200 nm radius and a sigmoid-like projection binarise the geometry; the paper
gives neither formula, so the usual forms are read in): a conic density filter
rho~_i = sum_j w_ij rho_j / sum_j w_ij with w_ij = max(0, R - |x_i - x_j|)
(distances in cells, sums over the design box), the tanh projection
rho^ = (tanh(b e) + tanh(b (rho~ - e))) / (tanh(b e) + tanh(b (1 - e))),
eps = eps_lo + rho^ (eps_hi - eps_lo), and the chain rule back to rho.

Eigenmode sources (Sec. III's multi-mode devices): guided modes of an
x-invariant cross-section eps(y) as eigenvectors of the y-part of the same
stencil (slab_modes).

Pins (tests/test_oracle.py): dense LAPACK solve on small grids, plane-wave
dispersion of the Yee stencil, plate-mode propagation constant and PML
absorption, reciprocity of the symmetrised operator, the bilinear transpose
identity, manufactured solutions, and central finite differences of F; for
the PML constants, the textbook normal-incidence reflection integral of the
graded layer (exact by Simpson's rule) and the decay of a guided wave inside
the layer; for the modes, the closed-form spectrum of a uniform line, the
continuum slab dispersion relation (second-order convergence), the mode count
of the slab's V number, and propagation of a mode through the 2D operator; for
the optimiser updates, closed forms of the sign step and of Adam's first,
second and constant-gradient steps; for the rank-one finite differences, the
plain definition (refactoring the perturbed operator).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

LN_R_DEFAULT = float(np.log(1e-8))
PML_ORDER_DEFAULT = 3.0


# ---------------------------------------------------------------------------
# Eq. 1-2: stretched-coordinate PML and the discrete operator
# ---------------------------------------------------------------------------
def pml_stretch(n: int, npml: int, k0dx: float, ln_R: float = LN_R_DEFAULT,
                order: float = PML_ORDER_DEFAULT):
    """Stretch factors s along one axis of n cells.

    Positions are in cell units: the domain spans [0, n], cell i has its centre
    at i + 0.5, and the half point between cells i and i+1 sits at i + 1.  The
    PML layer on each side is npml cells thick; depth d in [0, 1] grows
    polynomially toward the outer wall:
        sigma / (omega eps0) = -(order + 1) ln(R) / (2 k0dx npml) * d^order
        s = 1 - i sigma / (omega eps0).
    Returns (s_c, s_h): s_c[i] at cell centres (length n) and s_h[t] at the
    half points t = 0..n (s_h[t] lies between cells t-1 and t).
    """
    def s_at(u):
        u = np.asarray(u, dtype=np.float64)
        if npml <= 0:
            return np.ones_like(u, dtype=np.complex128)
        d = np.maximum(np.maximum(npml - u, u - (n - npml)), 0.0) / npml
        smax = -(order + 1.0) * ln_R / (2.0 * k0dx * npml)
        return 1.0 - 1j * smax * d ** order

    s_c = s_at(np.arange(n) + 0.5)
    s_h = s_at(np.arange(n + 1, dtype=np.float64))
    return s_c, s_h


def _npml_xy(npml):
    if isinstance(npml, (tuple, list)):
        return int(npml[0]), int(npml[1])
    return int(npml), int(npml)


def assemble(nx: int, ny: int, eps: np.ndarray, k0dx: float, npml,
             ln_R: float = LN_R_DEFAULT, order: float = PML_ORDER_DEFAULT) -> sp.csr_matrix:
    """Dimensionless FDFD operator A (complex128 CSR, n = i*ny + j), Eq. 1-2.

    npml is the PML thickness in cells, either one int for both axes or a
    pair (npml_x, npml_y).

    Row (i, j):
      A[(i,j),(i,j)]   = (1/sx_c[i]) (1/sx_h[i+1] + 1/sx_h[i])
                       + (1/sy_c[j]) (1/sy_h[j+1] + 1/sy_h[j]) - k0dx^2 eps[i,j]
      A[(i,j),(i+-1,j)] = -1 / (sx_c[i] sx_h[i+1 or i])   (dropped beyond the grid: PEC)
      A[(i,j),(i,j+-1)] = -1 / (sy_c[j] sy_h[j+1 or j])
    """
    eps = np.asarray(eps, dtype=np.float64).reshape(nx, ny)
    px, py = _npml_xy(npml)
    sxc, sxh = pml_stretch(nx, px, k0dx, ln_R, order)
    syc, syh = pml_stretch(ny, py, k0dx, ln_R, order)
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    row = (I * ny + J).ravel()
    xp = (-1.0 / (sxc[:, None] * sxh[1:, None]) * np.ones((1, ny)))     # to (i+1, j)
    xm = (-1.0 / (sxc[:, None] * sxh[:-1, None]) * np.ones((1, ny)))    # to (i-1, j)
    yp = (-1.0 / (syc[None, :] * syh[None, 1:]) * np.ones((nx, 1)))     # to (i, j+1)
    ym = (-1.0 / (syc[None, :] * syh[None, :-1]) * np.ones((nx, 1)))    # to (i, j-1)
    diag = -(xp + xm) - (yp + ym) - k0dx ** 2 * eps
    rows = [row]
    cols = [row]
    vals = [diag.ravel()]
    for off_i, off_j, v in ((1, 0, xp), (-1, 0, xm), (0, 1, yp), (0, -1, ym)):
        ii, jj = I + off_i, J + off_j
        ok = ((ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)).ravel()
        rows.append(row[ok])
        cols.append((ii * ny + jj).ravel()[ok])
        vals.append(v.ravel()[ok])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny)).tocsr()
    return A


def symmetrizer(nx: int, ny: int, k0dx: float, npml, ln_R: float = LN_R_DEFAULT,
                order: float = PML_ORDER_DEFAULT) -> np.ndarray:
    """Diagonal D = sx_c[i] sy_c[j] for which D A is complex symmetric (reciprocity)."""
    px, py = _npml_xy(npml)
    sxc, _ = pml_stretch(nx, px, k0dx, ln_R, order)
    syc, _ = pml_stretch(ny, py, k0dx, ln_R, order)
    return (sxc[:, None] * syc[None, :]).ravel()


# ---------------------------------------------------------------------------
# Eq. 5-6: direct solves on one factorisation (forward and transpose)
# ---------------------------------------------------------------------------
def nested_dissection(nx: int, ny: int, leaf: int = 64) -> np.ndarray:
    """Fill-reducing elimination order of the nx x ny grid (flat n = i*ny + j) by geometric nested
    dissection (A. George, SIAM J. Numer. Anal. 10, 1973): split the longer side of a block by one
    line of cells, order the two halves recursively, then the separating line; blocks of at most
    `leaf` cells are ordered row by row.  Any order gives the same solution up to rounding; this
    one keeps SuperLU's fill at O(N log N) on the 5-point stencil, where minimum degree fills
    several times more (the role of the METIS ordering in PARDISO, the paper's solver)."""
    parts = []

    def rec(i0, i1, j0, j1):
        w, h = i1 - i0, j1 - j0
        if w <= 0 or h <= 0:
            return
        if w * h <= leaf:
            I, J = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
            parts.append((I * ny + J).ravel())
            return
        if w >= h:
            m = (i0 + i1) // 2
            rec(i0, m, j0, j1)
            rec(m + 1, i1, j0, j1)
            parts.append(m * ny + np.arange(j0, j1))
        else:
            m = (j0 + j1) // 2
            rec(i0, i1, j0, m)
            rec(i0, i1, m + 1, j1)
            parts.append(np.arange(i0, i1) * ny + m)

    rec(0, nx, 0, ny)
    return np.concatenate(parts).astype(np.int64)


class Factor:
    """Sparse LU of A (SuperLU, complex128); solve() is Eq. 5, solve_T() Eq. 6.

    The unknowns are ordered by nested_dissection when the grid shape is given (else by
    SuperLU's minimum degree on A^T + A), and SuperLU factors the permuted matrix with threshold
    partial pivoting (a row is kept on the diagonal while its pivot is at least 0.1 of the
    column's largest).  Each solve is followed by one step of iterative refinement in
    complex128, x += A^-1 (b - A x), which takes the residual to rounding level."""

    def __init__(self, A: sp.spmatrix, shape: tuple | None = None):
        self.A = A.tocsc()
        n = self.A.shape[0]
        if shape is not None and shape[0] * shape[1] == n:
            self.p = nested_dissection(*shape)
            Ap = self.A[self.p][:, self.p].tocsc()
            self.lu = spla.splu(Ap, permc_spec="NATURAL", diag_pivot_thresh=0.1,
                                options=dict(SymmetricMode=True))
        else:
            self.p = None
            self.lu = spla.splu(self.A, permc_spec="MMD_AT_PLUS_A")

    def _raw(self, b: np.ndarray, trans: str) -> np.ndarray:
        if self.p is None:
            return self.lu.solve(b, trans=trans)
        x = np.empty_like(b)
        x[self.p] = self.lu.solve(b[self.p], trans=trans)
        return x

    def _solve(self, b: np.ndarray, trans: str) -> np.ndarray:
        b = np.asarray(b, dtype=np.complex128)
        x = self._raw(b, trans)
        M = self.A.T if trans == "T" else self.A
        return x + self._raw(b - M @ x, trans)

    def solve(self, b: np.ndarray) -> np.ndarray:
        return self._solve(b, "N")

    def solve_T(self, b: np.ndarray) -> np.ndarray:
        """Solves A^T x = b (plain transpose, not conjugate)."""
        return self._solve(b, "T")


def symmetric_ldlt(M: np.ndarray, order: np.ndarray):
    """M[order][:, order] = L diag(d) L^T for a complex symmetric dense M, by Gaussian elimination
    without pivoting in the given order (L unit lower triangular, plain transpose).  The reference
    for the factors of the symmetric form of D A (reciprocity makes D A complex symmetric).
    Returns (L, d) in the permuted order."""
    Mp = np.array(M, dtype=np.complex128)[np.ix_(order, order)]
    n = Mp.shape[0]
    d = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        d[j] = Mp[j, j]
        Mp[j + 1:, j] /= d[j]
        Mp[j + 1:, j + 1:] -= np.outer(Mp[j + 1:, j], Mp[j + 1:, j]) * d[j]
    L = np.tril(Mp, -1) + np.eye(n)
    return L, d


# ---------------------------------------------------------------------------
# Eq. 3-4: objective, adjoint source and pixel gradient
# ---------------------------------------------------------------------------
def overlap(E: np.ndarray, g: np.ndarray) -> complex:
    """o = g^T E (no conjugation on g), E and g flat of length nx*ny."""
    return complex(np.sum(g * E))


def adjoint_source(E: np.ndarray, g: np.ndarray, weight: float = 1.0) -> np.ndarray:
    """(dF/dE)^T for F = weight |g^T E|^2 (Wirtinger, E* fixed): weight conj(o) g."""
    return weight * np.conj(overlap(E, g)) * g


def target_objective(o: complex, target: float, weight: float = 1.0) -> float:
    """Squared transmission error w (|o|^2 - t)^2 of one port (Sec. III-IV: the devices minimise the
    difference between calculated and target transmissions)."""
    return weight * (abs(o) ** 2 - target) ** 2


def target_adjoint_source(E: np.ndarray, g: np.ndarray, target: float, weight: float = 1.0) -> np.ndarray:
    """(dF/dE)^T for F = w (|g^T E|^2 - t)^2 (Wirtinger, E* fixed): 2 w (|o|^2 - t) conj(o) g."""
    o = overlap(E, g)
    return 2.0 * weight * (abs(o) ** 2 - target) * np.conj(o) * g


def grad_eps(E: np.ndarray, E_adj: np.ndarray, k0dx: float) -> np.ndarray:
    """dF/deps_p = -2 Re{E_adj[p] (dA/deps_p) E[p]} = 2 k0dx^2 Re(E_adj[p] E[p]), Eq. 3."""
    return 2.0 * k0dx ** 2 * np.real(E_adj * E)


def design_box_of(v: np.ndarray, nx: int, ny: int, box) -> np.ndarray:
    x0, y0, w, h = box
    return v.reshape(nx, ny)[x0:x0 + w, y0:y0 + h]


def design_iteration(wl, rho: np.ndarray, eps_of_rho, delta_eps: float, targets=None):
    """One forward + adjoint iteration (Sec. II), all wavelengths and sources.

    wl: a workloads.Workload.  Returns (F, dF/drho [w, h], fields) with
    F = sum_{omega, s} |g_{omega,s}^T E_{omega,s}|^2, or with targets[w][s] given the squared
    transmission error sum_{omega, s} (|g^T E|^2 - t_{omega,s})^2, and fields[(w, s)] = (E, E_adj).
    """
    eps = eps_of_rho(rho)
    F = 0.0
    g_eps = np.zeros(wl.box[2:4])
    fields = {}
    for w, k0dx in enumerate(wl.k0dx()):
        fac = Factor(assemble(wl.nx, wl.ny, eps, k0dx, wl.npml), (wl.nx, wl.ny))
        for s in range(wl.n_src):
            b = wl.source_dense(s, w)
            g = wl.monitor_dense(w, s)
            E = fac.solve(b)
            o = overlap(E, g)
            if targets is None:
                F += abs(o) ** 2
                E_adj = fac.solve_T(adjoint_source(E, g))
            else:
                F += target_objective(o, targets[w][s])
                E_adj = fac.solve_T(target_adjoint_source(E, g, targets[w][s]))
            g_eps += design_box_of(grad_eps(E, E_adj, k0dx), wl.nx, wl.ny, wl.box)
            fields[(w, s)] = (E, E_adj)
    return F, delta_eps * g_eps, fields


def objective_pixel_differences(wl, rho: np.ndarray, pixels, h: float, delta_eps: float) -> np.ndarray:
    """Central differences (F(rho + h e_p) - F(rho - h e_p)) / (2 h) of the objective of
    design_iteration at the listed design pixels p (flat indices into the [w, h] box).

    Raising rho_p by t changes eps at the pixel's cell q by t delta_eps, so A changes by
    d e_q e_q^T with d = -(k0 dx)^2 t delta_eps (Eq. 1-2): a rank-one change.  Each F(rho +- h e_p)
    is evaluated exactly on the perturbed operator by the Sherman-Morrison identity
        (A + d e_q e_q^T)^-1 b = x - d x_q / (1 + d u_q) u,   x = A^-1 b,  u = A^-1 e_q,
    so that the perturbed overlap is o' = o - d x_q (g^T u) / (1 + d u_q) with g^T u = (A^-T g)_q.
    Library steps: one SuperLU factorisation per wavelength, solves for x and A^-T g per source,
    and one solve with the unit vectors of all pixels for the u_q = (A^-1)_qq.
    """
    x0, y0, bw, bh = wl.box
    pixels = np.asarray(pixels, dtype=np.int64)
    cells = (x0 + pixels // bh) * wl.ny + (y0 + pixels % bh)
    eps = wl.eps_full(rho).reshape(-1)
    Fp = np.zeros(len(pixels))
    Fm = np.zeros(len(pixels))
    for w, k0dx in enumerate(wl.k0dx()):
        fac = Factor(assemble(wl.nx, wl.ny, eps, k0dx, wl.npml), (wl.nx, wl.ny))
        unit = np.zeros((wl.n, len(pixels)), dtype=np.complex128)
        unit[cells, np.arange(len(pixels))] = 1.0
        uqq = fac.solve(unit)[cells, np.arange(len(pixels))]
        for s in range(wl.n_src):
            g = wl.monitor_dense(w, s)
            E = fac.solve(wl.source_dense(s, w))
            o = overlap(E, g)
            gu = fac.solve_T(g)[cells]
            for sign, acc in ((1.0, Fp), (-1.0, Fm)):
                d = -k0dx ** 2 * sign * h * delta_eps
                acc += np.abs(o - d * E[cells] * gu / (1.0 + d * uqq)) ** 2
    return (Fp - Fm) / (2.0 * h)


# ---------------------------------------------------------------------------
# Optimiser updates applied between iterations (outside the timed hot path)
# ---------------------------------------------------------------------------
def sign_step(rho: np.ndarray, grad: np.ndarray, step: float) -> np.ndarray:
    """Ascent step rho += step * sign(grad), sign(0) = 0, clipped to [0, 1]."""
    return np.clip(rho + step * np.sign(grad), 0.0, 1.0)


def adam_step(rho, grad, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) ascent on F; state = dict(m, v, t)."""
    t = state.get("t", 0) + 1
    m = beta1 * state.get("m", np.zeros_like(rho)) + (1 - beta1) * grad
    v = beta2 * state.get("v", np.zeros_like(rho)) + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    state.update(t=t, m=m, v=v)
    return np.clip(rho + lr * mh / (np.sqrt(vh) + eps), 0.0, 1.0)


# ---------------------------------------------------------------------------
# Error metrics used by the parity tests
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Sec. III: smoothing filter and projection of the design density
# ---------------------------------------------------------------------------
def filter_offsets(radius: float):
    """Integer offsets (di, dj) with distance d < radius and their weights radius - d."""
    r = int(np.ceil(radius))
    out = []
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            d = float(np.hypot(di, dj))
            if d < radius:
                out.append((di, dj, radius - d))
    return out


def _shift_sum(v: np.ndarray, radius: float, weight_in=None):
    """sum over offsets of weight * v[i + di, j + dj] (entries outside the box count as absent)."""
    w, h = v.shape
    acc = np.zeros_like(v, dtype=np.float64)
    for di, dj, wt in filter_offsets(radius):
        src = np.zeros_like(v, dtype=np.float64)
        i0, i1 = max(0, -di), min(w, w - di)
        j0, j1 = max(0, -dj), min(h, h - dj)
        if i0 < i1 and j0 < j1:
            src[i0:i1, j0:j1] = v[i0 + di:i1 + di, j0 + dj:j1 + dj]
        acc += wt * src
    return acc


def filter_norm(w: int, h: int, radius: float) -> np.ndarray:
    """N_i = sum of the weights of the pixels of a w x h box around pixel i."""
    return _shift_sum(np.ones((w, h)), radius)


def density_filter(rho: np.ndarray, radius: float) -> np.ndarray:
    """rho~ = W rho with W_ij = w_ij / N_i (rho: [w, h], x-major like the design box)."""
    return _shift_sum(rho, radius) / filter_norm(*rho.shape, radius)


def density_filter_adjoint(y: np.ndarray, radius: float) -> np.ndarray:
    """W^T y = sum_i w_ij y_i / N_i (the weights are symmetric in i and j)."""
    return _shift_sum(y / filter_norm(*y.shape, radius), radius)


def projection(rt: np.ndarray, beta: float, eta: float) -> np.ndarray:
    a = np.tanh(beta * eta)
    return (a + np.tanh(beta * (rt - eta))) / (a + np.tanh(beta * (1.0 - eta)))


def projection_slope(rt: np.ndarray, beta: float, eta: float) -> np.ndarray:
    a = np.tanh(beta * eta)
    t = np.tanh(beta * (rt - eta))
    return beta * (1.0 - t * t) / (a + np.tanh(beta * (1.0 - eta)))


def filter_project(rho: np.ndarray, radius: float, beta: float, eta: float, eps_lo: float, eps_hi: float):
    """eps of the design box from the raw density: filter, project, map to permittivity."""
    rt = density_filter(rho, radius)
    return eps_lo + projection(rt, beta, eta) * (eps_hi - eps_lo)


def filter_project_grad(rho: np.ndarray, g_eps: np.ndarray, radius: float, beta: float, eta: float,
                        eps_lo: float, eps_hi: float) -> np.ndarray:
    """dF/drho from dF/deps by the chain rule through the projection and the filter."""
    rt = density_filter(rho, radius)
    return density_filter_adjoint(g_eps * (eps_hi - eps_lo) * projection_slope(rt, beta, eta), radius)


# ---------------------------------------------------------------------------
# Eigenmode sources (Sec. III: the multi-mode devices launch and monitor
# waveguide modes; the paper does not say how they are computed)
# ---------------------------------------------------------------------------
def mode_sign(phi: np.ndarray) -> np.ndarray:
    """Sign convention of a mode profile: the first entry whose magnitude reaches half the
    largest is positive."""
    phi = np.asarray(phi, dtype=np.float64)
    j = int(np.argmax(np.abs(phi) >= 0.5 * np.max(np.abs(phi))))
    return phi if phi[j] > 0 else -phi


def slab_modes(eps_line: np.ndarray, k0dx: float, n_modes: int):
    """Modes of an x-invariant guide eps[i, j] = eps_line[j] on the grid of Eq. 1-2 (no PML on the
    cross-section, PEC one cell beyond both ends, as in assemble with npml_y = 0).

    Source-free fields E[i, j] = phi[j] exp(-i theta i) of the operator A satisfy
        (k0dx^2 diag(eps_line) + D2) phi = mu phi,   D2 = tridiag(1, -2, 1),
        mu = 2 - 2 cos theta = 4 sin^2(theta / 2)
    (the x-part of the stencil acting on exp(-i theta i)).  The n_modes largest eigenvalues mu
    are the most strongly guided modes; a mode is bound when mu > k0dx^2 max(eps at both ends).
    Library step: SciPy's symmetric tridiagonal eigensolver (LAPACK).

    Returns (mu [n_modes], descending; theta [n_modes], NaN where mu is not in (0, 4);
    phi [n_modes, ny], unit 2-norm, signs by mode_sign).
    """
    import scipy.linalg as sla
    eps_line = np.asarray(eps_line, dtype=np.float64)
    ny = eps_line.size
    d = k0dx ** 2 * eps_line - 2.0
    e = np.ones(ny - 1)
    mu, V = sla.eigh_tridiagonal(d, e, select="i", select_range=(ny - n_modes, ny - 1))
    order = np.argsort(-mu)
    mu = mu[order]
    phi = np.stack([mode_sign(V[:, k] / np.linalg.norm(V[:, k])) for k in order])
    with np.errstate(invalid="ignore"):
        theta = np.where((mu > 0) & (mu < 4), 2.0 * np.arcsin(np.sqrt(np.clip(mu, 0, 4)) / 2.0), np.nan)
    return mu, theta, phi


def rel_err(x, ref) -> float:
    x = np.asarray(x).ravel()
    ref = np.asarray(ref).ravel()
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def residual_rel(A: sp.spmatrix, x: np.ndarray, b: np.ndarray) -> float:
    return float(np.linalg.norm(A @ x - b) / np.linalg.norm(b))
