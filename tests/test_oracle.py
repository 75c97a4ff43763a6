"""Pins for the CPU oracle: each checks it against something other than itself.

Every test here runs on the CPU.  A plausible slip anywhere in the oracle (a
dropped PML term, a sign of the eps term, a swapped half-point index, a
conjugate in place of a transpose, a wrong gradient constant) fails at least
one of them; the mapping is given in each docstring.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fdfd_oracle as O


def _rand_eps(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return W.EPS_SIO2 + W.DELTA_EPS * rng.uniform(0, 1, size=(nx, ny))


@pytest.mark.parametrize("nx,ny,npml", [(12, 17, 3), (9, 6, 2), (20, 20, 4)])
def test_dense_lapack_solve(nx, ny, npml):
    """SuperLU forward and transpose solves equal dense LAPACK solves (Eq. 5, 6)."""
    k0dx = 2 * np.pi * 0.05 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 1), k0dx, npml)
    b = W.random_complex(nx * ny, 2)
    fac = O.Factor(A)
    Ad = A.toarray()
    x_ref = np.linalg.solve(Ad, b)
    xt_ref = np.linalg.solve(Ad.T, b)
    assert O.rel_err(fac.solve(b), x_ref) < 1e-11
    assert O.rel_err(fac.solve_T(b), xt_ref) < 1e-11


def test_plane_wave_dispersion():
    """A homogeneous-medium plane wave obeying the Yee dispersion relation
    4 sin^2(kx/2) + 4 sin^2(ky/2) = (k0 dx)^2 eps  is annihilated by A at interior
    nodes (pins the 4 / -1 stencil and the sign of the -(k0 dx)^2 eps term)."""
    nx, ny = 30, 26
    eps = 2.085
    k0dx = 2 * np.pi * 0.05 / 1.55
    kx = 0.21
    ky = 2 * np.arcsin(np.sqrt((k0dx ** 2 * eps - 4 * np.sin(kx / 2) ** 2) / 4))
    A = O.assemble(nx, ny, np.full((nx, ny), eps), k0dx, 0)
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    E = np.exp(-1j * (kx * I + ky * J)).ravel()
    r = (A @ E).reshape(nx, ny)[1:-1, 1:-1]
    assert np.max(np.abs(r)) < 1e-13
    # a wavevector off the dispersion shell leaves a residual of order (dk)*k
    E2 = np.exp(-1j * (kx * I + 1.05 * ky * J)).ravel()
    r2 = (A @ E2).reshape(nx, ny)[1:-1, 1:-1]
    assert np.min(np.abs(r2)) > 1e-3


def test_plate_mode_propagation_and_pml():
    """Parallel-plate guide: PEC walls in y (no y-PML), PML only in x.  The lowest
    discrete plate mode sin(pi (j+1)/(ny+1)) propagates with the closed-form Yee
    wavenumber 4 sin^2(kx/2) = (k0dx)^2 eps - 4 sin^2(pi / (2 (ny+1))), away from the
    source, and the right PML absorbs it (small standing-wave ripple, strong decay).
    Pins PEC placement (ghost cell one beyond the grid), the e^{-i kx x} outgoing
    convention, the PML sign and its axis."""
    nx, ny, npml = 260, 7, 20
    eps = 12.11
    k0dx = 2 * np.pi * 0.04 / 1.55
    A = O.assemble(nx, ny, np.full((nx, ny), eps), k0dx, (npml, 0))
    mode = np.sin(np.pi * (np.arange(ny) + 1) / (ny + 1))
    b = np.zeros((nx, ny), complex)
    i_s = 40
    b[i_s, :] = mode
    E = O.Factor(A).solve(b.ravel()).reshape(nx, ny)
    # the field stays in the lowest mode
    Em = E @ mode / (mode @ mode)
    assert np.max(np.abs(E - Em[:, None] * mode[None, :])) < 1e-10 * np.max(np.abs(E))
    kx = 2 * np.arcsin(np.sqrt((k0dx ** 2 * eps - 4 * np.sin(np.pi / (2 * (ny + 1))) ** 2) / 4))
    ratio = Em[i_s + 20:nx - npml - 20 + 1] / Em[i_s + 20 - 1:nx - npml - 20]
    assert np.max(np.abs(ratio - np.exp(-1j * kx))) < 1e-4
    # decay inside the right PML, and a small ripple (reflection) in the interior
    assert abs(Em[nx - 2]) < 1e-5 * abs(Em[nx - npml - 1])
    amp = np.abs(Em[i_s + 20:nx - npml - 20])
    assert (amp.max() - amp.min()) / amp.mean() < 1e-4


def test_symmetrized_operator_is_symmetric():
    """D A is complex symmetric for D = sx_c sy_c (the discrete form of reciprocity)."""
    nx, ny, npml = 15, 11, 4
    k0dx = 2 * np.pi * 0.05 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 3), k0dx, npml)
    D = O.symmetrizer(nx, ny, k0dx, npml)
    S = (np.diag(D) @ A.toarray())
    assert np.max(np.abs(S - S.T)) < 1e-14 * np.max(np.abs(S))
    assert np.max(np.abs(A.toarray() - A.toarray().T)) > 1e-3   # A itself is not symmetric in the PML


def test_reciprocity():
    """x_a(source e_b) = x_b(source e_a) for points a, b outside the PML."""
    nx, ny, npml = 24, 21, 5
    k0dx = 2 * np.pi * 0.05 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 4), k0dx, npml)
    fac = O.Factor(A)
    pts = [(npml + 1) * ny + npml + 2, (nx - npml - 2) * ny + ny // 2, 12 * ny + 9]
    for a in pts:
        for b in pts:
            ea = np.zeros(nx * ny, complex)
            eb = np.zeros(nx * ny, complex)
            ea[a] = 1
            eb[b] = 1
            xa = fac.solve(eb)[a]
            xb = fac.solve(ea)[b]
            assert abs(xa - xb) < 1e-12 * max(abs(xa), 1e-30)


def test_bilinear_transpose_identity():
    """c^T (A^-1 b) = (A^-T c)^T b: solve_T is the plain transpose, not the adjoint."""
    nx, ny, npml = 18, 14, 4
    k0dx = 2 * np.pi * 0.05 / 1.31
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 5), k0dx, npml)
    fac = O.Factor(A)
    b = W.random_complex(nx * ny, 6)
    c = W.random_complex(nx * ny, 7)
    lhs = c @ fac.solve(b)
    rhs = fac.solve_T(c) @ b
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the conjugate-transpose solve does not satisfy it (A is not Hermitian)
    wrong = fac.lu.solve(c, trans="H") @ b
    assert abs(wrong - lhs) > 1e-3 * abs(lhs)


def test_manufactured_solution():
    nx, ny, npml = 33, 29, 6
    k0dx = 2 * np.pi * 0.04 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 8), k0dx, npml)
    x_star = W.random_complex(nx * ny, 9)
    b = A @ x_star
    x = O.Factor(A).solve(b)
    assert O.rel_err(x, x_star) < 1e-10


@pytest.mark.parametrize("n_omega,n_src", [(1, 1), (2, 2)])
def test_gradient_central_differences(n_omega, n_src):
    """Adjoint gradient (Eq. 3, 4) equals central finite differences of F in rho."""
    wl = W.make_small(22, 19, 4, (7, 6, 7, 6), n_omega=n_omega, n_src=n_src, seed=11)
    F0, g, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    h = 1e-4
    fd = np.zeros_like(wl.rho)
    for idx in np.ndindex(wl.rho.shape):
        rp = wl.rho.copy()
        rm = wl.rho.copy()
        rp[idx] += h
        rm[idx] -= h
        Fp, _, _ = O.design_iteration(wl, rp, wl.eps_full, W.DELTA_EPS)
        Fm, _, _ = O.design_iteration(wl, rm, wl.eps_full, W.DELTA_EPS)
        fd[idx] = (Fp - Fm) / (2 * h)
    assert O.rel_err(g, fd) < 1e-6


def test_gradient_sign_and_scale_special_case():
    """One design pixel, monitor = that pixel: F = |E_p|^2.  With A E = b,
    dE/deps_p = (k0dx)^2 G_pp E_p where G = A^-1, so dF/deps_p =
    2 (k0dx)^2 Re(conj(E_p) G_pp E_p) -- checked against the oracle's Eq. 3 path."""
    nx, ny, npml = 16, 15, 4
    k0dx = 2 * np.pi * 0.05 / 1.55
    eps = _rand_eps(nx, ny, 12)
    A = O.assemble(nx, ny, eps, k0dx, npml)
    fac = O.Factor(A)
    p = 8 * ny + 7
    b = W.random_complex(nx * ny, 13)
    E = fac.solve(b)
    g = np.zeros(nx * ny, complex)
    g[p] = 1
    E_adj = fac.solve_T(O.adjoint_source(E, g))
    grad = O.grad_eps(E, E_adj, k0dx)[p]
    ep = np.zeros(nx * ny, complex)
    ep[p] = 1
    Gpp = fac.solve(ep)[p]
    expect = 2 * k0dx ** 2 * np.real(np.conj(E[p]) * Gpp * E[p])
    assert abs(grad - expect) < 1e-10 * abs(expect)


def test_c1_oracle_iteration_runs():
    wl = W.make("c1")
    F, g, fields = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    assert np.isfinite(F) and F > 0
    assert g.shape == (40, 40) and np.all(np.isfinite(g))
    E, Ea = fields[(0, 0)]
    A = O.assemble(wl.nx, wl.ny, wl.eps_full(), wl.k0dx()[0], wl.npml)
    assert O.residual_rel(A, E, wl.source_dense(0)) < 1e-12


# ---------------------------------------------------------------------------
# Sec. III: smoothing filter and projection (the step before the hot path)
# ---------------------------------------------------------------------------
def _filter_brute(rho, radius):
    """rho~ by a double loop over all pixel pairs (independent of the offset form)."""
    w, h = rho.shape
    out = np.zeros_like(rho)
    for i in range(w):
        for j in range(h):
            s = n = 0.0
            for p in range(w):
                for q in range(h):
                    wt = max(0.0, radius - float(np.hypot(i - p, j - q)))
                    s += wt * rho[p, q]
                    n += wt
            out[i, j] = s / n
    return out


@pytest.mark.parametrize("w,h,radius", [(9, 7, 2.5), (5, 11, 5.0), (12, 12, 1.2)])
def test_filter_matches_pair_sum_and_keeps_constants(w, h, radius):
    """The filter equals the normalised hat-weighted pair sum and leaves a constant density
    unchanged (catches a missing normalisation, a wrong weight or a boundary slip)."""
    rho = np.random.default_rng(3).uniform(0, 1, (w, h))
    assert np.max(np.abs(O.density_filter(rho, radius) - _filter_brute(rho, radius))) < 1e-13
    assert np.max(np.abs(O.density_filter(np.full((w, h), 0.37), radius) - 0.37)) < 1e-14


@pytest.mark.parametrize("w,h,radius", [(9, 7, 2.5), (13, 4, 5.0)])
def test_filter_adjoint_identity(w, h, radius):
    """<W x, y> = <x, W^T y> (catches an adjoint without the per-pixel normalisation)."""
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=(w, h)), rng.normal(size=(w, h))
    lhs = np.sum(O.density_filter(x, radius) * y)
    rhs = np.sum(x * O.density_filter_adjoint(y, radius))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_projection_closed_forms():
    """P(0) = 0, P(1) = 1, P(eta) = tanh(b e) / (tanh(b e) + tanh(b (1 - e))), and P(x) -> x as b -> 0."""
    for beta, eta in [(8.0, 0.5), (32.0, 0.3), (2.0, 0.7)]:
        assert abs(O.projection(np.array(0.0), beta, eta)) < 1e-15
        assert abs(O.projection(np.array(1.0), beta, eta) - 1.0) < 1e-15
        a = np.tanh(beta * eta)
        assert abs(O.projection(np.array(eta), beta, eta) - a / (a + np.tanh(beta * (1 - eta)))) < 1e-15
    x = np.linspace(0, 1, 11)
    assert np.max(np.abs(O.projection(x, 1e-4, 0.5) - x)) < 1e-8


def test_projection_slope_central_differences():
    x = np.linspace(-0.2, 1.2, 29)
    h = 1e-6
    for beta, eta in [(8.0, 0.5), (20.0, 0.4)]:
        fd = (O.projection(x + h, beta, eta) - O.projection(x - h, beta, eta)) / (2 * h)
        assert np.max(np.abs(fd - O.projection_slope(x, beta, eta))) < 1e-6 * beta


def test_filter_project_chain_rule_central_differences():
    """dF/drho through projection and filter against central differences of F = sum c * eps(rho)."""
    rng = np.random.default_rng(5)
    w, h, radius, beta, eta = 10, 8, 3.0, 6.0, 0.5
    rho = rng.uniform(0, 1, (w, h))
    c = rng.normal(size=(w, h))
    F = lambda r: float(np.sum(c * O.filter_project(r, radius, beta, eta, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)))
    g = O.filter_project_grad(rho, c, radius, beta, eta, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    step = 1e-6
    for (i, j) in [(0, 0), (4, 3), (9, 7), (2, 6)]:
        e = np.zeros_like(rho)
        e[i, j] = step
        fd = (F(rho + e) - F(rho - e)) / (2 * step)
        assert abs(fd - g[i, j]) < 1e-6 * max(1.0, abs(g[i, j]))


# ---------------------------------------------------------------------------
# Eigenmode sources
# ---------------------------------------------------------------------------
def test_slab_modes_uniform_line_closed_form():
    """Uniform line: mu_q = k0dx^2 eps - 4 sin^2(q pi / (2 (n + 1))), phi_q ~ sin(q pi (j + 1) / (n + 1)),
    q = 1, 2, ... (the Dirichlet second difference).  Pins the stencil, its sign and the PEC ends."""
    n, eps, k0dx = 37, 2.085, 2 * np.pi * 0.04 / 1.55
    mu, theta, phi = O.slab_modes(np.full(n, eps), k0dx, 4)
    q = np.arange(1, 5)
    np.testing.assert_allclose(mu, k0dx ** 2 * eps - 4 * np.sin(q * np.pi / (2 * (n + 1))) ** 2, rtol=0, atol=1e-13)
    for k in range(4):
        s = np.sin((k + 1) * np.pi * (np.arange(n) + 1) / (n + 1))
        np.testing.assert_allclose(phi[k], O.mode_sign(s / np.linalg.norm(s)), atol=1e-10)
    prop = mu > 0                                   # evanescent along x where mu <= 0: theta is NaN
    assert prop[:2].all() and not prop[3] and np.isnan(theta[~prop]).all()
    np.testing.assert_allclose(4 * np.sin(theta[prop] / 2) ** 2, mu[prop], rtol=1e-12)


def _slab(dx, d=0.48, width=4.0):
    ncore = int(round(d / dx))
    ny = int(round(width / dx))
    ny += (ny - ncore) % 2
    eps = np.full(ny, W.EPS_SIO2)
    a = (ny - ncore) // 2
    eps[a:a + ncore] = W.EPS_SI
    return eps


def _slab_neff_continuum(m, d=0.48, lam=1.55):
    """TE modes of a symmetric slab: tan(kappa d / 2 - m pi / 2) = gamma / kappa (textbook)."""
    from scipy.optimize import brentq
    n1, n2, k0 = np.sqrt(W.EPS_SI), np.sqrt(W.EPS_SIO2), 2 * np.pi / lam

    def f(ne):
        ka, ga = k0 * np.sqrt(n1 ** 2 - ne ** 2), k0 * np.sqrt(ne ** 2 - n2 ** 2)
        return np.tan(ka * d / 2 - m * np.pi / 2) - ga / ka
    xs = np.linspace(n2 + 1e-9, n1 - 1e-9, 40001)
    v = f(xs)
    for a, b, fa, fb in zip(xs[:-1], xs[1:], v[:-1], v[1:]):
        if np.sign(fa) != np.sign(fb) and abs(fa) < 50 and abs(fb) < 50:
            return brentq(f, a, b)
    raise AssertionError("no root")


def test_slab_modes_converge_to_the_continuum_dispersion_at_second_order():
    """480 nm Si slab in SiO2 at 1.55 um: the grid's effective indices theta / k0dx approach the
    continuum TE0 / TE1 roots with error ~ dx^2 (ratio 4 per halving); the Richardson value agrees
    to 1e-4.  A wrong eps term, D2 sign or mu -> theta relation breaks the limit."""
    for m in (0, 1):
        ref = _slab_neff_continuum(m)
        errs = []
        for dx in (0.02, 0.01):
            _, theta, _ = O.slab_modes(_slab(dx), 2 * np.pi * dx / 1.55, 2)
            errs.append(theta[m] / (2 * np.pi * dx / 1.55) - ref)
        assert 3.5 < errs[0] / errs[1] < 4.5
        assert abs((4 * errs[1] - errs[0]) / 3) < 1e-4


def test_slab_mode_count_parity_and_orthonormality():
    """V = (k0 d / 2) sqrt(n1^2 - n2^2) = 3.08 gives floor(2 V / pi) + 1 = 2 bound TE modes; TE0 even,
    TE1 odd about the slab centre; profiles orthonormal."""
    dx = 0.02
    eps = _slab(dx)
    k0dx = 2 * np.pi * dx / 1.55
    mu, _, phi = O.slab_modes(eps, k0dx, 4)
    bound = mu > k0dx ** 2 * W.EPS_SIO2
    V = (np.pi / 1.55 * 0.48) * np.sqrt(W.EPS_SI - W.EPS_SIO2)
    assert bound.sum() == int(np.floor(2 * V / np.pi)) + 1 == 2
    np.testing.assert_allclose(phi[0], phi[0][::-1], atol=1e-12)
    np.testing.assert_allclose(phi[1], -phi[1][::-1], atol=1e-12)
    np.testing.assert_allclose(phi @ phi.T, np.eye(4), atol=1e-12)


def test_slab_mode_propagates_through_the_2d_operator():
    """A guide along x (PEC walls in y, PML in x) fed by a mode on one column: the field stays
    phi(y) u(x) and advances by exp(-i theta) per cell away from the source.  Ties slab_modes to
    assemble: the cross-section operator is exactly the y-part of A."""
    nx, npml, dx = 200, 20, 0.04
    eps_line = _slab(dx, width=2.0)
    ny = eps_line.size
    k0dx = 2 * np.pi * dx / 1.55
    _, theta, phi = O.slab_modes(eps_line, k0dx, 2)
    for m in (0, 1):
        b = np.zeros((nx, ny), complex)
        b[40, :] = phi[m]
        E = O.Factor(O.assemble(nx, ny, np.tile(eps_line, (nx, 1)), k0dx, (npml, 0))).solve(b.ravel())
        E = E.reshape(nx, ny)
        u = E @ phi[m]
        assert np.max(np.abs(E - u[:, None] * phi[m][None, :])) < 1e-10 * np.max(np.abs(E))
        ratio = u[61:nx - npml - 20] / u[60:nx - npml - 21]
        assert np.max(np.abs(ratio - np.exp(-1j * theta[m]))) < 1e-4


def test_mode_overlap_selection_rules_in_a_straight_guide():
    """Straight symmetric guide (PEC walls in y, PML in x), TE0 launched: the TE1 overlap vanishes by
    parity, the TE0 overlap keeps its modulus along the guide (lossless, single mode content), and
    the adjoint gradient of F = |o_TE1|^2 is zero (F is stationary at 0)."""
    nx, npml, dx = 160, 20, 0.04
    eps_line = _slab(dx, width=2.0)
    ny = eps_line.size
    k0dx = 2 * np.pi * dx / 1.55
    _, _, phi = O.slab_modes(eps_line, k0dx, 2)
    fac = O.Factor(O.assemble(nx, ny, np.tile(eps_line, (nx, 1)), k0dx, (npml, 0)))
    b = np.zeros((nx, ny), complex)
    b[30, :] = phi[0]
    E = fac.solve(b.ravel())
    mags = []
    for col in range(60, nx - npml - 10, 10):
        g0 = np.zeros((nx, ny))
        g0[col] = phi[0]
        g1 = np.zeros((nx, ny))
        g1[col] = phi[1]
        assert abs(O.overlap(E, g1.ravel())) < 1e-12 * abs(O.overlap(E, g0.ravel()))
        mags.append(abs(O.overlap(E, g0.ravel())))
    assert (max(mags) - min(mags)) / np.mean(mags) < 1e-4
    g1 = np.zeros((nx, ny))
    g1[100] = phi[1]
    Ea = fac.solve_T(O.adjoint_source(E, g1.ravel()))
    assert np.max(np.abs(O.grad_eps(E, Ea, k0dx))) < 1e-12


# ---------------------------------------------------------------------------
# PML constants: the graded profile against the textbook reflection integral and
# against the decay of a guided wave inside the layer
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,npml,k0dx,order,R", [(100, 10, 2 * np.pi * 0.05 / 1.55, 3.0, 1e-8),
                                                  (340, 20, 2 * np.pi * 0.04 / 1.55, 3.0, 1e-8),
                                                  (60, 12, 0.3, 2.0, 1e-6),
                                                  (45, 7, 0.5, 3.0, 1e-4)])
def test_pml_profile_meets_the_target_reflection(n, npml, k0dx, order, R):
    """A graded layer of thickness L in front of a PEC wall reflects a normally incident wave by
    R = exp(-2 k0 int_0^L sigma(x) / (omega eps0) dx) (Taflove and Hagness, Ch. 7), with
    -Im s = sigma / (omega eps0).  Simpson's rule on the half-cell lattice of the oracle's
    s values (centres and half points, spacing dx / 2) integrates a polynomial grade of order <= 3
    exactly, so 2 k0dx int (-Im s) du over each layer must equal -ln R to rounding.  The interior has
    s = 1, the real part is 1 everywhere, and Im s <= 0 (absorption for e^{+i w t}).  A factor-2
    slip in sigma_max, a wrong (order + 1), or the layer on the wrong side fails here."""
    sc, sh = O.pml_stretch(n, npml, k0dx, ln_R=np.log(R), order=order)
    assert np.all(sc.real == 1.0) and np.all(sh.real == 1.0)
    assert np.all(sc.imag <= 0.0) and np.all(sh.imag <= 0.0)
    assert np.all(sc[npml:n - npml] == 1.0) and np.all(sh[npml:n - npml + 1] == 1.0)
    for hs, cs in ((sh[:npml + 1], sc[:npml]), (sh[n - npml:], sc[n - npml:])):
        integral = np.sum((-hs.imag[:-1] - 4.0 * cs.imag - hs.imag[1:]) / 6.0)
        assert abs(2.0 * k0dx * integral + np.log(R)) < 1e-12 * abs(np.log(R))
    # the grade vanishes toward the interior and is largest at the wall
    assert abs(sh[0].imag) > abs(sc[0].imag) > abs(sc[npml - 1].imag) > 0.0


def test_pml_decay_profile_of_a_guided_wave():
    """Inside the layer a wave travelling along x with propagation constant kx goes as
    exp(-i kx int s du), so its amplitude falls by exp(-kx int_0^u (-Im s) du') with depth u; for the
    cubic grade the exponent is -kx sigma_max' L d^4 / 4 at depth d = u / L.  The plate mode of
    test_plate_mode_propagation_and_pml, solved with a 30-cell x-PML, follows this law within 3%
    at depths 0.2 - 0.75 (deeper, the grade is no longer resolved by the grid).  A quadratic grade
    or sigma_max off by 2 moves the exponent by 50 - 200%."""
    npml, ny, eps = 30, 7, 12.11
    nx = 200 + npml
    k0dx = 2 * np.pi * 0.04 / 1.55
    A = O.assemble(nx, ny, np.full((nx, ny), eps), k0dx, (npml, 0))
    mode = np.sin(np.pi * (np.arange(ny) + 1) / (ny + 1))
    b = np.zeros((nx, ny), complex)
    b[40, :] = mode
    E = O.Factor(A).solve(b.ravel()).reshape(nx, ny)
    Em = E @ mode / (mode @ mode)
    kx = 2 * np.arcsin(np.sqrt((k0dx ** 2 * eps - 4 * np.sin(np.pi / (2 * (ny + 1))) ** 2) / 4))
    smax = -4.0 * np.log(1e-8) / (2 * k0dx * npml)      # textbook sigma_max / (omega eps0), m = 3
    i0 = nx - npml - 1
    checked = 0
    for i in range(nx - npml, nx):
        d = (i + 0.5 - (nx - npml)) / npml
        if not 0.2 <= d <= 0.75:
            continue
        predicted = -kx * smax * npml * d ** 4 / 4.0
        measured = np.log(abs(Em[i]) / abs(Em[i0]))
        assert abs(measured - predicted) <= 0.03 * abs(predicted), (d, measured, predicted)
        checked += 1
    assert checked >= 15


# ---------------------------------------------------------------------------
# Optimiser updates between iterations (C1-C3, C5 sign step; C4 Adam)
# ---------------------------------------------------------------------------
def test_sign_step_values():
    """rho + step * sign(grad) with sign(0) = 0 (no move), an ascent direction, clipped to [0, 1]."""
    rho = np.array([0.5, 0.5, 0.5, 0.02, 0.99, 0.0, 1.0])
    g = np.array([2.0, -1e-300, 0.0, -5.0, 3.0, -1.0, 1.0])
    out = O.sign_step(rho, g, 0.05)
    np.testing.assert_array_equal(out, [0.55, 0.45, 0.5, 0.0, 1.0, 0.0, 1.0])


def test_adam_first_step_is_lr_times_sign_for_any_scale():
    """Adam's bias correction makes the first step lr g / (|g| + eps): lr sign(g) up to eps / |g|,
    whatever the gradient's scale (Kingma and Ba, Sec. 2.1), as an ascent step."""
    rho = np.full(4, 0.5)
    for scale in (1e-3, 1.0, 1e4):
        g = scale * np.array([1.0, -2.0, 0.5, -7.0])
        out = O.adam_step(rho, g, {}, lr=0.01)
        np.testing.assert_allclose(out - rho, 0.01 * np.sign(g), rtol=1e-4 / scale, atol=0)


def test_adam_second_step_closed_form():
    """Unrolling two Adam updates gives m^_2 = (b1 g1 + g2) / (1 + b1) and
    v^_2 = (b2 g1^2 + g2^2) / (1 + b2); the second step is lr m^_2 / (sqrt(v^_2) + eps).  A bias
    correction with t - 1, or b and 1 - b swapped in a moving average, fails here."""
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 0.01
    g1 = np.array([0.3, -1.0, 2.0, 0.0])
    g2 = np.array([-0.1, -1.0, 5.0, 0.4])
    st = {}
    r1 = O.adam_step(np.full(4, 0.5), g1, st, lr=lr)
    r2 = O.adam_step(r1, g2, st, lr=lr)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    np.testing.assert_allclose(r2 - r1, lr * mh / (np.sqrt(vh) + eps), rtol=1e-12, atol=1e-15)
    assert st["t"] == 2


def test_adam_constant_gradient_moves_lr_every_step_until_the_bound():
    """With a constant gradient both bias-corrected moments equal g and g^2 exactly at every t, so
    each step is lr (to eps / |g|) until the clip at 1 stops the walk."""
    rho = np.array([0.0, 0.5])
    g = np.array([3.0, 3.0])
    st = {}
    for t in range(60):
        new = O.adam_step(rho, g, st, lr=0.01)
        expect = np.minimum(rho + 0.01, 1.0)
        np.testing.assert_allclose(new, expect, rtol=0, atol=1e-9)
        rho = new
    assert rho[1] == 1.0 and abs(rho[0] - 0.6) < 1e-8


# ---------------------------------------------------------------------------
# Finite differences of F by rank-one updates (the large-grid gradient check)
# ---------------------------------------------------------------------------
def test_pixel_differences_by_rank_one_update_match_refactoring():
    """objective_pixel_differences evaluates F(rho +- h e_p) by Sherman-Morrison on one
    factorisation; the plain definition refactors the perturbed operator for each F.  Both agree
    to rounding on several wavelengths and sources, and the difference quotient approaches the
    adjoint gradient (Eq. 3)."""
    wl = W.make_small(22, 19, 4, (6, 5, 8, 7), n_omega=2, n_src=2, seed=31)
    rng = np.random.default_rng(4)
    pixels = rng.choice(wl.rho.size, 6, replace=False)
    h = 1e-3
    fd = O.objective_pixel_differences(wl, wl.rho, pixels, h, W.DELTA_EPS)
    brute = []
    for p in pixels:
        rp, rm = wl.rho.copy(), wl.rho.copy()
        rp.flat[p] += h
        rm.flat[p] -= h
        Fp, _, _ = O.design_iteration(wl, rp, wl.eps_full, W.DELTA_EPS)
        Fm, _, _ = O.design_iteration(wl, rm, wl.eps_full, W.DELTA_EPS)
        brute.append((Fp - Fm) / (2 * h))
    np.testing.assert_allclose(fd, brute, rtol=1e-9, atol=0)
    _, g, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    np.testing.assert_allclose(fd, g.ravel()[pixels], rtol=1e-5, atol=0)


# ---------------------------------------------------------------------------
# Transmission-target objective (Sec. III-IV: difference of calculated and target
# transmissions, minimised)
# ---------------------------------------------------------------------------
def test_target_objective_gradient_central_differences():
    """F = sum (|g^T E|^2 - t)^2 over two wavelengths and two sources: the adjoint gradient
    (Eq. 3 with the source 2 (|o|^2 - t) conj(o) g of Eq. 4) equals central differences of the
    oracle's own F on every design pixel, with targets on both sides of the current powers."""
    wl = W.make_small(16, 15, 3, (5, 4, 5, 6), n_omega=2, n_src=2, seed=8)
    F0, _, f0 = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    powers = [[abs(O.overlap(f0[(w, s)][0], wl.monitor_dense(w, s))) ** 2 for s in range(2)] for w in range(2)]
    targets = [[powers[w][s] * (0.5 if (w + s) % 2 else 1.7) for s in range(2)] for w in range(2)]
    F, g, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS, targets=targets)
    assert F > 0
    h = 1e-5
    fd = np.zeros_like(wl.rho)
    for idx in np.ndindex(wl.rho.shape):
        rp, rm = wl.rho.copy(), wl.rho.copy()
        rp[idx] += h
        rm[idx] -= h
        Fp, _, _ = O.design_iteration(wl, rp, wl.eps_full, W.DELTA_EPS, targets=targets)
        Fm, _, _ = O.design_iteration(wl, rm, wl.eps_full, W.DELTA_EPS, targets=targets)
        fd[idx] = (Fp - Fm) / (2 * h)
    assert O.rel_err(g, fd) < 1e-6


def test_target_objective_vanishes_at_the_target():
    """With every target equal to the current port power, F = 0 and its gradient is zero."""
    wl = W.make_small(14, 13, 3, (4, 4, 5, 4), n_omega=1, n_src=2, seed=9)
    _, _, f0 = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    targets = [[abs(O.overlap(f0[(0, s)][0], wl.monitor_dense(0, s))) ** 2 for s in range(2)]]
    F, g, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS, targets=targets)
    assert F < 1e-24 and np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("nx,ny,npml", [(12, 17, 3), (31, 9, 2), (20, 20, 4), (1, 13, 0), (40, 1, 0)])
def test_nested_dissection_factor_matches_dense_lapack(nx, ny, npml):
    """The nested-dissection order is a permutation of the grid with every separator line after
    the two halves it separates; SuperLU on the permuted matrix (threshold pivoting, one
    refinement step) gives the dense LAPACK solutions of Eq. 5 and 6."""
    p = O.nested_dissection(nx, ny, leaf=8)
    assert np.array_equal(np.sort(p), np.arange(nx * ny))
    k0dx = 2 * np.pi * 0.05 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 11), k0dx, npml)
    b = W.random_complex(nx * ny, 12)
    fac = O.Factor(A, (nx, ny))
    Ad = A.toarray()
    assert O.rel_err(fac.solve(b), np.linalg.solve(Ad, b)) < 1e-12
    assert O.rel_err(fac.solve_T(b), np.linalg.solve(Ad.T, b)) < 1e-12
    B = np.stack([b, W.random_complex(nx * ny, 13)], axis=1)
    np.testing.assert_allclose(fac.solve(B), np.linalg.solve(Ad, B), rtol=0, atol=1e-12 * np.abs(B).max() * 1e3)


def test_symmetric_ldlt_reconstructs_and_solves():
    """symmetric_ldlt: unit lower L and d with L diag(d) L^T = (D A)[order, order] to rounding, and the
    solve x = L^-T d^-1 L^-1 D b (in the permuted order) equals the dense LAPACK solve of A x = b."""
    nx, ny, npml = 9, 8, 2
    k0dx = 2 * np.pi * 0.05 / 1.55
    A = O.assemble(nx, ny, _rand_eps(nx, ny, 21), k0dx, npml).toarray()
    D = O.symmetrizer(nx, ny, k0dx, npml)
    M = D[:, None] * A
    order = O.nested_dissection(nx, ny, leaf=8)
    L, d = O.symmetric_ldlt(M, order)
    assert np.allclose(np.diag(L), 1) and np.abs(np.triu(L, 1)).max() == 0
    Mp = M[np.ix_(order, order)]
    assert np.abs(L @ np.diag(d) @ L.T - Mp).max() < 1e-12 * np.abs(Mp).max()
    b = W.random_complex(nx * ny, 22)
    y = np.linalg.solve(L, (D * b)[order])
    xp = np.linalg.solve(L.T, y / d)
    x = np.empty_like(xp)
    x[order] = xp
    assert O.rel_err(x, np.linalg.solve(A, b)) < 1e-11
