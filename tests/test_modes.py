"""Parity of the library's mode solver (fdfd_slab_modes, host code in libfdfd.so) with the
oracle's (LAPACK symmetric tridiagonal eigensolver), on the CPU.

The two share no code: bisection on Sturm counts plus inverse iteration against LAPACK.
Eigenvalues agree to a few units of rounding of the matrix norm.  Profiles agree to 1e-11
in the 2-norm, or 1e-10 for the nearly degenerate supermodes of a coupler (measured: below
5e-13).  The sign convention is the same documented rule on both sides and is compared
exactly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fdfd_oracle as O

fd = pytest.importorskip("paper_2307_05388_gb300.fdfd")


def _slab(dx, d=0.48, width=4.0, offset=0):
    ncore = int(round(d / dx))
    ny = int(round(width / dx))
    eps = np.full(ny, W.EPS_SIO2)
    a = (ny - ncore) // 2 + offset
    eps[a:a + ncore] = W.EPS_SI
    return eps


def _check(eps, k0dx, n_modes, vec_tol=1e-11):
    mu, th, phi = fd.slab_modes(eps, k0dx, n_modes)
    mu_o, th_o, phi_o = O.slab_modes(eps, k0dx, n_modes)
    scale = np.max(np.abs(k0dx ** 2 * eps - 2)) + 2
    np.testing.assert_allclose(mu, mu_o, rtol=0, atol=64 * np.finfo(float).eps * scale)
    np.testing.assert_array_equal(np.isnan(th), np.isnan(th_o))
    ok = ~np.isnan(th)
    np.testing.assert_allclose(th[ok], th_o[ok], rtol=1e-12, atol=1e-14)
    for k in range(n_modes):
        assert np.linalg.norm(phi[k] - phi_o[k]) < vec_tol, k
    np.testing.assert_allclose(phi @ phi.T, np.eye(n_modes), atol=1e-12)
    return mu, th, phi


@pytest.mark.parametrize("dx,offset", [(0.04, 0), (0.02, 0), (0.02, 7), (0.01, -3)])
def test_slab_modes_match_oracle(dx, offset):
    eps = _slab(dx, offset=offset)
    k0dx = 2 * np.pi * dx / 1.55
    _check(eps, k0dx, 3)


def test_two_guides_and_wavelengths():
    """Two 400 nm guides 300 nm apart (a coupler cross-section) at the band edges: nearly
    degenerate supermode pairs, the case inverse iteration needs re-orthogonalisation for."""
    dx = 0.02
    eps = np.full(240, W.EPS_SIO2)
    eps[90:110] = W.EPS_SI
    eps[125:145] = W.EPS_SI
    for lam in (1.50, 1.55, 1.60):
        _check(eps, 2 * np.pi * dx / lam, 4, vec_tol=1e-10)


def test_random_lines_and_edge_sizes():
    rng = np.random.default_rng(3)
    for ny, nm in ((1, 1), (2, 2), (3, 3), (17, 5), (64, 8)):
        eps = W.EPS_SIO2 + W.DELTA_EPS * rng.uniform(0, 1, ny)
        mu, th, phi = fd.slab_modes(eps, 0.3, nm)
        mu_o, _, phi_o = O.slab_modes(eps, 0.3, nm)
        np.testing.assert_allclose(mu, mu_o, rtol=0, atol=1e-13)
        # random lines can have close eigenvalues: compare the spanned subspace, then the convention
        np.testing.assert_allclose(np.abs(phi @ phi_o.T), np.eye(nm), atol=1e-7)


def test_sign_convention_and_uniform_closed_form():
    n, eps, k0dx = 41, 2.085, 0.2
    mu, th, phi = fd.slab_modes(np.full(n, eps), k0dx, 3)
    q = np.arange(1, 4)
    np.testing.assert_allclose(mu, k0dx ** 2 * eps - 4 * np.sin(q * np.pi / (2 * (n + 1))) ** 2, atol=1e-14)
    for k in range(3):
        j = int(np.argmax(np.abs(phi[k]) >= 0.5 * np.abs(phi[k]).max()))
        assert phi[k][j] > 0


def test_bad_arguments():
    with pytest.raises(fd.FdfdError):
        fd.slab_modes(np.ones(5), 0.2, 6)
    with pytest.raises(fd.FdfdError):
        fd.slab_modes(np.ones(5), 0.2, 0)
    with pytest.raises(fd.FdfdError):
        fd.slab_modes(np.array([1.0, np.nan, 1.0]), 0.2, 1)
    with pytest.raises(fd.FdfdError):
        fd.slab_modes(np.ones(4), float("inf"), 1)


def test_full_height_cross_section():
    """A cross-section as tall as the largest grid (1760 cells, 50 nm): three modes of a 480 nm
    guide, against the oracle."""
    dx = 0.05
    eps = np.full(1760, W.EPS_SIO2)
    eps[870:880] = W.EPS_SI
    _check(eps, 2 * np.pi * dx / 1.31, 3)
