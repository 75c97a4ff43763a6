"""Host-side checks of the symbolic plan (CPU only, no GPU needed).

The library's nested-dissection plan is read back through the C ABI and
replayed by a plain NumPy dense multifrontal factorisation with the same
front layout, restricted pivoting and the same four sweep formulas the CUDA
kernels use (L, U for A x = b; U^T, L^T for A^T x = b).  Agreement with a
sparse direct solve shows the plan (orderings, front index sets, ownership of
original entries) and the sweep algebra are right before any GPU runs.
This NumPy replay is a test helper, not the oracle.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fdfd_oracle as O

fd = pytest.importorskip("paper_2307_05388_gb300.fdfd")


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(fd.LIB_PATH)
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(fd.LIB_PATH), "..", "include", "fdfd.h")).read()
    declared = set(re.findall(r"\b(fdfd_[a-z_]+)\s*\(", hdr))
    declared -= {"fdfd_ctx"}
    assert declared == set(fd.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def _plan(nx, ny, box, leaf):
    s = fd.Solver(nx, ny, 0.05, [2 * np.pi / 1.55], 2, box=box, options=fd.default_options(leaf_area=leaf))
    s.analyze()
    k, m, par, lev, des, idx = s.plan_fronts()
    s.close()
    offs = np.concatenate([[0], np.cumsum(k + m)])
    fronts = [dict(k=int(k[f]), m=int(m[f]), parent=int(par[f]), level=int(lev[f]), design=int(des[f]),
                   idx=idx[offs[f]:offs[f + 1]].copy()) for f in range(len(k))]
    return fronts


@pytest.mark.parametrize("nx,ny,box,leaf", [(13, 11, (3, 2, 5, 6), 8), (20, 17, (4, 5, 10, 8), 16),
                                            (9, 23, (0, 0, 9, 23), 4), (16, 16, (0, 0, 0, 0), 32)])
def test_plan_structure(nx, ny, box, leaf):
    fronts = _plan(nx, ny, box, leaf)
    piv = np.concatenate([f["idx"][:f["k"]] for f in fronts])
    assert sorted(piv.tolist()) == list(range(nx * ny))
    pos = np.empty(nx * ny, int)
    pos[piv] = np.arange(nx * ny)
    x0, y0, w, h = box
    for fi, f in enumerate(fronts):
        # boundary variables are eliminated later, sorted by elimination position
        kp = pos[f["idx"][:f["k"]]]
        bp = pos[f["idx"][f["k"]:]]
        assert np.all(bp > kp.max())
        assert np.all(np.diff(bp) > 0)
        if f["parent"] >= 0:
            p = fronts[f["parent"]]
            assert p["level"] > f["level"]
            assert set(f["idx"][f["k"]:].tolist()) <= set(p["idx"].tolist())
        # design flag: own design pixel or a design child
        ii, jj = f["idx"][:f["k"]] // ny, f["idx"][:f["k"]] % ny
        own = np.any((ii >= x0) & (ii < x0 + w) & (jj >= y0) & (jj < y0 + h)) if w * h else False
        kids = [c for c in fronts if c["parent"] == fi]
        assert f["design"] == int(own or any(c["design"] for c in kids))
        # leaf subtrees are wholly inside or outside the design box
        if not kids and w * h:
            inside = (ii >= x0) & (ii < x0 + w) & (jj >= y0) & (jj < y0 + h)
            assert inside.all() or (~inside).all()


def _multifrontal_replay(A, fronts, n):
    """Dense multifrontal LU with pivoting restricted to each front's k rows."""
    A = A.tocsr()
    At = A.T.tocsr()
    pos = np.empty(n, int)
    piv = np.concatenate([f["idx"][:f["k"]] for f in fronts])
    pos[piv] = np.arange(n)
    out = []
    for fi, f in enumerate(fronts):
        idx = f["idx"]
        nn, k = len(idx), f["k"]
        loc = {c: a for a, c in enumerate(idx)}
        F = np.zeros((nn, nn), complex)
        # original entries owned by this front: min(pos r, pos c) is one of its pivots
        for a in range(k):
            p = idx[a]
            row = A.getrow(p)
            for q, v in zip(row.indices, row.data):
                if pos[q] >= pos[p]:
                    F[a, loc[q]] += v
            col = At.getrow(p)                      # column p of A
            for q, v in zip(col.indices, col.data):
                if pos[q] > pos[p]:
                    F[loc[q], a] += v
        for c in out:
            if c["parent"] == fi:
                cb = c["idx"][c["k"]:]
                ia = [loc[x] for x in cb]
                F[np.ix_(ia, ia)] += c["S"]
        perm = np.arange(k)
        for j in range(k):
            pr = j + int(np.argmax(np.abs(F[j:k, j])))
            if pr != j:
                F[[j, pr], :] = F[[pr, j], :]
                perm[[j, pr]] = perm[[pr, j]]
            F[j + 1:, j] /= F[j, j]
            F[j + 1:, j + 1:] -= np.outer(F[j + 1:, j], F[j, j + 1:])
        out.append(dict(f, F=F, perm=perm, S=F[k:, k:].copy()))
    return out


def _replay_solve(fr, b, transpose):
    n = len(b)
    x = np.zeros(n, complex)
    vec = [None] * len(fr)
    kids = [[] for _ in fr]
    for i, f in enumerate(fr):
        if f["parent"] >= 0:
            kids[f["parent"]].append(i)

    def gather(i, permute):
        f = fr[i]
        idx, k = f["idx"], f["k"]
        loc = {c: a for a, c in enumerate(idx)}
        v = np.zeros(len(idx), complex)
        v[:k] = b[idx[:k]]
        for c in kids[i]:
            cb = fr[c]["idx"][fr[c]["k"]:]
            for t, cell in enumerate(cb):
                v[loc[cell]] += vec[c][fr[c]["k"] + t]
        if permute:
            v[:k] = v[:k][f["perm"]]
        return v

    for i, f in enumerate(fr):                      # bottom-up
        F, k = f["F"], f["k"]
        v = gather(i, permute=not transpose)
        if not transpose:
            L = np.tril(F[:k, :k], -1) + np.eye(k)
            y = np.linalg.solve(L, v[:k])
            v[k:] -= F[k:, :k] @ y
            v[:k] = y
        else:
            U = np.triu(F[:k, :k])
            wv = np.linalg.solve(U.T, v[:k])
            v[k:] -= F[:k, k:].T @ wv
            v[:k] = wv
        vec[i] = v
    for i in reversed(range(len(fr))):             # top-down
        f = fr[i]
        F, k, idx = f["F"], f["k"], f["idx"]
        xm = x[idx[k:]]
        if not transpose:
            U = np.triu(F[:k, :k])
            x[idx[:k]] = np.linalg.solve(U, vec[i][:k] - F[:k, k:] @ xm)
        else:
            L = np.tril(F[:k, :k], -1) + np.eye(k)
            q = np.linalg.solve(L.T, vec[i][:k] - F[k:, :k].T @ xm)
            x[idx[f["perm"]]] = q
    return x


@pytest.mark.parametrize("nx,ny,box,leaf", [(13, 11, (3, 2, 5, 6), 8), (18, 15, (4, 3, 9, 7), 16)])
def test_multifrontal_replay_matches_sparse_solve(nx, ny, box, leaf):
    fronts = _plan(nx, ny, box, leaf)
    rng = np.random.default_rng(3)
    eps = W.EPS_SIO2 + W.DELTA_EPS * rng.uniform(0, 1, (nx, ny))
    A = O.assemble(nx, ny, eps, 2 * np.pi * 0.05 / 1.55, 3)
    fr = _multifrontal_replay(A, fronts, nx * ny)
    b = W.random_complex(nx * ny, 4)
    x = _replay_solve(fr, b, transpose=False)
    assert O.rel_err(x, spla.spsolve(A.tocsc(), b)) < 1e-10
    xt = _replay_solve(fr, b, transpose=True)
    assert O.rel_err(xt, spla.spsolve(A.T.tocsc(), b)) < 1e-10


def test_operation_counter_model_on_host():
    """The symbolic phase counts once however often fdfd_analyze is called (Sec. II, Fig. 1)."""
    s = fd.Solver(30, 30, 0.05, [4.0, 4.1], 4, box=(5, 5, 20, 20))
    s.analyze()
    s.analyze()
    assert s.stats()["sf"] == 1
    s.close()


def test_create_rejects_bad_arguments():
    with pytest.raises(fd.FdfdError):
        fd.Solver(10, 10, 0.05, [4.0], 6)                 # PML thicker than half the grid
    with pytest.raises(fd.FdfdError):
        fd.Solver(10, 10, 0.05, [4.0], 2, box=(5, 5, 8, 8))  # box outside the grid
    with pytest.raises(fd.FdfdError):
        fd.Solver(10, 10, 0.05, [-1.0], 2)
    with pytest.raises(fd.FdfdError):
        fd.Solver(10, 10, 0.05, [4.0], 2, options=fd.default_options(mode=3))   # no such mode
    # out-of-range options are clamped, not rejected
    s = fd.Solver(10, 10, 0.05, [4.0], 2, options=fd.default_options(ir_tol=float("nan"), growth_bound=-1.0,
                                                                      gmres_restart=99, tensor_form=9))
    s.analyze()
    s.close()


@pytest.mark.parametrize("nx,ny,npml,box,leaf,binary", [(30, 30, 4, (8, 8, 14, 14), 16, False),
                                                         (44, 36, 6, (10, 8, 24, 20), 32, True)])
def test_symmetric_ldlt_in_plan_order_without_pivoting(nx, ny, npml, box, leaf, binary):
    """The premise of a complex-symmetric variant: D A (symmetric by reciprocity) factors as
    L diag(d) L^T in the plan's elimination order with no pivoting at all, multifrontally (each
    front's update matrix extend-added into its parent), with modest growth.  Checked by
    rebuilding P^T (D A) P from the factors densely."""
    k0dx = 2 * np.pi * 0.04 / 1.55
    rng = np.random.default_rng(nx)
    eps = np.full((nx, ny), W.EPS_SIO2)
    x0, y0, w, h = box
    rho = rng.uniform(0, 1, (w, h))
    eps[x0:x0 + w, y0:y0 + h] += W.DELTA_EPS * ((rho > 0.5) if binary else rho)
    S = (O.symmetrizer(nx, ny, k0dx, npml)[:, None] * O.assemble(nx, ny, eps, k0dx, npml).toarray())
    fronts = _plan(nx, ny, box, leaf)
    n = nx * ny
    piv = np.concatenate([f["idx"][:f["k"]] for f in fronts])
    pos = np.empty(n, int)
    pos[piv] = np.arange(n)
    L = np.eye(n, dtype=complex)
    d = np.zeros(n, complex)
    upd = {}
    growth = 0.0
    for fi, f in enumerate(fronts):
        idx, k = f["idx"], f["k"]
        F = np.zeros((len(idx), len(idx)), complex)
        for a in range(k):                         # entries whose earlier variable is a pivot here
            for b_, q in enumerate(idx):
                if pos[q] >= pos[idx[a]]:
                    F[a, b_] = S[idx[a], q]
                    F[b_, a] = S[q, idx[a]]
        loc = {c: a for a, c in enumerate(idx)}
        for c, (cidx, cS) in list(upd.items()):
            if fronts[c]["parent"] == fi:
                ia = [loc[x] for x in cidx]
                F[np.ix_(ia, ia)] += cS
                del upd[c]
        for j in range(k):
            l = F[j + 1:, j] / F[j, j]
            growth = max(growth, float(np.abs(l).max()) if l.size else 0.0)
            F[j + 1:, j + 1:] -= np.outer(l, F[j, j + 1:])
            d[pos[idx[j]]] = F[j, j]
            L[pos[idx[j + 1:]], pos[idx[j]]] = l
        upd[fi] = (idx[k:], F[k:, k:].copy())
    Sp = S[np.ix_(piv, piv)]
    assert np.allclose(Sp, Sp.T, rtol=0, atol=1e-12)
    assert np.linalg.norm(L @ np.diag(d) @ L.T - Sp) <= 1e-11 * np.linalg.norm(Sp)
    assert growth < 1e4
