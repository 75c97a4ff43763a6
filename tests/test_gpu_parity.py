"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative field error <= 1e-8 and relative gradient error <= 1e-6
after refinement (both against the complex128 oracle); bit-exact equality
for the cached design refactor against a fresh factorisation (deterministic
kernels, no atomics), and exact integer operation counts (Sec. III-IV).
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import fdfd_oracle as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402
from tests import _gpu_util as U  # noqa: E402

FIELD_TOL = 1e-8
GRAD_TOL = 1e-6
DEV = "cuda"


def _oracle_fields(wl, eps, transpose=False, b=None):
    out = []
    for w, k0dx in enumerate(wl.k0dx()):
        fac = O.Factor(O.assemble(wl.nx, wl.ny, eps, k0dx, wl.npml), (wl.nx, wl.ny))
        for s in range(b.shape[1]):
            out.append(fac.solve_T(b[w, s]) if transpose else fac.solve(b[w, s]))
    return np.stack(out).reshape(b.shape)


def _solve_case(wl, nrhs, mode, seed=5, transpose=False, **opts):
    s = U.make_solver(wl, mode=mode, **opts)
    eps = wl.eps_full()
    s.factor(torch.from_numpy(eps.reshape(-1).copy()).to(DEV))
    b = W.random_complex((wl.n_omega, nrhs, wl.n), seed)
    x = s.solve(torch.from_numpy(b).to(DEV), transpose=transpose)
    torch.cuda.synchronize()
    ref = _oracle_fields(wl, eps, transpose, b)
    return x.cpu().numpy(), ref, s


@pytest.mark.parametrize("transpose", [False, True])
def test_c1_mixed_forward_and_transpose(transpose):
    wl = W.make("c1")
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, transpose=transpose)
    err = O.rel_err(x, ref)
    st = s.stats()
    print(f"c1 transpose={transpose} field err {err:.2e} iters {st['ir_iters']} resid {st['ir_resid']:.1e}")
    assert err <= FIELD_TOL


@pytest.mark.parametrize("transpose", [False, True])
def test_c1_f64_direct(transpose):
    wl = W.make("c1")
    x, ref, _ = _solve_case(wl, 1, FD.MODE_F64, transpose=transpose)
    assert O.rel_err(x, ref) <= 1e-10


def test_c1_raw_fp32_error_reported():
    """The unrefined FP32-factor solution is reported, not pinned (only sanity-bounded)."""
    wl = W.make("c1")
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, ir_max_iter=0)
    err = O.rel_err(x, ref)
    print(f"c1 raw FP32-factor field error {err:.3e}")
    assert err < 1e-2


@pytest.mark.parametrize("nx,ny,npml,box,n_omega,nrhs,leaf", [
    (37, 29, 5, (9, 7, 15, 11), 2, 3, 32),     # ragged, several wavelengths and sources
    (61, 45, 8, (13, 10, 30, 20), 1, 2, 16),   # more levels, large-front path
    (130, 97, 10, (20, 15, 90, 60), 1, 1, 32), # fronts above the shared-memory size
    (1, 40, 0, (0, 5, 1, 20), 1, 1, 4),        # one column, no PML
    (2, 2, 0, (0, 0, 2, 2), 1, 1, 1),          # degenerate 2 x 2
    (24, 24, 4, (0, 0, 0, 0), 1, 1, 64),       # no design box
])
@pytest.mark.parametrize("mode", [FD.MODE_MIXED, FD.MODE_F64])
def test_small_grids(nx, ny, npml, box, n_omega, nrhs, leaf, mode):
    wl = W.make_small(nx, ny, npml, box if box[2] else (0, 0, 1, 1), n_omega=n_omega, n_src=1, seed=7)
    if not box[2]:
        wl.box = (0, 0, 0, 0)
    for tr in (False, True):
        x, ref, _ = _solve_case(wl, nrhs, mode, transpose=tr, leaf_area=leaf)
        assert O.rel_err(x, ref) <= (FIELD_TOL if mode == FD.MODE_MIXED else 1e-10)


@pytest.mark.parametrize("nx,ny,npml,box,leaf", [(130, 97, 10, (20, 15, 90, 60), 32),
                                                 (61, 45, 8, (13, 10, 30, 20), 16)])
@pytest.mark.parametrize("mode", [FD.MODE_MIXED, FD.MODE_F64])
def test_block_local_pivoting(nx, ny, npml, box, leaf, mode):
    """Pivoting restricted to each panel's diagonal block still reaches the oracle."""
    wl = W.make_small(nx, ny, npml, box, n_omega=2, n_src=1, seed=23)
    for tr in (False, True):
        x, ref, _ = _solve_case(wl, 2, mode, transpose=tr, leaf_area=leaf, pivoting=1)
        assert O.rel_err(x, ref) <= (FIELD_TOL if mode == FD.MODE_MIXED else 1e-10)


def test_refactor_design_is_bitwise_fresh_factor():
    """Cached refactor of the design fronts == full factorisation of the new eps, bit for bit."""
    wl = W.make("c1")
    rho2 = np.random.default_rng(9).uniform(0, 1, wl.rho.shape)
    s1 = U.make_solver(wl, ir_max_iter=0)
    s1.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    s1.refactor_design(U.eps_design_tensor(wl, rho2))
    s2 = U.make_solver(wl, ir_max_iter=0)
    s2.factor(torch.from_numpy(wl.eps_full(rho2).reshape(-1).copy()).to(DEV))
    b = torch.from_numpy(W.random_complex((1, 2, wl.n), 3)).to(DEV)
    for tr in (False, True):
        x1 = s1.solve(b, transpose=tr)
        x2 = s2.solve(b, transpose=tr)
        assert torch.equal(x1, x2)
    # and the refined solution of the refactored system matches the oracle
    s1.set_options(ir_max_iter=40)
    x = s1.solve(b).cpu().numpy()
    ref = _oracle_fields(wl, wl.eps_full(rho2), False, b.cpu().numpy())
    assert O.rel_err(x, ref) <= FIELD_TOL


def test_design_iteration_c1_objective_and_gradient():
    wl = W.make("c1")
    prob = U.problem(wl)
    rho = wl.rho.copy()
    for it in range(wl.iterations):
        F, g = prob.iteration(U.eps_design_tensor(wl, rho))
        torch.cuda.synchronize()
        F_ref, g_ref, _ = O.design_iteration(wl, rho, wl.eps_full, W.DELTA_EPS)
        grad_rho = g.cpu().numpy().reshape(wl.rho.shape) * W.DELTA_EPS
        assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
        assert O.rel_err(grad_rho, g_ref) <= GRAD_TOL
        rho = O.sign_step(rho, g_ref, wl.step)       # same rho on both sides for the next step


def test_c2_design_loop_three_steps_lock_step():
    """The first three sign steps of C2's loop (340 x 340, the library's default options, the design
    refactor from the second step on): F at 1e-8 and dF/drho at 1e-6 of the oracle at every step,
    both sides stepping from the oracle's gradient so that they see the same design."""
    wl = W.make("c2")
    prob = U.problem(wl)
    rho = wl.rho.copy()
    for it in range(3):
        F, g = prob.iteration(U.eps_design_tensor(wl, rho))
        torch.cuda.synchronize()
        F_ref, g_ref, _ = O.design_iteration(wl, rho, wl.eps_full, W.DELTA_EPS)
        err = O.rel_err(g.cpu().numpy().reshape(wl.rho.shape) * W.DELTA_EPS, g_ref)
        print(f"c2 step {it}: F {float(F):.10g} (oracle {F_ref:.10g}), gradient error {err:.2e}")
        assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
        assert err <= GRAD_TOL
        rho = O.sign_step(rho, g_ref, wl.step)


def test_c4_recipe_adam_loop_through_the_autograd_function():
    """C4's differentiable loop -- four wavelengths 1.53-1.57 um at dx = 40 nm, Adam at lr 0.01
    ascending F, the gradient from FdfdObjective's backward (the transpose solves on the forward
    pass's cached factors) chained to rho by autograd -- on a 200 x 200 grid with a 150 x 150
    design, four steps in lock step with the oracle: F and dF/drho at every step, and the device
    Adam update of the device gradient against the oracle's Adam update of its own."""
    from paper_2307_05388_gb300 import optimize as OPT
    wl = W.make("c4", grid=200, design=150)
    assert wl.optimizer == "adam" and wl.n_omega == 4
    prob = U.problem(wl)
    opt, state = OPT.Adam(wl.step), {}
    rho = wl.rho.copy()
    for it in range(4):
        r = torch.from_numpy(rho.reshape(-1).copy()).to(DEV).requires_grad_(True)
        F = prob(W.EPS_SIO2 + W.DELTA_EPS * r)
        F.backward()
        F = F.detach()
        F_ref, g_ref, _ = O.design_iteration(wl, rho, wl.eps_full, W.DELTA_EPS)
        g = r.grad.cpu().numpy().reshape(wl.rho.shape)
        err = O.rel_err(g, g_ref)
        nxt = opt.step(r.detach(), r.grad).cpu().numpy().reshape(wl.rho.shape)
        rho = O.adam_step(rho, g_ref, state, lr=wl.step)
        step_err = np.abs(nxt - rho).max()
        print(f"c4@200 Adam step {it}: F {float(F):.10g} (oracle {F_ref:.10g}), gradient error {err:.2e}, "
              f"update difference {step_err:.1e}")
        assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
        assert err <= GRAD_TOL
        assert step_err <= 1e-7


def test_design_loop_checkpoint_resume_c1(tmp_path):
    """C1's loop with Adam (lr 0.05) through the library: four iterations without a break against
    two with a checkpoint, then a resume into a new solver (analysis and full factorisation again)
    and two more.  The densities agree to rounding: FGMRES sizes its first cycle from the solver's
    previous solve, which a new solver does not have, while a lost moment or step count would move
    pixels by lr.  The resumed loop's last F matches the oracle's F at its density."""
    from paper_2307_05388_gb300 import optimize as OPT
    wl = W.make("c1")
    rho0 = torch.from_numpy(wl.rho.reshape(-1).copy()).to(DEV)

    def loop_objective():
        p = U.problem(wl)
        return p, OPT.linear_density_objective(p, W.EPS_SIO2, W.EPS_SI)

    p1, f1 = loop_objective()
    whole = OPT.DesignLoop(f1, OPT.Adam(0.05), rho0)
    whole.run(4)
    ck = str(tmp_path / "c1_loop.pt")
    p2, f2 = loop_objective()
    OPT.DesignLoop(f2, OPT.Adam(0.05), rho0, checkpoint=ck, every=2).run(2)
    p3, f3 = loop_objective()
    resumed = OPT.DesignLoop.resume(ck, f3, OPT.Adam(0.05), device=DEV)
    assert resumed.iteration == 2 and resumed.rho.is_cuda
    resumed.run(2)
    diff = float((resumed.rho - whole.rho).abs().max())
    print(f"c1 loop resumed after 2 of 4 Adam steps: largest density difference {diff:.1e}")
    assert diff <= 1e-6
    assert np.allclose(resumed.history, whole.history, rtol=1e-8, atol=0)
    rho = resumed.rho.cpu().numpy().reshape(wl.rho.shape)
    F, _ = f3(resumed.rho)
    F_ref, _, _ = O.design_iteration(wl, rho, wl.eps_full, W.DELTA_EPS)
    assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
    for p in (p1, p2, p3):
        p.solver.close()


def test_multiwavelength_multisource_gradient():
    wl = W.make_small(40, 36, 6, (10, 9, 18, 16), n_omega=3, n_src=2, seed=13)
    prob = U.problem(wl)
    F, g = prob.iteration(U.eps_design_tensor(wl, wl.rho))
    F_ref, g_ref, _ = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    assert abs(float(F) - F_ref) <= 1e-8 * abs(F_ref)
    assert O.rel_err(g.cpu().numpy().reshape(wl.rho.shape) * W.DELTA_EPS, g_ref) <= GRAD_TOL


def test_autograd_function_matches_finite_differences():
    wl = W.make_small(20, 18, 4, (6, 5, 6, 5), n_omega=2, n_src=1, seed=17)
    prob = U.problem(wl)
    rho = torch.from_numpy(wl.rho.copy()).to(DEV).requires_grad_(True)
    F = prob(W.EPS_SIO2 + rho * W.DELTA_EPS)
    F.backward()
    g = rho.grad.cpu().numpy()
    h = 1e-4
    fd = np.zeros_like(wl.rho)
    for idx in np.ndindex(wl.rho.shape):
        rp, rm = wl.rho.copy(), wl.rho.copy()
        rp[idx] += h
        rm[idx] -= h
        Fp, _, _ = O.design_iteration(wl, rp, wl.eps_full, W.DELTA_EPS)
        Fm, _, _ = O.design_iteration(wl, rm, wl.eps_full, W.DELTA_EPS)
        fd[idx] = (Fp - Fm) / (2 * h)
    assert O.rel_err(g, fd) <= GRAD_TOL


def _counts(n_omega, n_src, mode, iters=2):
    wl = W.make_small(16, 16, 3, (5, 5, 6, 6), n_omega=n_omega, n_src=n_src, seed=1)
    prob = U.problem(wl, mode=mode)
    out = []
    for it in range(iters):
        prob.solver.reset_counters()
        prob.iteration(U.eps_design_tensor(wl, wl.rho))
        st = prob.solver.stats()
        out.append({"SF": st["sf"], "NF": st["nf"], "BS": st["bs"]})
    return out


def test_operation_counts_match_paper():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "operation_counts.json")))
    for key in ("duplexer_10_wavelengths_1_source", "mode_mux_6_wavelengths_3_sources"):
        case = gold[key]
        cached = _counts(case["n_omega"], case["n_src"], FD.MODE_MIXED)
        # first iteration: the symbolic phase runs once inside the first factorisation
        assert cached[0] == case["cached_first"]
        assert cached[1] == case["cached_later"]
        plain = _counts(case["n_omega"], case["n_src"], FD.MODE_PLAIN, iters=1)
        assert plain[0] == case["uncached"]


def test_growth_over_the_bound_repivots_and_keeps_converging_fp32_factors():
    """A growth bound below any real growth sends the block-local factors to complex FP32 LU with
    partial pivoting over all pivot rows; their growth is finite and refinement converges on them,
    so they are kept (no FP64 refactor) and the fields match the oracle."""
    wl = W.make("c1")
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, growth_bound=1e-30)
    st = s.stats()
    assert st["repivots"] >= 1 and st["fallbacks"] == 0
    assert O.rel_err(x, ref) <= FIELD_TOL


@pytest.mark.parametrize("restart", [8, 16])
def test_fgmres_long_cycles_with_a_weak_preconditioner(restart):
    """FGMRES with a cycle of 8 or 16 Krylov vectors on a deliberately weak preconditioner
    (TF32 update matrices in every front) and a tight tolerance (1e-13): the refined fields
    still match the oracle, forward and transpose, with no FP64 fallback."""
    wl = W.make("c1")
    for tp in (False, True):
        x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, transpose=tp, tensor_form=1, tensor_min_m=1,
                                tensor_min_tiles=1, gmres_restart=restart, ir_tol=1e-13)
        st = s.stats()
        err = O.rel_err(x, ref)
        print(f"restart {restart} transpose={tp}: {st['ir_iters']} iterations, residual {st['ir_resid']:.1e}, "
              f"field err {err:.1e}, FP64 fallbacks {st['fallbacks']}")
        assert st["ir_resid"] <= 1e-13 and st["fallbacks"] == 0
        assert err <= FIELD_TOL


def test_fgmres_cycle_beyond_eight_vectors():
    """C2 with TF32 update matrices in every front and a 1e-13 tolerance needs more than eight
    Krylov vectors in one 16-vector cycle, so the Arnoldi projections onto V_8.. are formed and
    reduced; the fields match the oracle."""
    wl = W.make("c2")
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, tensor_form=1, tensor_min_m=1, tensor_min_tiles=1,
                            gmres_restart=16, ir_tol=1e-13)
    st = s.stats()
    print(f"{st['ir_iters']} iterations, residual {st['ir_resid']:.1e}, field err {O.rel_err(x, ref):.1e}")
    assert st["ir_iters"] >= 9 and st["ir_resid"] <= 1e-13 and st["fallbacks"] == 0
    assert O.rel_err(x, ref) <= FIELD_TOL


def test_unconverged_refinement_sends_factorisation_to_f64():
    """One FGMRES iteration cannot reach 1e-12 on complex FP32 factors: the factorisation is
    redone in FP64 and the solve repeated, which then converges and matches the oracle."""
    wl = W.make("c1")
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, ir_max_iter=1, ir_tol=1e-12)
    st = s.stats()
    assert st["fallbacks"] == 1 and st["ir_resid"] <= 1e-12
    assert O.rel_err(x, ref) <= FIELD_TOL


def _raw_growth(wl, pivoting):
    s = U.make_solver(wl, pivoting=pivoting, ir_max_iter=0)
    s.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    s.solve(torch.from_numpy(W.random_complex((wl.n_omega, 1, wl.n), 3)).to(DEV))
    return s.stats()["growth"]


# a coarse (dx = 0.1 um) seeded grid whose block-local pivoting grows about twice as much as partial
# pivoting over all pivot rows (found by scanning seeds and spacings), so the rung always engages
REPIVOT_CASE = dict(nx=130, ny=97, npml=10, box=(20, 15, 90, 60), seed=5, dx=0.1)


@pytest.mark.parametrize("name", ["c1", "c2", "coarse130"])
def test_growth_repivot_rung_before_f64(name):
    """Block-local pivoting whose growth exceeds the bound is redone in complex FP32 with
    partial pivoting over all pivot rows; with that growth inside the bound there is no
    FP64 fallback, and the refined fields still match the oracle.  The coarse 130 x 97 case
    always engages the rung; C1 and C2 only where their growths differ enough."""
    wl = W.make_small(**REPIVOT_CASE) if name == "coarse130" else W.make(name)
    g_pp, g_bl = _raw_growth(wl, 0), _raw_growth(wl, 1)
    print(f"{name}: growth with partial pivoting {g_pp:.3g}, block-local {g_bl:.3g}")
    if name == "coarse130":
        assert g_bl > 1.5 * g_pp, "the seeded coarse case no longer separates the two pivoting rules"
    elif not g_bl > 1.5 * g_pp:
        pytest.skip("block-local growth not above the partial-pivoting growth here")
    bound = float(np.sqrt(g_pp * g_bl))
    x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, growth_bound=bound)
    st = s.stats()
    assert st["repivots"] == 1 and st["fallbacks"] == 0
    assert st["growth"] <= bound
    assert O.rel_err(x, ref) <= FIELD_TOL


def test_nan_permittivity_reports_pivot_error():
    wl = W.make_small(12, 12, 2, (3, 3, 4, 4), seed=2)
    s = U.make_solver(wl)
    eps = wl.eps_full().reshape(-1).copy()
    eps[40] = np.nan
    s.factor(torch.from_numpy(eps).to(DEV))
    b = torch.from_numpy(W.random_complex((1, 1, wl.n), 1)).to(DEV)
    with pytest.raises(FD.FdfdError) as e:
        s.solve(b)
    assert e.value.status == 5


@pytest.mark.parametrize("k,m,planes", [(16, 128, 3), (5, 129, 3), (37, 200, 3), (37, 200, 2), (37, 200, 1),
                                         (1, 1, 3), (340, 340, 3), (340, 340, 2), (250, 700, 3), (250, 700, 1),
                                         (512, 1900, 3)])
def test_tensor_core_update_matrix(k, m, planes):
    """The tcgen05 update matrix of one front, S = F22 - L21 U12 (Sec. II), against the same
    product in complex128: componentwise error relative to |L21| |U12| + |F22| within the
    bound of the operand form (BF16 three-way split or TF32 hi + lo: FP32-class; TF32: 2^-11);
    nothing outside F22 is written.  Sizes span one tile, ragged row/column/pivot tails and
    several tiles."""
    wl = W.make("c1")
    s = U.make_solver(wl)
    n = k + m
    ld = -(-n // 4) * 4 + 4
    g = torch.Generator().manual_seed(1000 * k + m)
    F = torch.complex(torch.randn(n, ld, generator=g), torch.randn(n, ld, generator=g)).to(torch.complex64)
    F_dev = F.to(DEV)
    s.selftest_schur_tc(F_dev, k, planes)
    out = F_dev.cpu()
    F64 = F.to(torch.complex128)
    ref = F64[k:n, k:n] - F64[k:n, :k] @ F64[:k, k:n]
    scale = F64[k:n, :k].abs() @ F64[:k, k:n].abs() + F64[k:n, k:n].abs()
    err = ((out[k:n, k:n].to(torch.complex128) - ref).abs() / scale).max().item()
    tol = 2e-3 if planes == 1 else 2e-6
    print(f"k={k} m={m} planes={planes}: componentwise error {err:.2e} (tol {tol:.0e})")
    assert err <= tol
    assert torch.equal(out[:k], F[:k]) and torch.equal(out[:, :k], F[:, :k]) and torch.equal(out[:, n:], F[:, n:])


@pytest.mark.parametrize("planes", [3, 2, 1])
def test_c1_tensor_core_update_matrices_every_front(planes):
    """Every large front with a boundary sends its update matrix through the tensor cores
    (tensor_min_m = tensor_min_tiles = 1): fields within 1e-8 of the oracle after refinement, forward and
    transpose; the raw FP32-factor error is reported beside the SIMT form's."""
    wl = W.make("c1")
    errs = {}
    for tp in (False, True):
        x, ref, s = _solve_case(wl, 1, FD.MODE_MIXED, transpose=tp, tensor_form=planes, tensor_min_m=1,
                                tensor_min_tiles=1)
        err = O.rel_err(x, ref)
        print(f"planes={planes} transpose={tp}: field err {err:.2e} iters {s.stats()['ir_iters']}")
        assert err <= FIELD_TOL
    for tp_planes in (0, planes):
        x, ref, _ = _solve_case(wl, 1, FD.MODE_MIXED, tensor_form=tp_planes, tensor_min_m=1, tensor_min_tiles=1,
                                ir_max_iter=0)
        errs[tp_planes] = O.rel_err(x, ref)
    print(f"raw FP32-factor error: SIMT {errs[0]:.2e}, tensor cores (form {planes}) {errs[planes]:.2e}")
    assert errs[planes] <= (1e4 if planes == 1 else 10.0) * errs[0]


def test_bounded_sweep_wait_gives_up_and_context_survives():
    """A dataflow-sweep wait on a counter nothing sets gives up (FDFD_ERR_TIMEOUT, about a
    second) instead of hanging; the context then still solves correctly."""
    wl = W.make("c1")
    s = U.make_solver(wl)
    assert s.selftest_wait() == 7
    x, ref, _ = _solve_case(wl, 1, FD.MODE_MIXED)
    assert O.rel_err(x, ref) <= FIELD_TOL
    s2 = U.make_solver(wl)
    s2.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    assert s2.selftest_wait() == 7
    b = torch.from_numpy(W.random_complex((1, 1, wl.n), 5)).to(DEV)
    x2 = s2.solve(b).cpu().numpy()
    ref2 = _oracle_fields(wl, wl.eps_full(), False, b.cpu().numpy())
    assert O.rel_err(x2, ref2) <= FIELD_TOL


def test_tensor_core_pipeline_wait_gives_up_and_context_survives():
    """The tensor-core update matrix's bounded mbarrier wait, run on a barrier nothing arrives at
    (1 ms limit), gives up with FDFD_ERR_TIMEOUT instead of hanging; the context then factorises
    (with the tensor-core update matrices) and solves correctly."""
    wl = W.make("c1")
    s = U.make_solver(wl, tensor_min_m=1, tensor_min_tiles=1)
    assert s.selftest_mbar_wait() == 7
    assert s.selftest_mbar_wait() == 7
    s.factor(torch.from_numpy(wl.eps_full().reshape(-1).copy()).to(DEV))
    b = torch.from_numpy(W.random_complex((1, 1, wl.n), 5)).to(DEV)
    x = s.solve(b).cpu().numpy()
    ref = _oracle_fields(wl, wl.eps_full(), False, b.cpu().numpy())
    assert O.rel_err(x, ref) <= FIELD_TOL


def test_solve_before_factor_is_state_error():
    wl = W.make_small(12, 12, 2, (3, 3, 4, 4), seed=2)
    s = U.make_solver(wl)
    b = torch.zeros((1, 1, wl.n), dtype=torch.complex128, device=DEV)
    with pytest.raises(FD.FdfdError) as e:
        s.solve(b)
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# Sec. III: smoothing filter and projection before the solve (NEXT-1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,box,radius,beta,eta", [(100, 100, (20, 20, 60, 60), 5.0, 8.0, 0.5),
                                                       (40, 36, (10, 9, 18, 13), 2.5, 20.0, 0.35),
                                                       (30, 30, (3, 4, 7, 5), 5.0, 4.0, 0.6)])
def test_filter_project_parity(nx, ny, box, radius, beta, eta):
    """Filtered, projected permittivity and the chain rule back to the density against the oracle
    (FP64 both sides; boxes smaller than the filter, ragged, and C1-sized)."""
    s = FD.Solver(nx, ny, 0.04, [2 * np.pi / 1.55], 3, box=box)
    w, h = box[2], box[3]
    rng = np.random.default_rng(21)
    rho = rng.uniform(0, 1, (w, h))
    g_eps = rng.normal(size=(w, h))
    eps, work = s.filter_project(torch.from_numpy(rho.reshape(-1).copy()).to(DEV), radius, beta, eta,
                                 W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    g_rho = s.filter_project_adjoint(torch.from_numpy(g_eps.reshape(-1).copy()).to(DEV), work, radius)
    torch.cuda.synchronize()
    eps_ref = O.filter_project(rho, radius, beta, eta, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    g_ref = O.filter_project_grad(rho, g_eps, radius, beta, eta, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    assert np.max(np.abs(eps.cpu().numpy().reshape(w, h) - eps_ref)) <= 1e-12 * W.DELTA_EPS
    assert O.rel_err(g_rho.cpu().numpy().reshape(w, h), g_ref) <= 1e-12


def test_filtered_design_gradient_through_autograd():
    """dF/drho of a design iteration through FilterProject and the solver Function equals the
    oracle's dF/deps pulled back through the oracle's filter and projection."""
    from paper_2307_05388_gb300 import autograd as AG
    wl = W.make_small(40, 36, 6, (10, 9, 18, 16), n_omega=2, n_src=1, seed=13)
    prob = U.problem(wl)
    radius, beta, eta = 2.5, 8.0, 0.5
    lo, hi = W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS
    rho = torch.from_numpy(wl.rho.copy()).to(DEV).requires_grad_(True)
    eps_d = AG.FilterProject.apply(rho, prob.solver, radius, beta, eta, lo, hi)
    F = prob(eps_d)
    F.backward()
    g = rho.grad.cpu().numpy()
    eps_ref = O.filter_project(wl.rho, radius, beta, eta, lo, hi)
    F_ref, g_eps_ref, _ = O.design_iteration(wl, (eps_ref - lo) / W.DELTA_EPS, wl.eps_full, W.DELTA_EPS)
    g_ref = O.filter_project_grad(wl.rho, g_eps_ref / W.DELTA_EPS, radius, beta, eta, lo, hi)
    assert abs(float(F.detach()) - F_ref) <= 1e-8 * abs(F_ref)
    assert O.rel_err(g, g_ref) <= GRAD_TOL


# ---------------------------------------------------------------------------
# Full-size configurations: a property that holds at any size
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["c2", "c3", "c4", "c5"])
def test_full_size_design_iteration_residuals(name):
    """At the full sizes (up to 3.1M unknowns per matrix, several wavelengths and sources) the
    complex128 residuals of the forward and adjoint solutions of one design iteration, measured with
    the oracle's own assembly of the operator, meet the refinement tolerance for every system."""
    wl = W.make(name)
    prob = U.problem(wl)
    s = prob.solver
    prob._load(U.eps_design_tensor(wl, wl.rho))
    x = s.solve(prob.b)
    F, o, badj = s.objective(x, prob.cols, prob.g, prob.weight)
    xa = s.solve(badj, transpose=True)
    g = s.grad(x, xa)
    torch.cuda.synchronize()
    assert np.isfinite(float(F)) and np.all(np.isfinite(g.cpu().numpy()))
    eps = wl.eps_full()
    b, ba = prob.b.cpu().numpy(), badj.cpu().numpy()
    xh, xah = x.cpu().numpy(), xa.cpu().numpy()
    tol = 2 * s.options.ir_tol
    for w, k0dx in enumerate(wl.k0dx()):
        A = O.assemble(wl.nx, wl.ny, eps, k0dx, wl.npml)
        At = A.T.tocsr()
        for j in range(wl.n_src):
            assert O.residual_rel(A, xh[w, j], b[w, j]) <= tol
            assert O.residual_rel(At, xah[w, j], ba[w, j]) <= tol
    s.close()
