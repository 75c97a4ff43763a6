"""The L-BFGS-B host loop on the CPU, with an objective whose optimum under the box bounds is
known in closed form (the GPU objective chain it drives is covered by the parity tests), and the
per-step sign and Adam updates against the oracle's."""
import numpy as np
import pytest
import torch

pytest.importorskip("scipy")
from paper_2307_05388_gb300 import optimize as OPT  # noqa: E402


def test_lbfgsb_maximises_under_the_box_bounds():
    """F = -sum (rho - c)^2 with c partly outside [0, 1]: the maximiser is clip(c, 0, 1)."""
    rng = np.random.default_rng(0)
    c = torch.from_numpy(rng.uniform(-0.5, 1.5, (6, 5)))
    calls = []

    def obj(rho):
        calls.append(rho.shape)
        return -((rho - c) ** 2).sum(), -2 * (rho - c)

    rho, F, res = OPT.lbfgsb(obj, torch.full((6, 5), 0.5, dtype=torch.float64), maxiter=50)
    assert rho.shape == (6, 5) and rho.dtype == torch.float64
    np.testing.assert_allclose(rho.numpy(), np.clip(c.numpy(), 0, 1), atol=1e-6)
    assert F == pytest.approx(-float(((np.clip(c.numpy(), 0, 1) - c.numpy()) ** 2).sum()), abs=1e-9)
    assert all(s == (6, 5) for s in calls)


def test_lbfgsb_minimise_and_callback():
    c = torch.linspace(0.1, 0.9, 8, dtype=torch.float64)
    seen = []
    rho, F, _ = OPT.lbfgsb(lambda r: (((r - c) ** 2).sum(), 2 * (r - c)), torch.zeros(8, dtype=torch.float64),
                           maximize=False, callback=lambda k, f, x: seen.append(f))
    np.testing.assert_allclose(rho.numpy(), c.numpy(), atol=1e-6)
    assert F == pytest.approx(0.0, abs=1e-10) and seen and seen[-1] <= seen[0]


def _oracle_problem():
    import workloads as W
    from paper_2307_05388_gb300 import autograd as AG
    from tests._oracle_solver import OracleSolver
    wl = W.make_small(26, 22, 4, (8, 6, 8, 7), n_omega=2, n_src=1, seed=41)
    s = OracleSolver(wl.nx, wl.ny, wl.dx, 2 * np.pi / np.asarray(wl.wavelengths), wl.npml, wl.box)
    b = np.stack([wl.source_dense(i) for i in range(wl.n_src)])
    b = np.broadcast_to(b, (wl.n_omega,) + b.shape).copy()
    cols = np.array([wl.monitors[w][i].col for w in range(wl.n_omega) for i in range(wl.n_src)], np.int32)
    g = np.stack([wl.monitors[w][i].values for w in range(wl.n_omega) for i in range(wl.n_src)])
    prob = AG.DesignProblem(s, torch.from_numpy(wl.eps_bg.reshape(-1).copy()), torch.from_numpy(b),
                            torch.from_numpy(cols), torch.from_numpy(g.astype(np.complex128)))
    return wl, prob


def test_density_objective_gradient_matches_central_differences():
    """The chain filter -> projection -> solver Function -> objective, through both autograd
    Functions, with the oracle standing in for the library (host plumbing only)."""
    import workloads as W
    wl, prob = _oracle_problem()
    f = OPT.density_objective(prob, 1.5, 4.0, 0.5, W.EPS_SIO2, W.EPS_SI)
    rho = torch.from_numpy(wl.rho.reshape(-1).copy())
    F, g = f(rho)
    assert g.shape == rho.shape and float(F) > 0
    h = 1e-6
    for p in (0, 17, 55):
        e = torch.zeros_like(rho)
        e[p] = h
        Fp, _ = f(rho + e)
        Fm, _ = f(rho - e)
        fd = (float(Fp) - float(Fm)) / (2 * h)
        assert abs(float(g[p]) - fd) <= 1e-5 * max(abs(fd), 1e-3 * float(g.abs().max()))


def test_lbfgsb_on_the_design_objective_ascends():
    import workloads as W
    wl, prob = _oracle_problem()
    f = OPT.density_objective(prob, 1.5, 4.0, 0.5, W.EPS_SIO2, W.EPS_SI)
    rho0 = torch.from_numpy(wl.rho.reshape(-1).copy())
    F0, _ = f(rho0)
    rho, F, res = OPT.lbfgsb(f, rho0, maxiter=6)
    assert F > float(F0) and float(rho.min()) >= 0.0 and float(rho.max()) <= 1.0


# ---------------------------------------------------------------------------
# The per-step updates of the workloads' loops (SignStep, Adam), against the oracle's
# sign_step and adam_step, which tests/test_oracle.py pins by closed forms.
# ---------------------------------------------------------------------------
def _gradients(n, steps, seed):
    rng = np.random.default_rng(seed)
    # magnitudes from 1e-12 to 1e2, zeros included: Adam's eps and sign(0) both matter
    out = []
    for _ in range(steps):
        g = rng.standard_normal(n) * 10.0 ** rng.uniform(-12, 2, n)
        g[rng.integers(0, n, 3)] = 0.0
        out.append(g)
    return out


def test_adam_matches_the_oracle_over_a_trajectory():
    from oracle import fdfd_oracle as O
    rho = np.random.default_rng(1).uniform(0, 1, 64)
    st, opt = {}, OPT.Adam(0.01)
    r = torch.from_numpy(rho.copy())
    for g in _gradients(64, 12, 2):
        rho = O.adam_step(rho, g, st, lr=0.01)
        r = opt.step(r, torch.from_numpy(g))
        np.testing.assert_allclose(r.numpy(), rho, rtol=0, atol=1e-15)
    assert opt.t == 12 and r.min() >= 0 and r.max() <= 1


def test_adam_minimise_descends_and_state_round_trips():
    """Minimising mirrors maximising with the gradient negated; a loop resumed from state_dict
    continues exactly where an unbroken one goes."""
    gs = [torch.from_numpy(g) for g in _gradients(32, 6, 3)]
    rho0 = torch.full((32,), 0.5, dtype=torch.float64)
    up, down = OPT.Adam(0.02), OPT.Adam(0.02, maximize=False)
    a, b = rho0, rho0
    for g in gs:
        a, b = up.step(a, g), down.step(b, -g)
    torch.testing.assert_close(a, b, rtol=0, atol=0)
    whole, first = OPT.Adam(0.02), OPT.Adam(0.02)
    w, f = rho0, rho0
    for g in gs[:3]:
        w, f = whole.step(w, g), first.step(f, g)
    resumed = OPT.Adam(0.02)
    resumed.load_state_dict(first.state_dict())
    for g in gs[3:]:
        w, f = whole.step(w, g), resumed.step(f, g)
    torch.testing.assert_close(w, f, rtol=0, atol=0)


def test_sign_step_matches_the_oracle():
    from oracle import fdfd_oracle as O
    rho = np.random.default_rng(4).uniform(0, 1, 64)
    opt = OPT.design_optimizer("sign", 0.05)
    for g in _gradients(64, 5, 5):
        ref = O.sign_step(rho, g, 0.05)
        np.testing.assert_array_equal(opt.step(torch.from_numpy(rho), torch.from_numpy(g)).numpy(), ref)
        rho = ref
    assert isinstance(OPT.design_optimizer("adam", 0.01), OPT.Adam)
    with pytest.raises(ValueError):
        OPT.design_optimizer("sgd", 0.1)


# ---------------------------------------------------------------------------
# The checkpointed design loop (DesignLoop), with the oracle standing in for the library
# ---------------------------------------------------------------------------
def test_design_loop_resumes_on_the_same_trajectory(tmp_path):
    """Five Adam iterations without a break against three with a checkpoint every two, then a
    resume (a new problem, its factors from scratch) and three more: the same densities and the
    same F history, bit for bit (the stand-in solver is deterministic); the log shows every
    iteration, those since the last checkpoint twice."""
    import json
    import workloads as W
    wl, prob = _oracle_problem()
    rho0 = torch.from_numpy(wl.rho.reshape(-1).copy())
    f = OPT.linear_density_objective(prob, W.EPS_SIO2, W.EPS_SI)
    whole = OPT.DesignLoop(f, OPT.Adam(0.05), rho0)
    whole.run(5)
    ck, log = str(tmp_path / "loop.pt"), str(tmp_path / "loop.jsonl")
    first = OPT.DesignLoop(f, OPT.Adam(0.05), rho0, checkpoint=ck, every=2, log=log, stats=prob.solver.stats)
    first.run(3)
    assert first.iteration == 3 and not (tmp_path / "loop.pt.tmp").exists()
    wl2, prob2 = _oracle_problem()
    f2 = OPT.linear_density_objective(prob2, W.EPS_SIO2, W.EPS_SI)
    resumed = OPT.DesignLoop.resume(ck, f2, OPT.Adam(0.05), checkpoint=ck, every=2, log=log,
                                    stats=prob2.solver.stats)
    assert resumed.iteration == 2 and resumed.optimizer.t == 2 and len(resumed.history) == 2
    resumed.run(3)
    torch.testing.assert_close(resumed.rho, whole.rho, rtol=0, atol=0)
    assert resumed.history == whole.history
    recs = [json.loads(line) for line in open(log)]
    assert [r["iteration"] for r in recs] == [0, 1, 2, 2, 3, 4]
    assert [r["F"] for r in recs[3:]] == whole.history[2:]
    assert all({"F", "grad_norm", "seconds", "ir_iters", "growth", "fallbacks"} <= set(r) for r in recs)
    assert torch.load(ck)["iteration"] == 4


def test_linear_density_objective_chain_rule():
    """dF/drho of the unfiltered map is (eps_hi - eps_lo) dF/deps: against central differences of
    the stand-in's F."""
    import workloads as W
    wl, prob = _oracle_problem()
    f = OPT.linear_density_objective(prob, W.EPS_SIO2, W.EPS_SI)
    rho = torch.from_numpy(wl.rho.reshape(-1).copy())
    F, g = f(rho)
    h = 1e-6
    for p in (3, 29):
        e = torch.zeros_like(rho)
        e[p] = h
        fd = (float(f(rho + e)[0]) - float(f(rho - e)[0])) / (2 * h)
        assert abs(float(g[p]) - fd) <= 1e-5 * max(abs(fd), 1e-3 * float(g.abs().max()))


def test_design_loop_rejects_a_zero_interval():
    with pytest.raises(ValueError):
        OPT.DesignLoop(lambda r: (r.sum(), r), OPT.SignStep(0.1), torch.zeros(3, dtype=torch.float64), every=0)


# ---------------------------------------------------------------------------
# The seeded workload recipe at test size (the GPU loop tests run C4's recipe at 200^2)
# ---------------------------------------------------------------------------
def test_workload_recipe_at_a_smaller_grid():
    """make(name, grid=, design=) keeps the workload's recipe (dx, PML, wavelengths, sources,
    optimiser) on a smaller centred box, and refuses a design that does not fit."""
    import workloads as W
    full, small = W.make("c4"), W.make("c4", grid=200, design=150)
    assert (small.nx, small.ny, small.box) == (200, 200, (25, 25, 150, 150))
    assert small.dx == full.dx and small.npml == full.npml and small.optimizer == full.optimizer == "adam"
    np.testing.assert_array_equal(small.wavelengths, full.wavelengths)
    assert small.rho.shape == (150, 150) and 0 <= small.rho.min() and small.rho.max() <= 1
    assert small.eps_bg.shape == (200, 200) and small.name == "c4@200"
    c3 = W.make("c3", grid=240, design=180)
    assert len(c3.monitors) == 8 and len({m[0].values.argmax() for m in c3.monitors}) == 4
    with pytest.raises(ValueError):
        W.make("c2", grid=100, design=90)
