"""Host logic of the autotuner (CPU only): the search, the accuracy gate, error handling, the
cache and the interface it drives.

The solver and the CUDA events are replaced by fakes that advance a virtual clock by a cost
model of the candidate's parameters; every line of the tuner runs except the default event
and synchronisation callables.  The real interface the tuner calls is checked against the
binding, so that the fakes cannot drift from it.
"""
import inspect
import json

import pytest
import torch

fd = pytest.importorskip("paper_2307_05388_gb300.fdfd")
from paper_2307_05388_gb300 import autograd as AG  # noqa: E402
from paper_2307_05388_gb300 import autotune as AT  # noqa: E402


class Clock:
    t = 0.0


class FakeEvent:
    def __init__(self, clock):
        self.clock = clock
        self.at = None

    def record(self):
        self.at = self.clock.t

    def elapsed_time(self, other):
        return other.at - self.at


class FakeSolver:
    def __init__(self, opts, model, book):
        self.options = opts
        self.nx, self.ny, self.dx, self.n_omega, self.box = 100, 100, 0.04, 1, (30, 30, 40, 40)
        self.model = model
        self.book = book
        self.fallbacks = 0
        self.closed = False

    def stats(self):
        p = {k: getattr(self.options, k) for k in AT.TUNED}
        r = self.model(p)
        return {"fallbacks": r.get("fallbacks", 0), "ir_resid": r.get("resid", 1e-10),
                "ir_iters": r.get("iters", 3), "growth": 10.0, "factor_form": r.get("form", p["factor_form"])}

    def close(self):
        self.closed = True
        self.book["closed"] += 1


class FakeProblem:
    def __init__(self, opts, model, clock, book):
        self.solver = FakeSolver(opts, model, book)
        self.b = torch.zeros(1, 2, 4, dtype=torch.complex128)
        self.clock = clock
        self.model = model
        p = {k: getattr(opts, k) for k in AT.TUNED}
        book["built"].append(p)
        r = model(p)
        if "error" in r:
            raise fd.FdfdError(3, r["error"])

    def iteration(self, eps_design, grad_out=None):
        p = {k: getattr(self.solver.options, k) for k in AT.TUNED}
        self.clock.t += self.model(p)["ms"]


def _run(model, **kw):
    clock = Clock()
    book = {"built": [], "closed": 0}
    res = AT.tune(lambda o: FakeProblem(o, model, clock, book), torch.zeros(4, dtype=torch.float64),
                  flush_bytes=0, event=lambda: FakeEvent(clock), sync=lambda: None, **kw)
    return res, book


def _model(p):
    """Milliseconds per iteration: TF32 fastest but not admissible (FP64 fallback); BF16x6 with
    m >= 256 and no split the fastest admissible; leaf 64 runs out of memory."""
    if p["leaf_area"] == 64:
        return {"error": "out of device memory"}
    ms = {3: 10.0, 2: 11.0, 1: 6.0, 0: 14.0}[p["tensor_form"]]
    out = {"ms": ms}
    if p["tensor_form"] == 1:
        out["fallbacks"] = 1
    if p["tensor_form"] in (2, 3):
        ms -= {128: 0.0, 256: 1.5, 512: 0.5}[p["tensor_min_m"]]
        ms -= 0.25 if p["tensor_min_tiles"] == 1 else 0.0
    ms += {32: 0.0, 16: 0.75}[p["leaf_area"]]
    out["ms"] = ms
    return out


def test_search_picks_fastest_admissible_and_gates_on_refinement():
    res, book = _run(_model)
    assert res.params == {"factor_form": 0, "tensor_form": 3, "tensor_offdiag": 0, "tensor_min_m": 256,
                          "tensor_min_tiles": 1, "leaf_area": 32}
    assert not res.cached
    ok = [t for t in res.trials if t.ok]
    assert min(t.ms for t in ok) == pytest.approx(10.0 - 1.5 - 0.25)
    tf32 = [t for t in res.trials if t.params["tensor_form"] == 1]
    assert tf32 and all(not t.ok and "FP64" in t.status for t in tf32)
    oom = [t for t in res.trials if t.params["leaf_area"] == 64]
    assert oom and oom[0].status.startswith("error:") and oom[0].ms is None
    # every problem built was closed again, also the one whose construction failed before it existed
    assert book["closed"] == len(book["built"]) - len(oom)
    assert res.options.tensor_min_m == 256 and res.options.tensor_min_tiles == 1
    assert res.options.mode == fd.MODE_MIXED


def test_each_candidate_measured_once_and_simt_ignores_tensor_parameters():
    res, book = _run(_model)
    keys = [tuple(sorted(p.items())) for p in book["built"]]
    assert len(keys) == len(set(keys))
    simt = [p for p in book["built"] if p["tensor_form"] == 0]
    assert len(simt) == 1 and simt[0]["tensor_min_m"] == 128 and simt[0]["tensor_min_tiles"] == 0


def test_residual_gate():
    def model(p):
        out = {"ms": 5.0 if p["tensor_form"] == 2 else 9.0}
        if p["tensor_form"] == 2:
            out["resid"] = 3e-8
        return out
    res, _ = _run(model, base=fd.default_options(ir_tol=1e-9))
    assert res.params["tensor_form"] != 2
    bad = [t for t in res.trials if t.params["tensor_form"] == 2]
    assert bad and "residual" in bad[0].status


def test_symmetric_form_taken_only_while_it_stays_symmetric():
    """The symmetric form wins when it is faster and its factors stay symmetric; a symmetric
    candidate whose growth sent it back to pivoted LU is rejected."""
    res, _ = _run(lambda p: {"ms": 4.0 if p["factor_form"] == 1 else 6.0})
    assert res.params["factor_form"] == 1 and res.options.factor_form == 1
    res, _ = _run(lambda p: {"ms": 4.0, "form": 0} if p["factor_form"] == 1 else {"ms": 6.0})
    assert res.params["factor_form"] == 0
    bad = [t for t in res.trials if t.params["factor_form"] == 1]
    assert bad and "symmetric form" in bad[0].status


def test_no_admissible_candidate_raises():
    with pytest.raises(RuntimeError, match="no admissible"):
        _run(lambda p: {"ms": 1.0, "fallbacks": 2})


def test_only_mixed_precision_is_tuned():
    with pytest.raises(ValueError):
        _run(_model, base=fd.default_options(mode=fd.MODE_F64))


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    res, book = _run(_model, cache_path=path)
    assert res.key is not None and res.key.startswith("cpu|100x100|")
    data = json.load(open(path))
    assert data[res.key]["params"] == res.params
    assert len(data[res.key]["trials"]) == len(res.trials)
    # a second run with the key reads the cache and builds nothing
    res2, book2 = _run(_model, cache_path=path, key=res.key)
    assert res2.cached and res2.params == res.params and book2["built"] == []
    assert res2.options.tensor_min_m == 256
    # another key in the same file leaves the first entry alone
    res3, _ = _run(lambda p: {"ms": 2.0}, cache_path=path, key="other")
    data = json.load(open(path))
    assert set(data) == {res.key, "other"} and data["other"]["params"] == res3.params


def test_restricted_search():
    res, book = _run(_model, search=(("tensor_form", (3, 2)),))
    assert {p["tensor_form"] for p in book["built"]} == {3, 2}
    assert all(p["leaf_area"] == 32 and p["tensor_min_m"] == 128 for p in book["built"])
    assert res.params["tensor_form"] == 3


def test_interface_the_tuner_drives_exists():
    """The fakes mirror the binding: the tuner's calls exist with these names and fields."""
    stats = {n for n, _ in fd.Stats._fields_}
    assert {"fallbacks", "ir_resid", "ir_iters", "growth"} <= stats
    opts = {n for n, _ in fd.Options._fields_}
    assert set(AT.TUNED) <= opts and {"mode", "ir_tol", "gmres_restart", "pivoting"} <= opts
    for name in ("stats", "close"):
        assert callable(getattr(fd.Solver, name))
    assert "grad_out" in inspect.signature(AG.DesignProblem.iteration).parameters
    d = fd.default_options()
    for name, values in AT.SEARCH:
        assert getattr(d, name) == values[0], name   # the search starts from the library defaults
    o = AT.with_params(d, {"tensor_form": 1, "leaf_area": 16})
    assert (o.tensor_form, o.leaf_area, o.ir_tol) == (1, 16, d.ir_tol) and d.tensor_form == 3


def test_key_from_a_real_solver_without_gpu():
    s = fd.Solver(40, 30, 0.05, [4.0, 4.1], 4, box=(10, 8, 12, 10))
    try:
        k = AT.problem_key(s, 2, device_tag="dev")
    finally:
        s.close()
    assert k == "dev|40x30|dx=0.05|omega=2|nrhs=2|box=10,8,12,10|tol=1e-09|restart=8|pivoting=1"


def test_key_before_any_solver_matches_the_solver_key():
    o = fd.default_options()
    k = AT.problem_key_for(40, 30, 0.05, 2, 2, (10, 8, 12, 10), o, device_tag="dev")
    s = fd.Solver(40, 30, 0.05, [4.0, 4.1], 4, box=(10, 8, 12, 10), options=o)
    try:
        assert AT.problem_key(s, 2, device_tag="dev") == k
    finally:
        s.close()


def test_bad_step_counts():
    with pytest.raises(ValueError):
        _run(_model, steps=0)
    with pytest.raises(ValueError):
        _run(_model, warmup=-1)


def test_tuner_drives_the_real_design_problem_class():
    """The tuner around autograd.DesignProblem (the class the bench passes it), with the oracle
    standing in for the library and a virtual clock that prefers TF32 hi+lo."""
    import numpy as np
    import workloads as W
    from tests._oracle_solver import OracleSolver
    wl = W.make_small(20, 18, 3, (6, 5, 6, 6), n_omega=1, n_src=1, seed=3)
    b = torch.from_numpy(wl.source_dense(0).reshape(1, 1, -1).copy())
    cols = torch.tensor([wl.monitors[0][0].col], dtype=torch.int32)
    g = torch.from_numpy(wl.monitors[0][0].values.astype(np.complex128).reshape(1, -1))
    eps_bg = torch.from_numpy(wl.eps_bg.reshape(-1).copy())
    clock = Clock()
    built = []

    class Timed(AG.DesignProblem):
        def iteration(self, eps_design, grad_out=None):
            clock.t += 2.0 if self.solver.options.tensor_form == 2 else 3.0
            return super().iteration(eps_design, grad_out)

    def make(opts):
        built.append(opts.tensor_form)
        s = OracleSolver(wl.nx, wl.ny, wl.dx, 2 * np.pi / np.asarray(wl.wavelengths), wl.npml, wl.box, opts)
        return Timed(s, eps_bg, b, cols, g)

    eps_d = torch.from_numpy(np.ascontiguousarray(wl.eps_design(wl.rho)).reshape(-1))
    res = AT.tune(make, eps_d, search=(("tensor_form", (3, 2)),), steps=2, warmup=1, flush_bytes=0,
                  event=lambda: FakeEvent(clock), sync=lambda: None)
    assert built == [3, 2] and res.params["tensor_form"] == 2
    assert [t.ms for t in res.trials] == [3.0, 2.0]
