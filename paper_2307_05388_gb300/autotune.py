"""Autotuner for the factorisation's launch parameters (host side, above the C ABI).

The kernels' tile shapes are fixed by their design: 128 x 128 output tiles fed
8 pivots at a time on the tensor cores, 32-pivot panel steps, and fronts of up
to 64 unknowns factored whole in shared memory.  What depends on the problem
and the device is which fronts take which path, and how a level's contraction
is spread over the SMs.  The tuner picks these per problem:

* ``tensor_form``: the operand form of the tensor-core update matrices
  S = F22 - L21 U12 (3 = BF16 three-way split, 2 = TF32 hi + lo, 1 = TF32), or
  0 = SIMT FP32.  The cheaper forms are accepted only where refinement still
  converges on the FP32 factors.
* ``tensor_offdiag``: whether the tensor-core fronts also form L21 and U12 on
  the tensor cores, as products with the triangular inverses (1), or by
  substitution in their panel steps (0).  Faster factors, but the inverses'
  conditioning can cost FGMRES iterations, which the timed iterations include.
* ``tensor_min_m``: the smallest front boundary size m sent to the tensor
  cores.  This is the front-size bucket boundary between SIMT and tensor-core
  update matrices.
* ``tensor_min_tiles``: the split rule, either one wave of CTAs (0) or never
  split the contraction (1).
* ``leaf_area``: the nested-dissection leaf size.  It sets how many small
  fronts there are, and how large the separators above them get.
* ``factor_form``: LU of A with block-local pivoting (0), or the symmetric form
  L diag(d) L^T of D A without pivoting (1: half the update work; admitted only
  where its pivot growth stays inside the bound, which the accuracy gate below
  checks through the absence of fallbacks).

Each candidate is measured the way a design iteration runs.  A solver is built
with the candidate's options and gets a full factorisation, followed by timed
design iterations: refactor of the design fronts, refined forward solves,
objective and adjoint source, refined transpose solves, gradient.  These are
timed with CUDA events on the current stream, with the L2 flushed between them.

Accuracy gates admission.  A candidate is admissible only if its FP32 factors
carried every solve to the refinement tolerance: the solver never refactored
in FP64, and the last solve's relative residual is within ``ir_tol``.

The search is coordinate-wise, starting from the defaults.  Each parameter's
values are tried in turn with the best choice so far for the others, and the
fastest admissible candidate wins.  Results can be cached in a JSON file keyed
by the device and the problem's shape, so a later run skips the measurement.
"""
from __future__ import annotations

import dataclasses
import json
import os
import tempfile
from typing import Callable

import torch

from . import fdfd

#: (option, values) in search order; the first value of each is the library default.
SEARCH = (
    ("factor_form", (0, 1)),
    ("tensor_form", (3, 2, 1, 0)),
    ("tensor_offdiag", (0, 1)),
    ("tensor_min_m", (128, 256, 512)),
    ("tensor_min_tiles", (0, 1)),
    ("leaf_area", (32, 16, 64)),
)
TUNED = tuple(name for name, _ in SEARCH)
L2_FLUSH_BYTES = 512 << 20


@dataclasses.dataclass
class Trial:
    params: dict
    ms: float | None          # mean milliseconds per timed design iteration (None if not measured)
    status: str               # "ok", or why the candidate was rejected
    ir_iters: int = 0         # FGMRES iterations of the last solve
    growth: float = 0.0       # largest |L| entry of the last FP32 factorisation

    @property
    def ok(self) -> bool:
        return self.status == "ok"


@dataclasses.dataclass
class TuneResult:
    options: fdfd.Options     # base options with the chosen parameters
    params: dict              # the chosen values of TUNED
    trials: list              # every candidate measured (empty when read from the cache)
    cached: bool
    key: str | None


def options_dict(o: fdfd.Options) -> dict:
    return {name: getattr(o, name) for name, _ in o._fields_}


def with_params(base: fdfd.Options, params: dict) -> fdfd.Options:
    o = fdfd.Options()
    for name, value in options_dict(base).items():
        setattr(o, name, value)
    for name, value in params.items():
        setattr(o, name, value)
    return o


def problem_key(solver, nrhs: int, device_tag: str | None = None) -> str:
    """Cache key of a built solver (see ``problem_key_for``)."""
    return problem_key_for(solver.nx, solver.ny, solver.dx, solver.n_omega, nrhs, solver.box, solver.options,
                           device_tag)


def problem_key_for(nx: int, ny: int, dx: float, n_omega: int, nrhs: int, box, options: fdfd.Options,
                    device_tag: str | None = None) -> str:
    """Cache key: device, grid, spacing, wavelengths, sources, design box and the solve options
    that change the work of a design iteration."""
    if device_tag is None:
        device_tag = device_name()
    x0, y0, w, h = (int(v) for v in box)
    return (f"{device_tag}|{nx}x{ny}|dx={dx:.6g}|omega={n_omega}|nrhs={nrhs}"
            f"|box={x0},{y0},{w},{h}|tol={options.ir_tol:.3g}|restart={options.gmres_restart}"
            f"|pivoting={options.pivoting}")


def device_name() -> str:
    if not torch.cuda.is_available():
        return "cpu"
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


def _normalise(params: dict, base: dict) -> dict:
    """Without tensor-core update matrices the tensor parameters do nothing: map them to the base
    values so that such candidates are measured once."""
    p = dict(params)
    if p["tensor_form"] == 0:
        p["tensor_min_m"] = base["tensor_min_m"]
        p["tensor_min_tiles"] = base["tensor_min_tiles"]
        p["tensor_offdiag"] = base["tensor_offdiag"]
    return p


def _cuda_event():
    return torch.cuda.Event(enable_timing=True)


def measure(prob, eps_design: torch.Tensor, steps: int, warmup: int, flush: torch.Tensor | None,
            event: Callable = _cuda_event, sync: Callable = torch.cuda.synchronize) -> float:
    """Mean milliseconds per design iteration of ``prob`` (its first iteration factors fully and
    is part of the warm-up)."""
    for _ in range(max(1, warmup)):
        prob.iteration(eps_design)
    sync()
    evs = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = event(), event()
        a.record()
        prob.iteration(eps_design)
        b.record()
        evs.append((a, b))
    sync()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def _admission(stats: dict, ir_tol: float, params: dict | None = None) -> str:
    if stats["fallbacks"] > 0:
        return f"FP64 refactorisation ({stats['fallbacks']}): the FP32 factors did not carry refinement"
    if params and params.get("factor_form") == 1 and stats.get("factor_form", 1) != 1:
        return "the symmetric form exceeded the growth bound and fell back to pivoted LU"
    if not stats["ir_resid"] <= ir_tol:
        return f"residual {stats['ir_resid']:.3g} above ir_tol {ir_tol:.3g}"
    return "ok"


def _load_cache(path: str) -> dict:
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _store_cache(path: str, key: str, base: dict, params: dict, trials: list):
    data = _load_cache(path)
    data[key] = {"params": params,
                 "base": {k: base[k] for k in ("mode", "ir_tol", "ir_max_iter", "gmres_restart", "pivoting")},
                 "trials": [{"params": t.params, "ms": t.ms, "status": t.status, "ir_iters": t.ir_iters}
                            for t in trials]}
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".autotune", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def tune(make_problem: Callable[[fdfd.Options], object], eps_design: torch.Tensor,
         base: fdfd.Options | None = None, search=SEARCH, steps: int = 3, warmup: int = 2,
         cache_path: str | None = None, key: str | None = None, flush_bytes: int = L2_FLUSH_BYTES,
         event: Callable = _cuda_event, sync: Callable = torch.cuda.synchronize,
         log: Callable[[str], None] | None = None) -> TuneResult:
    """Chooses factor_form, tensor_form, tensor_offdiag, tensor_min_m, tensor_min_tiles and leaf_area
    for one design problem.

    make_problem(options) builds a fresh problem with those options: an object with
    ``iteration(eps_design)`` and a ``solver`` (an ``fdfd.Solver``), e.g. an
    ``autograd.DesignProblem``.  The tuner closes each problem's solver after measuring it.
    eps_design: the design-box permittivity every timed iteration uses.
    base: options that stay fixed (mode must be mixed precision); default the library's.
    search: (option, values) pairs, searched in order.
    cache_path, key: a JSON cache; with both given and the key present, nothing is measured
    (``problem_key_for`` makes a key before any solver exists).  Without a key, the result is
    stored under the key of the first problem built (``problem_key``).
    Raises RuntimeError if no candidate is admissible.
    """
    if steps < 1 or warmup < 0:
        raise ValueError("steps must be >= 1 and warmup >= 0")
    base = base if base is not None else fdfd.default_options()
    if base.mode != fdfd.MODE_MIXED:
        raise ValueError("the tuner chooses parameters of the mixed-precision path (mode 0)")
    base_d = options_dict(base)
    if cache_path and key:
        hit = _load_cache(cache_path).get(key)
        if hit is not None:
            return TuneResult(with_params(base, hit["params"]), dict(hit["params"]), [], True, key)

    flush = None
    if flush_bytes > 0:
        flush = torch.empty(flush_bytes, dtype=torch.uint8, device=eps_design.device)
    say = log or (lambda s: None)
    trials: dict[tuple, Trial] = {}

    def run(params: dict) -> Trial:
        nonlocal key
        params = _normalise(params, base_d)
        tk = tuple(sorted(params.items()))
        if tk in trials:
            return trials[tk]
        opts = with_params(base, params)
        prob = None
        try:
            prob = make_problem(opts)
            if key is None:
                key = problem_key(prob.solver, prob.b.shape[1] if hasattr(prob, "b") else 1)
            ms = measure(prob, eps_design, steps, warmup, flush, event, sync)
            st = prob.solver.stats()
            status = _admission(st, opts.ir_tol, params)
            t = Trial(params, ms, status, int(st["ir_iters"]), float(st["growth"]))
        except RuntimeError as e:
            t = Trial(params, None, f"error: {e}")
        finally:
            if prob is not None:
                prob.solver.close()
            del prob
        trials[tk] = t
        say(f"autotune {params}: {t.status}" + (f", {t.ms:.3f} ms" if t.ms is not None else ""))
        return t

    def best() -> Trial | None:
        ok = [t for t in trials.values() if t.ok]
        return min(ok, key=lambda t: t.ms) if ok else None

    cur = {name: base_d[name] for name in TUNED}
    run(cur)
    for name, values in search:
        for v in values:
            run(dict(cur, **{name: v}))
        b = best()
        if b is not None:
            cur = dict(b.params)
    b = best()
    if b is None:
        reasons = "; ".join(f"{t.params}: {t.status}" for t in trials.values())
        raise RuntimeError(f"autotune: no admissible candidate ({reasons})")
    out = list(trials.values())
    if cache_path and key:
        _store_cache(cache_path, key, base_d, b.params, out)
    return TuneResult(with_params(base, b.params), dict(b.params), out, False, key)
