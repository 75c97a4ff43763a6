#!/usr/bin/env python3
"""Benchmark: forward + adjoint FDFD design iterations per second on one GB300.

Default workload "c5": 1760 x 1760 grid (86 x 86 um + 20-cell PML at dx = 50 nm,
3,097,600 unknowns per matrix), wavelengths 1.31 and 1.55 um, TE0 and TE1 sources
(eigenmodes of the 1.2 um input guide, from the library's mode solver), 1680 x 1680
design box with an 8x8-blurred seeded density: four systems per design iteration.
One step is one design iteration: the design-box permittivity from the density (a
library kernel), design refactor of the cached factors of both wavelengths, forward
solves with FGMRES refinement, mode-overlap objective and adjoint sources, transpose
solves on the same factors, pixel gradient.  The sign-step update of rho between
steps is not timed; the L2 is flushed between steps.

Beside the headline (cached complex FP32 factors + FP64 FGMRES refinement):
  e2e          the same design path through fdfd_design_iteration with host buffers
               (the host -> device copy of the design and the device -> host copy of
               F and the gradient inside the timed region)
  uncached_f64 the paper's reference procedure on the same GPU (symbolic and numeric
               FP64 factorisation for every solve), and the cached FP64 form
  factor       full factorisation against design refactor: time, flops, factor memory
  cpu_baseline the CPU oracle (SciPy SuperLU, nested-dissection order, complex128) on
               the same workload: one design iteration at the initial design, one
               process per wavelength, started before the first GPU call; its fields
               and gradient also give the accuracy of the GPU path element by element.
Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(N > 1 via torch.distributed.run: the (wavelength, source) pairs of the one problem
are sharded over the ranks, one all-reduce of [gradient, F] per iteration).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "fwd+adjoint design iterations/s, cached vs uncached FP64, at field err <=1e-8"
UNIT = "iterations/s"
L2_FLUSH_BYTES = 512 << 20
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM = 2       # FP64 FMAs per SM per clock on this part (ncu dfma peak_sustained)
# DRAM bytes (read + write) of one sweep launch over its algorithmic bytes, from the ncu capture of
# a C4 one-wavelength L sweep (profiles/flow_sweep_c4_one_wavelength.md: 927.9 + 99.3 MB against
# 559.8 MB of L11^-1 and L21 entries); a full launch's traffic is scaled from it by its algorithmic bytes
SWEEP_TRAFFIC_RATIO = (927.9 + 99.3) / 559.8
DATA = "synthetic (seeded design density and guide; the paper's devices are not published)"
DTYPE = "c64 factors + c128 refinement"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, src="fallback")


TENSOR_FORMS = {0: "SIMT complex FP32", 1: "tcgen05 TF32", 2: "tcgen05 TF32 hi+lo (3 products)",
                3: "tcgen05 BF16 three-way split (6 products), FP32 register sum every 8 pivots"}


def workload_config(wl):
    x0, y0, w, h = wl.box
    srcs = ("TE0/TE1 eigenmodes of the input guide" if any(isinstance(s, W.ModeLine) for s in wl.sources)
            else "Gaussian line source")
    return {"workload": f"{wl.name}: {wl.nx}x{wl.ny} grid ({wl.n:,} unknowns), dx {wl.dx * 1e3:.0f} nm, "
                        f"{wl.n_omega} wavelength(s) x {wl.n_src} source(s), {w}x{h} design box",
            "nx": wl.nx, "ny": wl.ny, "n_omega": wl.n_omega, "nrhs": wl.n_src, "design_box": [x0, y0, w, h],
            "wavelengths_um": [float(v) for v in wl.wavelengths], "sources": srcs,
            "factor": "complex FP32 multifrontal + FP64 FGMRES refinement (tol 1e-9)",
            "l2": "flushed between timed steps (512 MB write)"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        rows = []
        for line in open(self.f.name).read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle: the cpu_baseline leg and the reference arm (one process per wavelength)
# ---------------------------------------------------------------------------
def _oracle_wavelength(name: str, w: int, seed: int, want_fields: bool):
    """One wavelength's share of an oracle design iteration at the initial design (runs in a
    spawned child).  Returns (seconds, F_w, dF/drho_w [w, h], {s: (E, E_adj)} or None)."""
    from oracle import fdfd_oracle as O
    wl = W.with_modes(W.make(name, seed=seed), O.slab_modes).select_wavelengths([w])
    t = time.perf_counter()
    F, g, fields = O.design_iteration(wl, wl.rho, wl.eps_full, W.DELTA_EPS)
    dt = time.perf_counter() - t
    return dt, F, g, ({s: fields[(0, s)] for s in range(wl.n_src)} if want_fields else None)


class OracleLeg:
    """The oracle's design iteration of a workload, its wavelengths in parallel spawned processes
    (each process gets an equal share of the host cores for its BLAS threads)."""

    def __init__(self, name: str, n_omega: int, want_fields: bool, seed: int = 0):
        import concurrent.futures as cf
        import multiprocessing as mp
        # the host cores split over the processes, read by each child's BLAS at start-up
        threads = str(max(1, (os.cpu_count() or 1) // n_omega))
        os.environ["OPENBLAS_NUM_THREADS"] = threads
        os.environ["OMP_NUM_THREADS"] = threads
        self.ex = cf.ProcessPoolExecutor(max_workers=n_omega, mp_context=mp.get_context("spawn"))
        self.t0 = time.perf_counter()
        self.jobs = [self.ex.submit(_oracle_wavelength, name, w, seed, want_fields) for w in range(n_omega)]
        self.n = n_omega

    def result(self, budget_s: float):
        """[(seconds, F_w, g_w, fields_w)] per wavelength, or None if the budget ran out."""
        import concurrent.futures as cf
        left = max(1.0, budget_s - (time.perf_counter() - self.t0))
        done, pending = cf.wait(self.jobs, timeout=left)
        if pending:
            self.kill()
            return None
        return [j.result() for j in self.jobs]

    def kill(self):
        for p in list(getattr(self.ex, "_processes", {}).values()):
            try:
                p.kill()
            except Exception:
                pass
        self.ex.shutdown(wait=False, cancel_futures=True)


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (a job's time is its slowest rank's); value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def oracle_sample(name: str, budget_s: float):
    """Times full oracle design iterations of workload `name` at its initial design until the
    budget is spent (at least one), one process per wavelength: (seconds per iteration, count)."""
    n_w = W.make(name, seed=0).n_omega
    times = []
    t_start = time.perf_counter()
    while True:
        leg = OracleLeg(name, n_w, False)
        res = leg.result(max(budget_s, 60.0))
        leg.ex.shutdown(wait=True)
        if res is None:
            break
        times.append(max(r[0] for r in res))
        if time.perf_counter() - t_start + times[-1] > budget_s:
            break
    return (float(np.mean(times)) if times else None), len(times), n_w


def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only): each step one full design
    iteration of the sample workload at its initial design, one process per wavelength."""
    if rank != 0:
        return 0
    name = args.cpu_sample
    wl = W.make(name, seed=0)
    n_w = wl.n_omega
    times = []
    t_start = time.perf_counter()
    for k in range(args.steps):
        per, n, _ = oracle_sample(name, 0.0)
        if per is None:
            break
        times.append(per)
        if time.perf_counter() - t_start + per > args.cpu_budget:
            break
    if not times:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"one oracle design iteration of {name} did not finish within {args.cpu_budget:.0f} s"}))
        return 0
    per = float(np.mean(times))
    value = 1.0 / per
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(times),
            "steps_requested": args.steps, "warmup": 0, "ms_per_step": 1e3 * per, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "c128", "data": DATA,
            "config": workload_config(wl), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{len(times)} full design iteration(s) of the {name} workload at its initial "
                                       f"design (SciPy SuperLU complex128, nested-dissection order, one process per "
                                       f"wavelength sharing the host cores); {name} is the sample because an oracle "
                                       f"iteration of the largest workload takes tens of minutes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--cpu-sample", default="c2",
                    help="workload of the bounded CPU-oracle sample (cpu_baseline and the reference arm)")
    ap.add_argument("--cpu-budget", type=float, default=150.0,
                    help="seconds of oracle iterations the CPU sample and the reference arm aim for")
    ap.add_argument("--cpu-accuracy", action="store_true",
                    help="also run the oracle on the benchmarked workload itself (one iteration, one process per "
                         "wavelength, started before the GPU work) for the element-wise accuracy of the GPU path; "
                         "at the largest sizes this takes tens of minutes")
    ap.add_argument("--no-plain", action="store_true", help="skip the uncached and cached FP64 arms")
    ap.add_argument("--omegas", type=int, default=0,
                    help="run only the first N wavelengths of the workload (0 = all; for small profiling cases)")
    ap.add_argument("--tensor-form", type=int, default=3, choices=[0, 1, 2, 3],
                    help="update matrices on the tensor cores: 0 off (SIMT), 1 TF32, 2 TF32 hi+lo, "
                         "3 BF16 three-way split (default)")
    ap.add_argument("--factor-form", type=int, default=0, choices=[0, 1],
                    help="complex FP32 factors: 0 LU with block-local pivoting (default), 1 symmetric "
                         "L diag(d) L^T of D A without pivoting")
    ap.add_argument("--pivoting", type=int, default=1, choices=[0, 1],
                    help="LU pivot search: 1 within 32 x 32 diagonal blocks (default), 0 partial pivoting over "
                         "all pivot rows of a front")
    ap.add_argument("--offdiag-tc", type=int, default=0, choices=[0, 1],
                    help="L21 and U12 of tensor-core fronts as products with the triangular inverses on the "
                         "tensor cores (1) or by substitution in the panel steps (0, default)")
    ap.add_argument("--gmres-restart", type=int, default=0,
                    help="Krylov vectors per FGMRES cycle (0: the library default, 8)")
    ap.add_argument("--rhs-pairs", type=int, default=0, choices=[0, 1],
                    help="sweeps take a wavelength's right-hand sides two at a time (1) or one at a time (0, default)")
    ap.add_argument("--optimizer", default="workload", choices=["workload", "sign", "adam"],
                    help="the design update between iterations (not timed): the workload's own (default; "
                         "Adam at lr 0.01 for c4, a sign step for the others), or the one named")
    ap.add_argument("--autotune", default="", metavar="CACHE.json",
                    help="choose tensor_form, tensor_min_m, tensor_min_tiles and leaf_area by measured design "
                         "iterations before the timed run (starting from --tensor-form), cached in this file")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    wl0 = W.make(args.workload, seed=0)
    n_omega_run = args.omegas if 0 < args.omegas < wl0.n_omega else wl0.n_omega
    # the oracle leg starts first: spawned children, before any CUDA call in this process
    leg = None
    if (args.impl == "ours" and rank == 0 and world == 1 and args.cpu_accuracy and not args.no_cpu
            and n_omega_run == wl0.n_omega):
        leg = OracleLeg(args.workload, wl0.n_omega, True)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2307_05388_gb300 import autograd as AG
    from paper_2307_05388_gb300 import fdfd as FD
    from paper_2307_05388_gb300 import optimize as OPT
    from paper_2307_05388_gb300 import shard as SH

    wl = W.with_modes(wl0, FD.slab_modes)
    if n_omega_run < wl.n_omega:   # a smaller case of the same workload (profiling)
        wl = wl.select_wavelengths(range(n_omega_run))
    x0, y0, bw, bh = wl.box
    nd = bw * bh
    optimizer = wl.optimizer if args.optimizer == "workload" else args.optimizer
    k0 = 2 * np.pi / np.asarray(wl.wavelengths)
    eps_bg = torch.from_numpy(wl.eps_bg.reshape(-1).copy()).to(dev)
    lo, hi = W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS

    def make_problem(ws, ss, opts):
        s = FD.Solver(wl.nx, wl.ny, wl.dx, k0[ws], wl.npml, box=wl.box, options=opts)
        b = np.stack([np.stack([wl.source_dense(i, w) for i in ss]) for w in ws])
        cols = np.array([wl.monitors[w][i].col for w in ws for i in ss], np.int32)
        g = np.stack([wl.monitors[w][i].values for w in ws for i in ss]).astype(np.complex128)
        return AG.DesignProblem(s, eps_bg, torch.from_numpy(b).to(dev), torch.from_numpy(cols).to(dev),
                                torch.from_numpy(g).to(dev))

    def build(opts):
        return SH.ShardedProblem(lambda ws, ss: make_problem(ws, ss, opts), wl.n_omega, wl.n_src, nd, dev,
                                 group=dist.group.WORLD if dist is not None else None)

    def close(sp):
        for p in sp.problems:
            p.solver.close()

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rho0 = torch.from_numpy(wl.rho.reshape(-1).copy()).to(dev)

    def density(sp, rho, out):
        if sp.problems:
            sp.problems[0].solver.density_eps(rho, lo, hi, out=out)    # library kernel
        else:
            out.copy_(lo + rho * (hi - lo))                           # a rank with no systems

    def run_arm(sp, steps, warmup, clocks=False):
        rho = rho0.clone()
        upd = OPT.design_optimizer(optimizer, wl.step)      # state on the device
        eps = torch.empty(nd, dtype=torch.float64, device=dev)
        grad = torch.empty(nd, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            density(sp, rho, eps)
            F, g = sp.iteration(eps, grad_out=grad)
            rho = upd.step(rho, g)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        for k in range(steps):
            flush.zero_()                                # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            density(sp, rho, eps)
            F, g = sp.iteration(eps, grad_out=grad)
            ev[k][1].record(stream)
            rho = upd.step(rho, g)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        run_arm.step_ms = [a.elapsed_time(b) for a, b in ev]
        return sum(run_arm.step_ms), clk

    def run_e2e(sp, steps, warmup):
        """Host design in, host F and gradient out, every step; host wall clock."""
        h_eps = torch.empty(nd, dtype=torch.float64, pin_memory=True)
        h_F = torch.empty(1, dtype=torch.float64, pin_memory=True)
        h_g = torch.empty(nd, dtype=torch.float64, pin_memory=True)
        d_eps = torch.empty(nd, dtype=torch.float64, device=dev)
        rho = torch.from_numpy(wl.rho.reshape(-1).copy())
        upd = OPT.design_optimizer(optimizer, wl.step)      # the caller's host-side loop
        single = dist is None and len(sp.problems) == 1
        total = 0.0
        for k in range(warmup + steps):
            h_eps.numpy()[:] = lo + rho.numpy() * (hi - lo)   # the caller's host-side design (not timed)
            flush.zero_()
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t = time.perf_counter()
            if single:
                p = sp.problems[0]
                p.solver.design_iteration(h_eps, p.b, p.cols, p.g, F_out=h_F, grad_out=h_g)
            else:
                d_eps.copy_(h_eps, non_blocking=True)
                F, g = sp.iteration(d_eps)
                h_g.copy_(g, non_blocking=True)
                h_F.copy_(F.reshape(1), non_blocking=True)
                torch.cuda.current_stream().synchronize()
            dt = time.perf_counter() - t
            if k >= warmup:
                total += dt
            rho = upd.step(rho, h_g)
        return 1e3 * total

    # ---- launch parameters: library defaults, or measured by the autotuner (not timed) ----
    opts = FD.default_options(mode=FD.MODE_MIXED, tensor_form=args.tensor_form, factor_form=args.factor_form,
                              sweep_rhs_pairs=args.rhs_pairs, pivoting=args.pivoting,
                              tensor_offdiag=args.offdiag_tc)
    if args.gmres_restart > 0:
        opts.gmres_restart = args.gmres_restart
    tuned = None
    if args.autotune:
        from paper_2307_05388_gb300 import autotune as AT
        key = AT.problem_key_for(wl.nx, wl.ny, wl.dx, wl.n_omega, wl.n_src, wl.box, opts)
        t_tune = time.perf_counter()
        res = AT.tune(lambda o: make_problem(list(range(wl.n_omega)), list(range(wl.n_src)), o),
                      (lo + rho0 * (hi - lo)), base=opts, cache_path=args.autotune, key=key)
        opts = res.options
        tuned = {"params": res.params, "cached": res.cached, "candidates": len(res.trials),
                 "seconds": time.perf_counter() - t_tune}
    form = opts.tensor_form

    # ---- cached mixed-precision arm (the headline) --------------------------
    sp = build(opts)
    t_setup = time.perf_counter()
    eps0 = torch.empty(nd, dtype=torch.float64, device=dev)
    density(sp, rho0, eps0)
    sp.iteration(eps0)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    ms, clk = run_arm(sp, args.steps, args.warmup, clocks=True)
    step_ms = sorted(run_arm.step_ms)
    step_pct = {"p50": float(np.percentile(step_ms, 50)), "p90": float(np.percentile(step_ms, 90)),
                "min": step_ms[0], "max": step_ms[-1]}
    ms_max = max_over_ranks(ms, dist, dev)
    value = args.steps / (ms_max / 1e3)
    stats = [p.solver.stats() for p in sp.problems]

    # ---- end to end through the public API with host buffers -----------------
    ms_e2e = run_e2e(sp, args.steps, args.warmup)
    e2e_value = args.steps / (max_over_ranks(ms_e2e, dist, dev) / 1e3)

    # ---- per-kernel profile (separate pass; events around every launch) -----
    prof_steps = 2
    for p in sp.problems:
        p.solver.profile(True)
    run_arm(sp, prof_steps, 0)
    kern = {}
    for p in sp.problems:
        for k, v in p.solver.profile_get().items():
            if v["launches"] > 0:
                a = kern.setdefault(k, dict(launches=0, ms=0.0, flops=0.0, bytes=0.0))
                for f in a:
                    a[f] += v[f]
        p.solver.profile(False)
    pk = peaks()
    roof = roof_tc = roof_sw = None
    kernels = {}
    launches_per_step = 0.0
    if kern:
        tot_ms = sum(v["ms"] for v in kern.values())
        # the four sweep directions are one kernel (flow_kernel, one template instance per direction)
        classes = {k: v for k, v in kern.items() if not k.startswith("sweep_")}
        sweeps = [v for k, v in kern.items() if k.startswith("sweep_")]
        if sweeps:
            classes["flow_kernel"] = {f: sum(v[f] for v in sweeps) for f in ("launches", "ms", "flops", "bytes")}
        dom = max(classes, key=lambda k: classes[k]["ms"])
        d = classes[dom]
        per_launch_ms = d["ms"] / d["launches"]
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = nsm * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        fp64_peak = nsm * FP64_FMA_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        if dom == "flow_kernel":
            per_launch_bytes = d["bytes"] / d["launches"]
            roof = {"bound": "hbm", "achieved": per_launch_bytes / (per_launch_ms / 1e3) / 1e9,
                    "peak": pk["hbm"], "unit": "GB/s",
                    "traffic": per_launch_bytes * SWEEP_TRAFFIC_RATIO,
                    "traffic_unit": "bytes per launch",
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a C4 one-wavelength L "
                                      "sweep (1.027 GB against 0.560 GB algorithmic), scaled to this launch by its "
                                      "algorithmic bytes",
                    "algorithmic_bytes_per_launch": per_launch_bytes,
                    "peak_source": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        elif dom.startswith("gmres_"):
            roof = {"bound": "alu", "achieved": d["flops"] / d["launches"] / (per_launch_ms / 1e3) / 1e12,
                    "peak": fp64_peak, "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"FP64 FMA: {nsm} SMs x {FP64_FMA_PER_SM} x 2 x {pk['sm_max_mhz']:.0f} MHz"}
        elif dom == "lu_schur_tc":
            mult = {1: 1, 2: 3, 3: 6}[form]
            peak_tc = pk["bf16_sus"] * (1.0 if form == 3 else 0.5)
            ach = d["flops"] / d["launches"] / (per_launch_ms / 1e3) / 1e12 * mult
            roof = {"bound": "tensor", "achieved": ach, "peak": peak_tc, "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"{pk['src']} sustained bf16 dense GEMM (MEASURED_PEAKS.json)"}
        elif dom.startswith("lu_"):
            roof = {"bound": "alu", "achieved": d["flops"] / d["launches"] / (per_launch_ms / 1e3) / 1e12,
                    "peak": fp32_peak, "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"FP32 SIMT: {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {pk['sm_max_mhz']:.0f} MHz"}
        else:
            roof = {"bound": "hbm", "achieved": d["bytes"] / d["launches"] / (per_launch_ms / 1e3) / 1e9,
                    "peak": pk["hbm"], "unit": "GB/s", "traffic": None,
                    "peak_source": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        roof["kernel"] = dom
        roof["launches_per_step"] = d["launches"] / prof_steps
        roof["frac"] = roof["achieved"] / roof["peak"]
        sw = [v for k, v in kern.items() if k.startswith("sweep_")]
        if sw:
            sw_ms = sum(v["ms"] for v in sw)
            sw_gbs = sum(v["bytes"] for v in sw) / (sw_ms / 1e3) / 1e9
            sw_tf = sum(v["flops"] for v in sw) / (sw_ms / 1e3) / 1e12
            roof_sw = {"kernels": "flow_kernel (L, U, U^T, L^T)", "bound": "hbm", "achieved": sw_gbs, "unit": "GB/s",
                       "peak": pk["hbm"], "frac": sw_gbs / pk["hbm"], "ms_per_step": sw_ms / prof_steps,
                       "alu_tflops": sw_tf, "alu_frac": sw_tf / fp32_peak,
                       "peak_source": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs); alu_frac "
                                      "against the FP32 SIMT peak"}
        if "lu_schur_tc" in kern:
            d_tc = kern["lu_schur_tc"]
            mult = {1: 1, 2: 3, 3: 6}[form]
            peak_tc = pk["bf16_sus"] * (1.0 if form == 3 else 0.5)
            ach = d_tc["flops"] / (d_tc["ms"] / 1e3) / 1e12
            roof_tc = {"kernel": "lu_schur_tc", "bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
                       "tensor_op_tflops": ach * mult, "peak": peak_tc, "frac": ach * mult / peak_tc,
                       "peak_source": f"{pk['src']} sustained bf16 dense GEMM peak" + ("" if form == 3 else " x 0.5 (TF32)"),
                       "note": f"achieved counts 8 flops per complex multiply-add; the operand form issues {mult}x "
                               "as many tensor flops (tile padding not counted)"}
        fac_keys = [k for k in kern if k.startswith("lu_") or k == "front_build"]
        fac_ms = sum(kern[k]["ms"] for k in fac_keys) / prof_steps
        fac_fl = sum(kern[k]["flops"] for k in fac_keys) / prof_steps
        tc_fl = sum(kern[k]["flops"] for k in ("lu_schur_tc", "lu_trsm_tc") if k in kern) / prof_steps
        roof_fac = {"kernels": "the whole design refactor (" + ", ".join(sorted(fac_keys)) + ")",
                    "tensor_core_flop_share": tc_fl / fac_fl if fac_fl else None,
                    "achieved": fac_fl / (fac_ms / 1e3) / 1e12 if fac_ms else None, "unit": "TFLOP/s",
                    "ms_per_step": fac_ms, "peak_tf32_tensor": pk["bf16_sus"] * 0.5,
                    "frac_of_tf32_tensor": (fac_fl / (fac_ms / 1e3) / 1e12) / (pk["bf16_sus"] * 0.5) if fac_ms else None,
                    "peak_source": f"{pk['src']} sustained bf16 dense GEMM x 0.5"}
        launches_per_step = sum(v["launches"] for v in kern.values()) / prof_steps
        kernels = {k: {"launches_per_step": v["launches"] / prof_steps, "ms_per_step": v["ms"] / prof_steps,
                       "share": v["ms"] / tot_ms,
                       "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["flops"] else None,
                       "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["bytes"] else None}
                   for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"])}
        kernels["_factorisation"] = roof_fac

    # ---- full factorisation against design refactor, factor memory (N = 1) ---
    factor = None
    if dist is None and len(sp.problems) == 1:
        p = sp.problems[0]
        eps_full = eps_bg.clone().reshape(wl.nx, wl.ny)
        eps_full[x0:x0 + bw, y0:y0 + bh] = eps0.reshape(bw, bh)
        eps_full = eps_full.reshape(-1).contiguous()
        times = {"full": [], "design": []}
        for rep in range(3):
            for kind in ("full", "design"):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if kind == "full":
                    p.solver.factor(eps_full)
                else:
                    p.solver.refactor_design(eps0)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    times[kind].append(e0.elapsed_time(e1))
        st0 = stats[0]
        factor = {"full_factor_ms": float(np.mean(times["full"])), "design_refactor_ms": float(np.mean(times["design"])),
                  "refactor_time_fraction": float(np.mean(times["design"]) / np.mean(times["full"])),
                  "full_factor_gflop": st0["flops_factor"] * wl.n_omega / 1e9,
                  "design_refactor_gflop": st0["flops_design"] * wl.n_omega / 1e9,
                  "refactor_flop_fraction": st0["flops_design"] / st0["flops_factor"],
                  "factor_memory_gb": st0["store_bytes"] / 1e9,
                  "factor_entries_per_wavelength": st0["factor_entries"],
                  "note": "factor memory: the complex64 fronts of all wavelengths (L, U and the retained "
                          "update matrices that make the design refactor possible)"}

    # ---- accuracy of the measured path: GPU fields at the initial design -----
    fields_gpu = None
    if leg is not None:
        p = sp.problems[0]
        F0_t, g0_t = p.iteration(eps0)
        torch.cuda.synchronize()
        F0, g0 = float(F0_t), g0_t.cpu().numpy()
        fields_gpu = (p.x.cpu().numpy(), p.xa.cpu().numpy())
        p.solver.set_options(ir_max_iter=0)
        x_raw = p.solver.solve(p.b).cpu().numpy()
        p.solver.set_options(ir_max_iter=opts.ir_max_iter)

    # ---- uncached FP64 arm (paper's reference procedure, on the same GPU) -----
    plain = None
    if not args.no_plain:
        psp = build(FD.default_options(mode=FD.MODE_PLAIN))
        for pp in psp.problems:
            pp.solver.reset_counters()
        pms, _ = run_arm(psp, 1, 0)
        pst = [pp.solver.stats() for pp in psp.problems]
        plain = {"value": 1 / (max_over_ranks(pms, dist, dev) / 1e3), "unit": UNIT, "ms_per_step": pms,
                 "what": "every solve re-runs the symbolic phase and a full complex128 multifrontal "
                         "factorisation (no refinement), forward and adjoint (one timed iteration)",
                 "sf_nf_bs_per_step": [sum(s["sf"] for s in pst), sum(s["nf"] for s in pst),
                                       sum(s["bs"] for s in pst)]}
        close(psp)
        del psp
        fsp = build(FD.default_options(mode=FD.MODE_F64))
        fsp.iteration(eps0)
        torch.cuda.synchronize()
        fms, _ = run_arm(fsp, 2, 0)
        plain["cached_f64"] = {"value": 2 / (max_over_ranks(fms, dist, dev) / 1e3), "unit": UNIT,
                               "ms_per_step": fms / 2,
                               "what": "cached complex128 factors (design refactor), no refinement"}
        plain["speedup_of_headline"] = value / plain["value"]
        close(fsp)
        del fsp

    # ---- the CPU oracle: a bounded sample (cpu_baseline); accuracy when asked for ----
    cpu = None
    acc = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        per, n_it, n_w = oracle_sample(args.cpu_sample, args.cpu_budget)
        if per is not None:
            cpu = {"value": 1.0 / per, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "workload": args.cpu_sample,
                   "sample": f"{n_it} full design iteration(s) of the {args.cpu_sample} workload at its initial "
                             f"design ({per:.1f} s each; SciPy SuperLU complex128 with a nested-dissection order, "
                             f"{n_w} process(es), one per wavelength, sharing the host cores); the benchmarked "
                             f"workload's own oracle iteration takes tens of minutes, so a smaller workload of the "
                             f"same family is the bounded sample"}
    if leg is not None:
        res = leg.result(args.cpu_budget if args.cpu_budget > 600 else 3600.0)
        if res is not None:
            leg.ex.shutdown(wait=True)
            wall = max(r[0] for r in res)
            from oracle import fdfd_oracle as O
            F_ref = sum(r[1] for r in res)
            g_ref = sum(r[2] for r in res).reshape(-1)
            xf, xa = fields_gpu
            fe, ae, re_ = [], [], []
            for w, r in enumerate(res):
                for s_, (E, Ea) in r[3].items():
                    fe.append(O.rel_err(xf[w, s_], E))
                    ae.append(O.rel_err(xa[w, s_], Ea))
                    re_.append(O.rel_err(x_raw[w, s_], E))
            acc = {"field_err_max": max(fe), "adjoint_field_err_max": max(ae),
                   "grad_err": O.rel_err(g0 * W.DELTA_EPS, g_ref), "objective_err": abs(F0 - F_ref) / abs(F_ref),
                   "raw_fp32_factor_field_err_max": max(re_), "oracle_iteration_s": wall,
                   "what": "relative 2-norm errors against the oracle over all unknowns (PML included), every "
                           "wavelength and source, at the initial design; gates 1e-8 (fields) and 1e-6 (gradient)"}

    if not acc and stats:
        acc = {"refinement_residual_max": max(s["ir_resid"] for s in stats),
               "what": "the largest FP64 relative residual |b - A x| / |b| at the end of the last refined solve "
                       "(tolerance 1e-9); element-wise parity with the oracle at C1-C4 sizes is in the -m gpu tests, "
                       "and --cpu-accuracy adds it here for the benchmarked workload"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "step_ms_this_rank": step_pct,
            "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": DTYPE, "data": DATA,
            "config": dict(workload_config(wl), update_matrices=TENSOR_FORMS[form],
                           parallelism=("one GPU" if world == 1 else
                                        f"(wavelength, source) pairs sharded over {world} ranks, "
                                        "all-reduce of [dF/deps, F] per iteration"),
                           factor_form=("symmetric L diag(d) L^T of D A, no pivoting" if opts.factor_form == 1
                                        else "LU of A, pivoting within 32 x 32 diagonal blocks" if opts.pivoting == 1
                                        else "LU of A, partial pivoting over each front's pivot rows"),
                           design_update=(f"Adam, lr {wl.step}, ascent, clipped to [0, 1]" if optimizer == "adam"
                                          else f"sign step {wl.step}, clipped to [0, 1]") + " (not timed)",
                           launch_parameters={"tensor_min_m": opts.tensor_min_m,
                                              "tensor_min_tiles": opts.tensor_min_tiles,
                                              "leaf_area": opts.leaf_area, "autotuned": tuned}),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nd,
                    "d2h_bytes_per_step": 8 * (nd + 1),
                    "what": "fdfd_design_iteration with host design in and host F and gradient out, host wall clock"},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roof, "roofline_tensor": roof_tc, "roofline_sweeps": roof_sw,
            "accuracy": acc, "uncached_f64": plain, "cpu_baseline": cpu, "factor": factor,
            "solves_per_s": value * 2 * wl.n_omega * wl.n_src,
            "solver": {"ir_iters_last_solve": max(s["ir_iters"] for s in stats) if stats else None,
                       "ir_resid": max(s["ir_resid"] for s in stats) if stats else None,
                       "n_fronts": stats[0]["n_fronts"] if stats else None,
                       "n_levels": stats[0]["n_levels"] if stats else None,
                       "max_front": stats[0]["max_front"] if stats else None,
                       "growth_last": max(s["growth"] for s in stats) if stats else None,
                       "repivots_fp32": sum(s["repivots"] for s in stats),
                       "fallbacks_fp64": sum(s["fallbacks"] for s in stats),
                       "first_iteration_s": t_setup},
            "kernels": kernels}
    if rank == 0:
        print(json.dumps(line), flush=True)
    close(sp)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
