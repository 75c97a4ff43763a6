#!/usr/bin/env python3
"""Benchmark: forward + adjoint FDFD design iterations per second on one GB300.

Workload (default "c2"): 340 x 340 grid (12 x 12 um + 20-cell PML at dx = 40 nm,
115,600 unknowns), lambda = 1.55 um, 250 x 250 design box with 8x8-blurred
seeded density and Si waveguide stubs, one source.  One step is one design
iteration: design refactor of the cached factors, forward solve with FGMRES
refinement, mode-overlap objective and adjoint source, transpose solve on the
same factors, pixel gradient.  The sign-step update of rho between steps is
not timed.  The uncached FP64 arm (symbolic + numeric factorisation per solve,
as in the paper's reference arm) and the CPU oracle are reported beside it.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(N > 1 via torch.distributed.run: each rank runs its own seeded replica).
"""
from __future__ import annotations

import argparse
import json
import math
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
N_SM = 152


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], sm_max_mhz=d.get("sm_max_mhz", 2070.0), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, sm_max_mhz=2070.0, src="fallback")


TENSOR_FORMS = {0: "SIMT complex FP32", 1: "tcgen05 TF32", 2: "tcgen05 TF32 hi+lo (3 products)",
                3: "tcgen05 BF16 three-way split (6 products), FP32 register sum every 8 pivots"}


def workload_config(wl):
    x0, y0, w, h = wl.box
    return {"workload": f"{wl.name}: {wl.nx}x{wl.ny} grid ({wl.n:,} unknowns), dx {wl.dx * 1e3:.0f} nm, "
                        f"{wl.n_omega} wavelength(s) x {wl.n_src} source(s), {w}x{h} design box",
            "nx": wl.nx, "ny": wl.ny, "n_omega": wl.n_omega, "nrhs": wl.n_src, "design_box": [x0, y0, w, h],
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
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_iteration(wl, rho):
    from oracle import fdfd_oracle as O
    t = time.perf_counter()
    F, g, fields = O.design_iteration(wl, rho, wl.eps_full, W.DELTA_EPS)
    return time.perf_counter() - t, F, g, fields


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (a job's time is its slowest rank's); value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = W.make(args.workload, seed=0)
    budget_s = 150.0
    rho = wl.rho.copy()
    t_first, F, g, _ = oracle_iteration(wl, rho)   # warm-up / sizing step
    times = []
    from oracle import fdfd_oracle as O
    for k in range(max(0, args.warmup - 1)):
        if t_first * (k + 2) > budget_s / 3:
            break
        rho = O.sign_step(rho, g, wl.step)
        _, F, g, _ = oracle_iteration(wl, rho)
    steps = max(1, min(args.steps, int(budget_s / max(t_first, 1e-3))))
    for _ in range(steps):
        rho = O.sign_step(rho, g, wl.step)
        dt, F, g, _ = oracle_iteration(wl, rho)
        times.append(dt)
    total = sum(times)
    value = len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "steps_timed": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded design density; the paper's devices are not published)",
            "config": workload_config(wl), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} full design iterations (SciPy SuperLU complex128, "
                                       "single-threaded) of the same workload"},
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
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the uncached FP64 arm")
    ap.add_argument("--omegas", type=int, default=0,
                    help="run only the first N wavelengths of the workload (0 = all; for small profiling cases)")
    ap.add_argument("--tensor-form", type=int, default=3, choices=[0, 1, 2, 3],
                    help="update matrices on the tensor cores: 0 off (SIMT), 1 TF32, 2 TF32 hi+lo, "
                         "3 BF16 three-way split (default)")
    ap.add_argument("--autotune", default="", metavar="CACHE.json",
                    help="choose tensor_form, tensor_min_m, tensor_min_tiles and leaf_area by measured design "
                         "iterations before the timed run (starting from --tensor-form), cached in this file")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

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

    wl = W.make(args.workload, seed=rank)
    if 0 < args.omegas < wl.n_omega:   # a smaller case of the same workload (profiling)
        wl.wavelengths = wl.wavelengths[:args.omegas]
        wl.monitors = wl.monitors[:args.omegas]
    x0, y0, bw, bh = wl.box
    k0 = 2 * np.pi / wl.wavelengths

    def make_problem(mode, opts=None):
        s = FD.Solver(wl.nx, wl.ny, wl.dx, k0, wl.npml, box=wl.box,
                      options=opts if opts is not None else FD.default_options(mode=mode, tensor_form=args.tensor_form))
        b = np.stack([wl.source_dense(i) for i in range(wl.n_src)])
        b = np.broadcast_to(b, (wl.n_omega,) + b.shape).copy()
        cols = np.array([wl.monitors[w][i].col for w in range(wl.n_omega) for i in range(wl.n_src)], np.int32)
        g = np.stack([wl.monitors[w][i].values for w in range(wl.n_omega) for i in range(wl.n_src)])
        return AG.DesignProblem(s, torch.from_numpy(wl.eps_bg.reshape(-1).copy()).to(dev),
                                torch.from_numpy(b).to(dev), torch.from_numpy(cols).to(dev),
                                torch.from_numpy(g.astype(np.complex128)).to(dev))

    def eps_of(rho_t):
        return (W.EPS_SIO2 + rho_t * W.DELTA_EPS).reshape(-1).contiguous()

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rho0 = torch.from_numpy(wl.rho.copy()).to(dev)

    def run_arm(prob, steps, warmup, clocks=False, host_io=False):
        rho = rho0.clone()
        grad = torch.empty(bw * bh, dtype=torch.float64, device=dev)
        h_eps = torch.empty(bw * bh, dtype=torch.float64, pin_memory=True)
        h_out = torch.empty(bw * bh + 1, dtype=torch.float64, pin_memory=True)
        d_eps = torch.empty(bw * bh, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            F, g = prob.iteration(eps_of(rho), grad_out=grad)
            rho = torch.clamp(rho + wl.step * torch.sign(g.reshape(bw, bh)), 0.0, 1.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        for k in range(steps):
            flush.zero_()                                # L2 flush between timed steps (not timed)
            if host_io:
                h_eps.copy_(eps_of(rho).cpu())           # the caller's host-side design (not timed)
            ev[k][0].record(stream)
            if host_io:
                d_eps.copy_(h_eps, non_blocking=True)
                F, g = prob.iteration(d_eps, grad_out=grad)
                h_out[:bw * bh].copy_(g, non_blocking=True)
                h_out[bw * bh:].copy_(F.reshape(1), non_blocking=True)
            else:
                F, g = prob.iteration(eps_of(rho), grad_out=grad)
            ev[k][1].record(stream)
            rho = torch.clamp(rho + wl.step * torch.sign(g.reshape(bw, bh)), 0.0, 1.0)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        ms = sum(a.elapsed_time(b) for a, b in ev)
        return ms, clk

    # ---- launch parameters: library defaults, or measured by the autotuner (not timed) ----
    opts = FD.default_options(mode=FD.MODE_MIXED, tensor_form=args.tensor_form)
    tuned = None
    if args.autotune:
        from paper_2307_05388_gb300 import autotune as AT
        key = AT.problem_key_for(wl.nx, wl.ny, wl.dx, wl.n_omega, wl.n_src, wl.box, opts)
        t_tune = time.perf_counter()
        res = AT.tune(lambda o: make_problem(FD.MODE_MIXED, o), eps_of(rho0), base=opts,
                      cache_path=args.autotune, key=key)
        opts = res.options
        tuned = {"params": res.params, "cached": res.cached, "candidates": len(res.trials),
                 "seconds": time.perf_counter() - t_tune}
    form = opts.tensor_form

    # ---- cached mixed-precision arm (the headline) --------------------------
    prob = make_problem(FD.MODE_MIXED, opts)
    t_setup = time.perf_counter()
    prob.iteration(eps_of(rho0))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    ms, clk = run_arm(prob, args.steps, args.warmup, clocks=True)
    ms_max = max_over_ranks(ms, dist, dev)
    value = world * args.steps / (ms_max / 1e3)
    st = prob.solver.stats()

    # ---- accuracy of the measured path against the oracle (rank 0, N = 1) ----
    acc = {}
    cpu = None
    run_cpu = (rank == 0 and world == 1 and not args.no_cpu)
    if run_cpu:
        F, g = prob.iteration(eps_of(rho0))
        torch.cuda.synchronize()
        x_gpu = prob.x.cpu().numpy().reshape(-1)
        dt, F_ref, g_ref, fields = oracle_iteration(wl, wl.rho.copy())
        from oracle import fdfd_oracle as O
        acc = {"field_err": O.rel_err(x_gpu, fields[(0, 0)][0]),
               "grad_err": O.rel_err(g.cpu().numpy().reshape(bw, bh) * W.DELTA_EPS, g_ref),
               "objective_err": abs(float(F) - F_ref) / abs(F_ref)}
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "1 full design iteration at the initial design (SciPy SuperLU complex128 factor, "
                         f"forward + transpose solve, gradient; single-threaded), {dt:.1f} s"}

    # ---- end to end through the public API with host buffers -----------------
    ms_e2e, _ = run_arm(prob, args.steps, args.warmup, host_io=True)   # the same design path as the timed arm
    e2e_value = world * args.steps / (max_over_ranks(ms_e2e, dist, dev) / 1e3)

    # ---- per-kernel profile (separate pass; events around every launch) -----
    prof_steps = 3
    prob.solver.profile(True)
    run_arm(prob, prof_steps, 0)
    prof = prob.solver.profile_get()
    prob.solver.profile(False)
    kern = {k: v for k, v in prof.items() if v["launches"] > 0}
    tot_ms = sum(v["ms"] for v in kern.values())
    dom = max(kern, key=lambda k: kern[k]["ms"])
    pk = peaks()
    d = kern[dom]
    per_launch_ms = d["ms"] / d["launches"]
    if dom.startswith("lu_"):
        fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": d["flops"] / d["launches"] / (per_launch_ms / 1e3) / 1e12,
                "peak": fp32_peak, "unit": "TFLOP/s", "traffic": None,
                "peak_source": f"FP32 SIMT: {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {pk['sm_max_mhz']:.0f} MHz"}
    else:
        roof = {"bound": "hbm", "achieved": d["bytes"] / d["launches"] / (per_launch_ms / 1e3) / 1e9,
                "peak": pk["hbm"], "unit": "GB/s", "traffic": None,
                "peak_source": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    roof["kernel"] = dom
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the tensor-core update matrices: algorithmic rate (8 flops per complex multiply-add) and the
    # tensor-op rate it takes in the chosen operand form, against the dense peak of that input type
    # the cached solves: the four sweep directions together, algorithmic bytes (every factor entry
    # of the swept triangle and off-diagonal block once per right-hand side) against the HBM peak
    sw = [v for k, v in kern.items() if k.startswith("sweep_")]
    roof_sw = None
    if sw:
        sw_ms = sum(v["ms"] for v in sw)
        sw_gbs = sum(v["bytes"] for v in sw) / (sw_ms / 1e3) / 1e9
        roof_sw = {"kernels": "flow_kernel (L, U, U^T, L^T)", "bound": "hbm", "achieved": sw_gbs, "unit": "GB/s",
                   "peak": pk["hbm"], "frac": sw_gbs / pk["hbm"], "ms_per_step": sw_ms / prof_steps,
                   "peak_source": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    roof_tc = None
    if "lu_schur_tc" in kern:
        d_tc = kern["lu_schur_tc"]
        mult = {1: 1, 2: 3, 3: 6}[form]
        peak_tc = pk["bf16"] * (1.0 if form == 3 else 0.5)
        ach = d_tc["flops"] / (d_tc["ms"] / 1e3) / 1e12
        roof_tc = {"kernel": "lu_schur_tc", "bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
                   "tensor_op_tflops": ach * mult, "peak": peak_tc, "frac": ach * mult / peak_tc, "traffic": None,
                   "peak_source": f"{pk['src']} bf16 dense GEMM peak" + ("" if form == 3 else " x 0.5 (TF32)"),
                   "note": f"achieved counts 8 flops per complex multiply-add; the operand form issues {mult}x "
                           "as many tensor flops (tile padding not counted)"}
    launches_per_step = sum(v["launches"] for v in kern.values()) / prof_steps
    kernels = {k: {"launches_per_step": v["launches"] / prof_steps, "ms_per_step": v["ms"] / prof_steps,
                   "share": v["ms"] / tot_ms,
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["flops"] else None,
                   "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["bytes"] else None}
               for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"])}

    # ---- smoothing filter + projection of the design density (Sec. III), C2 box ----
    radius_cells = 0.2 / wl.dx                       # the paper's 200 nm filter radius
    rho_f = rho0.reshape(-1).contiguous()
    eps_f, work_f = prob.solver.filter_project(rho_f, radius_cells, 8.0, 0.5, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    g_f = prob.solver.filter_project_adjoint(eps_f, work_f, radius_cells)
    reps = 50
    torch.cuda.synchronize()
    ef = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ef[0].record(stream)
    for _ in range(reps):
        prob.solver.filter_project(rho_f, radius_cells, 8.0, 0.5, W.EPS_SIO2, W.EPS_SIO2 + W.DELTA_EPS)
    ef[1].record(stream)
    for _ in range(reps):
        prob.solver.filter_project_adjoint(eps_f, work_f, radius_cells)
    ef[2].record(stream)
    torch.cuda.synchronize()
    rc = int(np.ceil(radius_cells))
    taps = sum(1 for i in range(-rc, rc + 1) for j in range(-rc, rc + 1) if np.hypot(i, j) < radius_cells)
    design_filter = {"what": "conic filter (200 nm radius) + tanh projection of the design density and its "
                             "chain rule, on the design box (FP64, one thread per pixel)",
                     "pixels": bw * bh, "taps": taps,
                     "us_forward": ef[0].elapsed_time(ef[1]) * 1e3 / reps,
                     "us_adjoint": ef[1].elapsed_time(ef[2]) * 1e3 / reps}
    del g_f

    # ---- uncached FP64 arm (paper's reference procedure, on the same GPU) -----
    plain = None
    if not args.no_plain:
        pprob = make_problem(FD.MODE_PLAIN)
        pprob.iteration(eps_of(rho0))
        torch.cuda.synchronize()
        pms, _ = run_arm(pprob, 2, 0)
        pst = pprob.solver.stats()
        plain = {"value": 2 / (pms / 1e3), "unit": UNIT, "ms_per_step": pms / 2,
                 "what": "every solve re-runs the symbolic phase and a full complex128 multifrontal "
                         "factorisation (no refinement), forward and adjoint",
                 "sf_nf_bs_per_step": [pst["sf"] / 3, pst["nf"] / 3, pst["bs"] / 3]}
        fprob = make_problem(FD.MODE_F64)
        fprob.iteration(eps_of(rho0))
        torch.cuda.synchronize()
        fms, _ = run_arm(fprob, 3, 1)
        plain["cached_f64"] = {"value": 3 / (fms / 1e3), "unit": UNIT, "ms_per_step": fms / 3}
        del pprob, fprob

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic (seeded design density; the paper's devices are not published)",
            "config": dict(workload_config(wl), update_matrices=TENSOR_FORMS[form],
                           launch_parameters={"tensor_min_m": opts.tensor_min_m,
                                              "tensor_min_tiles": opts.tensor_min_tiles,
                                              "leaf_area": opts.leaf_area, "autotuned": tuned}),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * bw * bh,
                    "d2h_bytes_per_step": 8 * (bw * bh + 1)},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roof, "roofline_tensor": roof_tc, "roofline_sweeps": roof_sw,
            "solves_per_s": value * 2 * wl.n_omega * wl.n_src, "cpu_baseline": cpu, "accuracy": acc, "uncached_f64": plain,
            "design_filter": design_filter,
            "solver": {"ir_iters_last_solve": st["ir_iters"], "ir_resid": st["ir_resid"],
                       "n_fronts": st["n_fronts"], "n_levels": st["n_levels"], "max_front": st["max_front"],
                       "factor_gflop": st["flops_factor"] / 1e9, "refactor_gflop": st["flops_design"] / 1e9,
                       "growth_last": st["growth"], "repivots_fp32": st["repivots"], "fallbacks_fp64": st["fallbacks"],
                       "store_mb": st["store_bytes"] / 1e6, "first_iteration_s": t_setup},
            "kernels": kernels}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
