#!/usr/bin/env python
"""Benchmark: FGMRES time to a 1e-8 relative residual and V-cycle HBM GB/s.

Workload (default): the one-group 3-component system on a 1024x1024 grid with
a 10^4 coefficient jump across a circular inclusion (3.1M unknowns, 15.7M
nonzeros, seeded synthetic coefficients), preconditioned by Schur1 with one
classical-AMG V(1,1) cycle per subsystem inverse (PMIS coarsening with
extended+i interpolation), FP64.  One step = the whole
hot path on that system: device setup (block extraction, strength, PMIS,
interpolation, Galerkin products, smoother diagonals, coarsest inverse) plus
the FGMRES(30) solve to ||b - A x|| <= 1e-8 ||b||.  Inputs are resident in HBM
before the timed region; the operator (201 MB) is larger than L2, so no flush
is needed between steps.

--impl reference times the FP64 CPU oracle on the same workload (host cores),
the deliberately slow program the GPU path is checked against.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = 1
KIND = "schur1"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier():
    """Barrier over the ranks of an initialised process group (no-op alone)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _max_over_ranks(v, device):
    """The largest of the ranks' values (each replica's step time; the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return v
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None
        self.enabled = enabled

    def start(self):
        if not self.enabled:
            return
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2002_04958_gb300 import inputs
    from paper_2002_04958_gb300 import mgdamg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2002_04958_gb300.build import build
    build()

    sysm = inputs.preset(args.config)
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(sysm.rowptr).to(dev)
    ci = torch.from_numpy(sysm.col).to(dev)
    va = torch.from_numpy(sysm.val).to(dev)
    b = torch.from_numpy(sysm.b).to(dev)
    ncyc = [int(t) for t in args.nvcyc.split(",")]
    opts = dict(precision=args.precision, batched=args.batched, use_graph=args.graph, autotune=1,
                keep_transpose=int(args.adjoint), max_it=args.max_it, interp_type=args.interp, pdl=args.pdl,
                inner_mode=args.inner, nvcyc_group=ncyc[0], nvcyc_E=ncyc[1], nvcyc_I=ncyc[2],
                smoother=args.smoother, agg_levels=args.agg)
    slv = mgdamg.Solver(**opts)
    adj = {}

    def step():
        slv.setup(sysm.G, sysm.N, rp, ci, va, args.kind)
        x, it, rr, rc = slv.solve(b, tol=args.tol)
        if args.adjoint:   # L = ||x||^2: lambda = A^-T (2x), dL/dvals = -lambda_row x_col
            lam, ita, rra = slv.solve_transpose(2.0 * x, tol=args.tol)
            g = slv.grad_values(x, lam)
            adj.update(iters_transpose=ita, relres_transpose=rra)
        return x, it, rr

    for _ in range(args.warmup):
        x, it, rr = step()
    torch.cuda.synchronize()

    barrier = _barrier

    clocks = ClockSampler(local, enabled=not args.no_clocks)
    # the dominant level-0 kernels are bracketed by CUDA events during the first
    # timed step only: event nodes between kernels cost a few percent of a step
    slv.profile(1)
    l0 = mgdamg.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    setup_ms, solve_ms, iters = [], [], []
    for k in range(args.steps):
        x, it, rr = step()
        st = slv.stats()
        setup_ms.append(st["setup_ms"])
        solve_ms.append(st["solve_ms"])
        iters.append(it)
        if k == 0:
            n0, t0, by0 = slv.profile_read(0)    # level-0 smoothing + residual kernels (dominant)
            f0 = slv.profile_read_fp64(0)        # their algorithmic FP64 lane operations
            slv.profile(0)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = mgdamg.kernel_launches() - l0
    ms = _max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    # V-cycle GB/s over every V-cycle kernel: one more (untimed) step with all V-cycle classes bracketed
    slv.profile(0b11)
    step()
    vcycles = slv.total_cycles()   # V-cycles of one solve (counted since its setup)
    n1, t1, by1 = slv.profile_read(1)
    slv.profile(0)
    # preconditioner bandwidth: 100 applies back to back (graph replays), no per-kernel events
    pms, pby = slv.precond_bench(b, 100)
    st = slv.stats()
    xg = x
    relres = rr

    # end to end through the C ABI with host buffers (pinned), copies timed
    h_rp = torch.from_numpy(sysm.rowptr).pin_memory()
    h_ci = torch.from_numpy(sysm.col).pin_memory()
    h_va = torch.from_numpy(sysm.val).pin_memory()
    h_b = torch.from_numpy(sysm.b).pin_memory()
    h_x = torch.zeros(sysm.n, dtype=torch.float64).pin_memory()
    d_rp, d_ci, d_va = torch.empty_like(rp), torch.empty_like(ci), torch.empty_like(va)
    # the adjoint step also returns the value gradient: x goes back to the
    # device for the transposed solve, the gradient comes to the host
    d_x = torch.empty(sysm.n, dtype=torch.float64, device=dev) if args.adjoint else None
    h_g = torch.empty(sysm.nnz, dtype=torch.float64).pin_memory() if args.adjoint else None
    e2e_ms = []
    for k in range(0 if args.no_e2e else max(2, args.steps // 2) + 1):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        d_rp.copy_(h_rp, non_blocking=True)
        d_ci.copy_(h_ci, non_blocking=True)
        d_va.copy_(h_va, non_blocking=True)
        slv.setup(sysm.G, sysm.N, d_rp, d_ci, d_va, args.kind)
        h_x.zero_()
        slv.solve_host_ptr(h_b.data_ptr(), h_x.data_ptr(), tol=args.tol)
        if args.adjoint:
            d_x.copy_(h_x, non_blocking=True)
            lam_e, _, _ = slv.solve_transpose(2.0 * d_x, tol=args.tol)
            h_g.copy_(slv.grad_values(d_x, lam_e), non_blocking=True)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append((time.perf_counter() - t_a) * 1e3)
    h2d = sysm.rowptr.nbytes + sysm.col.nbytes + sysm.val.nbytes + sysm.b.nbytes + sysm.n * 8
    d2h = sysm.n * 8
    if args.adjoint:
        h2d += sysm.n * 8
        d2h += sysm.nnz * 8

    # variants for context (one solve each, outside the timed region)
    variants = {}
    if not args.no_variants:
        for name, kind, o in [("monolithic_amg_fp64_classical_interp", "amg", dict(batched=1, use_graph=1)),
                              (f"{args.kind}_fp64_classical_modified_interp", args.kind,
                               dict(batched=1, use_graph=1)),
                              (f"{args.kind}_fp64_plain_launches", args.kind, dict(interp_type=args.interp)),
                              (f"{args.kind}_fp32_vcycle_batched_graph", args.kind,
                               dict(precision=1, batched=1, use_graph=1, interp_type=args.interp)),
                              (f"{args.kind}_fp64_option3_inner_1e-2", args.kind,
                               dict(inner_mode=1, batched=1, use_graph=1, interp_type=args.interp)),
                              (f"{args.kind}_fp64_vcycles_3_1_1", args.kind,
                               dict(nvcyc_group=3, batched=1, use_graph=1, interp_type=args.interp)),
                              (f"{args.kind}_fp64_cf_gauss_seidel", args.kind,
                               dict(smoother=1, batched=1, use_graph=1, interp_type=args.interp)),
                              ("monolithic_amg_fp64_cf_gauss_seidel", "amg",
                               dict(smoother=1, batched=1, use_graph=1, interp_type=args.interp)),
                              (f"{args.kind}_fp64_aggressive_level0", args.kind,
                               dict(agg_levels=1, batched=1, use_graph=1, interp_type=args.interp))]:
            try:
                v = mgdamg.Solver(autotune=1, **o)
                v.setup(sysm.G, sysm.N, rp, ci, va, kind)
                torch.cuda.synchronize()
                t_a = time.perf_counter()
                v.setup(sysm.G, sysm.N, rp, ci, va, kind)
                xv, itv, rrv, rc = v.solve(b, tol=args.tol, allow_noconv=True)
                torch.cuda.synchronize()
                tt = time.perf_counter() - t_a
                sv = v.stats()
                err = (torch.linalg.vector_norm(xv - xg) / torch.linalg.vector_norm(xg)).item()
                variants[name] = {"iters": itv, "relres": rrv, "status": rc, "time_s": round(tt, 5),
                                  "setup_ms": round(sv["setup_ms"], 3), "solve_ms": round(sv["solve_ms"], 3),
                                  "vcycles": v.total_cycles(), "op_complexity": round(sv["op_complexity"], 4),
                                  "rel_diff_vs_fp64_x": err}
                v.close()
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)}

    peak, peak_kind = _peaks()
    ach = by0 / (t0 * 1e-3) / 1e9 if t0 > 0 else None
    # the same kernels against the FP64 issue limit, measured on this GPU now
    # (outside the timed region): on GB300 one multiply-add per 12 bytes makes
    # FP64 issue as tight a bound as HBM
    fp64 = None
    if f0 > 0 and t0 > 0:
        rate = mgdamg.fp64_issue_rate() / 1e9
        a64 = f0 / (t0 * 1e-3) / 1e9
        fp64 = {"achieved": round(a64, 1), "peak": round(rate, 1), "unit": "G FP64 lane-ops/s",
                "frac": round(a64 / rate, 4), "ops": f0,
                "peak_source": "measured in this run (mgd_fp64_issue_rate: independent multiply-add chains, "
                               "every lane active)"}
    vgbs = by1 / (t1 * 1e-3) / 1e9 if t1 > 0 else None
    traffic = _traffic_from_profiles()
    out = {
        "metric": "FGMRES time-to-1e-8 residual (s) and V-cycle HBM GB/s, mixed/batched vs FP64",
        "value": round(ms / 1e3, 6),
        "unit": "s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f64-krylov/f32-vcycle",
        "data": "synthetic",
        "config": {"workload": inputs.PRESET_NAMES[args.config] if args.kind == KIND else
                   f"{inputs.PRESET_NAMES[args.config]}[{args.kind}]",
                   "G": sysm.G, "grid": list(sysm.dims), "n": sysm.n, "nnz": sysm.nnz,
                   "precond": args.kind, "krylov": "FGMRES(30), right preconditioned", "tol": args.tol,
                   "interpolation": "extended+i" if args.interp else "classical modified",
                   "inverses": ("option #3: V-cycles to 1e-2 for the Schur-type inverses" if args.inner else
                                "option #2: V-cycles per group/E/I inverse " + args.nvcyc.replace(",", "/")),
                   "smoother": "Gauss-Seidel in C/F order (multicolour)" if args.smoother else "l1-Jacobi",
                   "aggressive_levels": args.agg,
                   "step": "device setup + solve", "parallelism": f"replicas{ws}",
                   "launch": ("batched per-level launches" if args.batched else "per-operator launches") +
                             (", preconditioner replayed from a CUDA graph" if args.graph else ""),
                   "l2": _l2_note(sysm)},
        "iters": iters[-1],
        "vcycles_per_solve": vcycles,
        "final_relres": relres,
        "setup_ms": round(statistics.median(setup_ms), 3),
        "solve_ms": round(statistics.median(solve_ms), 3),
        "vcycle_gbs": round(vgbs, 1) if vgbs else None,
        "precond_gbs_back_to_back": round(pby / (pms * 1e-3) / 1e9, 1) if pms > 0 else None,
        "precond_ms_per_apply": round(pms, 4),
        "roofline": {"bound": "hbm", "kernel": "level-0 l1-Jacobi smoothing + residual (k_pre/k_post)",
                     "achieved": round(ach, 1) if ach else None, "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4) if ach else None, "traffic": traffic,
                     "peak_source": peak_kind, "launches": n0, "ms": round(t0, 4),
                     "sampled": "every launch of the class in the first timed step",
                     "fp64_issue": fp64},
        "e2e": {"value": round(statistics.median(e2e_ms) / 1e3, 6) if e2e_ms else None, "unit": "s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "stats": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()},
        "variants": variants,
    }
    if args.adjoint:
        out["adjoint"] = adj
        out["config"]["step"] = "device setup + solve + transposed solve + value gradient"
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, sysm, iters[-1])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _l2_note(sysm):
    mb = (sysm.nnz * 12 + (sysm.n + 1) * 4) / 1e6
    if mb > 129:
        return f"inputs larger than L2 (operator {mb:.0f} MB), no flush"
    return f"operator {mb:.0f} MB fits the 129 MB L2: timed steps are warm-L2"


def _oracle_opts(args):
    """The oracle's options for the preconditioner the GPU arm runs."""
    g, e, i = (int(t) for t in args.nvcyc.split(","))
    return dict(interp_type=args.interp, inner_mode=args.inner, nvcyc_group=g, nvcyc_E=e, nvcyc_I=i,
                smoother=args.smoother, agg_levels=args.agg)


def _traffic_from_profiles():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, when it was taken from the current kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_sha256") != kernel_source_sha256():
        return None
    return d.get("traffic_bytes_per_launch")


def kernel_source_sha256():
    """Hash of the V-cycle kernel sources (the dominant kernels' code)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("vcycle_kernels.cu", "row_dot.cuh"):
        with open(os.path.join(ROOT, "paper_2002_04958_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _host_cpu():
    """Host CPU model and logical core count (the oracle uses one core)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(args, sysm, gpu_iters):
    """The FP64 oracle on the same workload, single-threaded C on one host core."""
    from oracle import oracle as orc
    orc.build()
    A = orc.csr_of_system(sysm)
    t0 = time.perf_counter()
    M = orc.Block(A, sysm.G, sysm.N, args.kind, orc.opts(**_oracle_opts(args)))
    t1 = time.perf_counter()
    budget_its = args.cpu_iters
    x, it, rr, st, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=budget_its)
    t2 = time.perf_counter()
    full = st == 0
    solve = t2 - t1
    if not full:   # scale the sampled iterations to the iteration count of the solve
        solve = solve * max(gpu_iters, it) / max(it, 1)
    return {"value": round((t1 - t0) + solve, 4), "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"full oracle setup + FGMRES solve of the same system ({it} iterations)" if full else
                       f"full oracle setup + {it} FGMRES iterations scaled to {gpu_iters}"),
            "setup_s": round(t1 - t0, 4), "iters": it, "converged": full, "host": _host_cpu()}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2002_04958_gb300 import inputs
    orc.build()
    sysm = inputs.preset(args.config)
    A = orc.csr_of_system(sysm)
    times, iters = [], []

    def step():
        t0 = time.perf_counter()
        M = orc.Block(A, sysm.G, sysm.N, args.kind, orc.opts(**_oracle_opts(args)))
        t1 = time.perf_counter()
        x, it, rr, st, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=args.ref_iters)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, it, st

    for _ in range(args.warmup):
        step()
    samples = []
    for _ in range(args.steps):
        samples.append(step())
    # the iteration count of the full solve (one oracle solve, outside the samples)
    full_its = args.full_iters
    if full_its is None:
        M = orc.Block(A, sysm.G, sysm.N, args.kind, orc.opts(**_oracle_opts(args)))
        _, full_its, _, _, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=1000)
    vals = [su + so * full_its / max(it, 1) for su, so, it, st in samples]
    v = statistics.median(vals)
    out = {
        "metric": "FGMRES time-to-1e-8 residual (s) and V-cycle HBM GB/s, mixed/batched vs FP64",
        "value": round(v, 4), "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(v * 1e3, 2), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": inputs.PRESET_NAMES[args.config], "n": sysm.n, "nnz": sysm.nnz,
                   "precond": args.kind, "interpolation": "extended+i" if args.interp else "classical modified"},
        "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: full oracle setup + {args.ref_iters} FGMRES iterations, "
                                   f"scaled to the {full_its} iterations of the full solve",
                         "host": _host_cpu()},
        "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=WORKLOAD)
    ap.add_argument("--kind", default=KIND)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--batched", type=int, default=1)
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--cpu-iters", type=int, default=30)
    ap.add_argument("--ref-iters", type=int, default=4)
    ap.add_argument("--full-iters", type=int, default=None)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="no nvidia-smi sampling (profiler runs)")
    ap.add_argument("--max-it", type=int, default=1000)
    ap.add_argument("--pdl", type=int, default=1, help="programmatic dependent launch of solve kernels")
    ap.add_argument("--inner", type=int, default=0, help="1: option #3 inverses (V-cycles to 1e-2)")
    ap.add_argument("--smoother", type=int, default=0, help="0 l1-Jacobi, 1 Gauss-Seidel in C/F order")
    ap.add_argument("--agg", type=int, default=0, help="levels coarsened aggressively (from the finest)")
    ap.add_argument("--nvcyc", default="1,1,1", help="V-cycles per group, E and I inverse")
    ap.add_argument("--interp", type=int, default=None,
                    help="0 classical modified, 1 extended+i (default: 1 for the default workload, else 0)")
    args = ap.parse_args()
    if args.interp is None:
        args.interp = 1 if (args.config == WORKLOAD and args.kind == KIND) else 0
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
