#!/usr/bin/env python
"""Benchmark: FGMRES time to a 1e-8 relative residual and V-cycle HBM GB/s,
FP32-V-cycle/batched form against the FP64 form.

Workload (default): the 20-group system on a 96x96x96 grid (22 components,
7-point TPFA stencils, 19,464,192 unknowns, 166,938,624 nonzeros, seeded
synthetic coefficients), preconditioned by Schur2 (Section 3.5) with one
classical-AMG V(1,1) cycle per subsystem inverse (PMIS coarsening, classical
modified interpolation, l1-Jacobi smoothing).  One step = the whole hot path
on that system: device setup (block extraction, strength, PMIS, interpolation,
Galerkin products, smoother diagonals, coarsest inverse) plus the FGMRES(30)
solve to ||b - A x|| <= 1e-8 ||b||.

`value` is the FP64 form (FP64 hierarchy and Krylov; the 22 subsystem V-cycles
of a Schur2 stage batched into one launch per level and the preconditioner
replayed from a CUDA graph).  `mixed` is the same workload with the hierarchy
stored and smoothed in FP32 inside the FP64 FGMRES, timed the same way.  Both
report their final error against the stored FP64 oracle solve of the workload
(tests/golden/).  Inputs are resident in HBM before the timed region; the
operator (2.0 GB) is larger than L2, so no flush is needed between steps.

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

WORKLOAD = 3
METRIC = "FGMRES time-to-1e-8 residual (s) and V-cycle HBM GB/s, mixed/batched vs FP64"
# preconditioner of each workload (the bench's default for --config k)
KINDS_OF = {0: "amg", 1: "schur1", 2: "bd", 3: "schur2", 4: "amg"}
# stored oracle solves (written by the scripts beside them, which call only the oracle)
GOLDEN = {1: "oracle_fgmres_G1_1024x1024_schur1_exti.json", 3: "oracle_fgmres_G20_96x96x96_schur2.json"}
ARNOLDI_KERNEL = "FGMRES orthogonalisation (k_dot_partial2, k_mgs_step2 x (j+1), k_sum_partials, k_scale_by_norm2)"
MGS_KERNEL = "k_mgs_step2 (fused modified Gram-Schmidt step: w -= h_i v_i, partial <v_i+1, w>)"


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


def _golden(config):
    """The stored oracle solve of a workload (written by tests/golden/make_oracle_*.py,
    which call only the oracle), or None."""
    name = GOLDEN.get(config)
    if not name:
        return None
    p = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def _final_error(x, rec):
    """Error of a GPU solution against the stored FP64 oracle solve: the largest
    |x_i - x_oracle,i| over the stored entries (they include the oracle's
    largest entry) relative to max|x_oracle|, and the relative difference of
    the 2-norms."""
    import numpy as np
    if rec is None:
        return None
    idx = np.asarray(rec["sample_index"])
    xs = x[idx].cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)[idx]
    scale = rec.get("x_max_abs") or float(np.abs(np.asarray(rec["sample_x"])).max())
    import torch
    return {"max_abs_err_over_max_abs_x": float(np.abs(xs - np.asarray(rec["sample_x"])).max() / scale),
            "norm2_rel_diff": float(abs(torch.linalg.vector_norm(x).item() - rec["x_norm2"]) / rec["x_norm2"]),
            "oracle_iterations": rec["iterations"], "entries_compared": int(idx.size)}


def _timed_steps(step, steps, warmup, barrier, sync):
    """W untimed steps, then K steps bracketed by CUDA events; (ms per step, last result)."""
    import torch
    out = None
    for _ in range(warmup):
        out = step(-1)
    sync()
    barrier()
    sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        out = step(k)
    e1.record()
    sync()
    barrier()
    return e0.elapsed_time(e1) / steps, out


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
    rec = _golden(args.config) if args.kind == KINDS_OF.get(args.config) and args.interp == _default_interp(
        args.config) else None
    # the end-to-end leg's inputs in page-locked host memory, allocated before
    # any device work (as an application would set up its staging buffers once)
    if not args.no_e2e:
        h_rp = torch.from_numpy(sysm.rowptr).pin_memory()
        h_ci = torch.from_numpy(sysm.col).pin_memory()
        h_va = torch.from_numpy(sysm.val).pin_memory()
        h_b = torch.from_numpy(sysm.b).pin_memory()
        h_x = torch.zeros(sysm.n, dtype=torch.float64).pin_memory()
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(sysm.rowptr).to(dev)
    ci = torch.from_numpy(sysm.col).to(dev)
    va = torch.from_numpy(sysm.val).to(dev)
    b = torch.from_numpy(sysm.b).to(dev)
    ncyc = [int(t) for t in args.nvcyc.split(",")]
    base = dict(batched=args.batched, use_graph=args.graph, autotune=1, keep_transpose=int(args.adjoint),
                max_it=args.max_it, interp_type=args.interp, pdl=args.pdl, inner_mode=args.inner,
                nvcyc_group=ncyc[0], nvcyc_E=ncyc[1], nvcyc_I=ncyc[2], smoother=args.smoother,
                agg_levels=args.agg)
    slv = mgdamg.Solver(precision=args.precision, **base)
    adj = {}
    sync = torch.cuda.synchronize

    # -------------------------------------------------- headline: the FP64 form
    log = {"setup_ms": [], "solve_ms": [], "iters": []}
    prof = {}

    def step(k):
        if k == 0:   # the first timed step brackets the dominant kernel classes with events
            slv.profile(0b101001)
        slv.setup(sysm.G, sysm.N, rp, ci, va, args.kind)
        x, it, rr, rc = slv.solve(b, tol=args.tol)
        if args.adjoint:   # L = ||x||^2: lambda = A^-T (2x), dL/dvals = -lambda_row x_col
            lam, ita, rra = slv.solve_transpose(2.0 * x, tol=args.tol)
            slv.grad_values(x, lam)
            adj.update(iters_transpose=ita, relres_transpose=rra)
        if k >= 0:
            st = slv.stats()
            log["setup_ms"].append(st["setup_ms"])
            log["solve_ms"].append(st["solve_ms"])
            log["iters"].append(it)
        if k == 0:
            prof["l0"] = slv.profile_read(0)
            prof["l0_fp64"] = slv.profile_read_fp64(0)
            prof["arn"] = slv.profile_read(3)
            prof["mgs"] = slv.profile_read(5)
            slv.profile(0)
        return x, it, rr

    clocks = ClockSampler(local, enabled=not args.no_clocks)
    l0 = mgdamg.kernel_launches()
    clocks.start()
    ms, (x, it, rr) = _timed_steps(step, args.steps, args.warmup, _barrier, sync)
    clk = clocks.stop()
    launches = mgdamg.kernel_launches() - l0
    ms = _max_over_ranks(ms, dev)
    xg, relres = x, rr
    err64 = _final_error(xg, rec)

    # per-level V-cycle table: one more (untimed) solve with every V-cycle kernel bracketed
    slv.profile(0b11)
    x1, it1, rr1 = step(-1)
    vcycles = slv.total_cycles()   # V-cycles of one solve (counted since its setup)
    n1, t1, by1 = slv.profile_read(1)
    per_level = []
    for lvl in range(40):
        row = {"level": lvl}
        tot_ms = tot_by = 0.0
        for ph, name in enumerate(["pre", "restrict", "prolong", "post"]):
            nl, pm, pb = slv.profile_read(16 + 4 * lvl + ph)
            row[name + "_us"] = round(pm / max(it1, 1) * 1e3, 2)
            if pm > 0:
                row[name + "_GBps"] = round(pb / (pm * 1e-3) / 1e9, 1)
            tot_ms += pm
            tot_by += pb
        nl, pm, pb = slv.profile_read(400 + lvl)
        if pm > 0:
            row["coarse_us"] = round(pm / max(it1, 1) * 1e3, 2)
        tot_ms += pm
        tot_by += pb
        if tot_ms > 0:
            row["MB_per_apply"] = round(tot_by / max(it1, 1) / 1e6, 3)
            row["GBps"] = round(tot_by / (tot_ms * 1e-3) / 1e9, 1)
            per_level.append(row)
    slv.profile(0)
    # preconditioner bandwidth: 100 applies back to back (graph replays), no per-kernel events
    pms, pby = slv.precond_bench(b, 100)
    st = slv.stats()

    # -------------------------------------------------- the mixed form: FP32 V-cycles in FP64 FGMRES
    mixed = None
    if not args.no_mixed and args.precision == 0:
        slv_m = mgdamg.Solver(precision=1, **base)
        mlog = {"setup_ms": [], "solve_ms": [], "iters": []}

        def mstep(k):
            slv_m.setup(sysm.G, sysm.N, rp, ci, va, args.kind)
            xm, itm, rrm, rcm = slv_m.solve(b, tol=args.tol)
            if k >= 0:
                stm = slv_m.stats()
                mlog["setup_ms"].append(stm["setup_ms"])
                mlog["solve_ms"].append(stm["solve_ms"])
                mlog["iters"].append(itm)
            return xm, itm, rrm

        mclk = ClockSampler(local, enabled=not args.no_clocks)
        mclk.start()
        mms, (xm, itm, rrm) = _timed_steps(mstep, args.steps, max(3, min(args.warmup, 3)), _barrier, sync)
        mclk_r = mclk.stop()
        mms = _max_over_ranks(mms, dev)
        slv_m.profile(0b11)
        mstep(-1)
        mn1, mt1, mby1 = slv_m.profile_read(1)
        slv_m.profile(0)
        mpms, mpby = slv_m.precond_bench(b, 100)
        mixed = {"value": round(mms / 1e3, 6), "unit": "s", "ms_per_step": round(mms, 4),
                 "speedup_vs_fp64": round(ms / mms, 4), "iters": itm, "final_relres": rrm,
                 "setup_ms": round(statistics.median(mlog["setup_ms"]), 3),
                 "solve_ms": round(statistics.median(mlog["solve_ms"]), 3),
                 "vcycle_gbs": round(mby1 / (mt1 * 1e-3) / 1e9, 1) if mt1 > 0 else None,
                 "precond_gbs_back_to_back": round(mpby / (mpms * 1e-3) / 1e9, 1) if mpms > 0 else None,
                 "precond_ms_per_apply": round(mpms, 4),
                 "final_error_vs_oracle": _final_error(xm, rec),
                 "rel_diff_vs_fp64_gpu_x": (torch.linalg.vector_norm(xm - xg) /
                                            torch.linalg.vector_norm(xg)).item(),
                 "dtype": "f64-krylov/f32-vcycle", "clocks": mclk_r,
                 "launch": "batched per-level launches, preconditioner replayed from a CUDA graph"}
        slv_m.close()
        del slv_m

    # -------------------------------------------------- end to end through the C ABI with host buffers
    # the adjoint step also returns the value gradient: x goes back to the
    # device for the transposed solve, the gradient comes to the host
    d_x = torch.empty(sysm.n, dtype=torch.float64, device=dev) if args.adjoint else None
    h_g = torch.empty(sysm.nnz, dtype=torch.float64).pin_memory() if args.adjoint else None
    e2e_ms, e2e_parts = [], []
    for k in range(0 if args.no_e2e else max(2, args.steps // 2) + 1):
        sync()
        t_a = time.perf_counter()
        slv.setup_host(sysm.G, sysm.N, h_rp, h_ci, h_va, args.kind)
        t_s = time.perf_counter()
        h_x.zero_()
        slv.solve_host_ptr(h_b.data_ptr(), h_x.data_ptr(), tol=args.tol)
        if k > 0:
            st_e = slv.stats()
            ph = slv.setup_phases()
            e2e_parts.append(((t_s - t_a) * 1e3, st_e["setup_ms"], (time.perf_counter() - t_s) * 1e3,
                              st_e["solve_ms"], ph["h2d_copies"], ph["release_previous"]))
        if args.adjoint:
            d_x.copy_(h_x, non_blocking=True)
            lam_e, _, _ = slv.solve_transpose(2.0 * d_x, tol=args.tol)
            h_g.copy_(slv.grad_values(d_x, lam_e), non_blocking=True)
        sync()
        if k > 0:
            e2e_ms.append((time.perf_counter() - t_a) * 1e3)
    h2d = sysm.rowptr.nbytes + sysm.col.nbytes + sysm.val.nbytes + sysm.b.nbytes + sysm.n * 8
    d2h = sysm.n * 8
    if args.adjoint:
        h2d += sysm.n * 8
        d2h += sysm.nnz * 8
    del h_rp, h_ci, h_va

    # -------------------------------------------------- variants for context (one solve each, outside the timed region)
    variants = {}
    if not args.no_variants:
        for name, cfg, kind, o in _variants(args):
            try:
                vs = sysm if cfg == args.config else inputs.preset(cfg)
                vrec = rec if cfg == args.config else _golden(cfg)
                if cfg == args.config:
                    vrp, vci, vva, vb = rp, ci, va, b
                else:
                    vrp, vci, vva, vb = (torch.from_numpy(a).to(dev) for a in (vs.rowptr, vs.col, vs.val, vs.b))
                v = mgdamg.Solver(autotune=1, **o)
                v.setup(vs.G, vs.N, vrp, vci, vva, kind)
                sync()
                t_a = time.perf_counter()
                v.setup(vs.G, vs.N, vrp, vci, vva, kind)
                xv, itv, rrv, rc = v.solve(vb, tol=args.tol, allow_noconv=True)
                sync()
                tt = time.perf_counter() - t_a
                sv = v.stats()
                d = {"workload": inputs.PRESET_NAMES[cfg], "precond": kind, "iters": itv, "relres": rrv,
                     "status": rc, "converged": rc == 0, "time_s": round(tt, 5),
                     "setup_ms": round(sv["setup_ms"], 3), "solve_ms": round(sv["solve_ms"], 3),
                     "vcycles": v.total_cycles(), "op_complexity": round(sv["op_complexity"], 4)}
                if cfg == args.config:
                    d["rel_diff_vs_fp64_gpu_x"] = (torch.linalg.vector_norm(xv - xg) /
                                                   torch.linalg.vector_norm(xg)).item()
                if vrec is not None and o.get("interp_type", 0) == _default_interp(cfg) and kind == KINDS_OF.get(cfg):
                    d["final_error_vs_oracle"] = _final_error(xv, vrec)
                variants[name] = d
                v.close()
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)}

    peak, peak_kind = _peaks()
    out_workload = _config(args, sysm, ws)["workload"]
    n0, t0, by0 = prof["l0"]
    na, ta, bya = prof["arn"]
    l0_ach = by0 / (t0 * 1e-3) / 1e9 if t0 > 0 else None
    arn_ach = bya / (ta * 1e-3) / 1e9 if ta > 0 else None
    # the same level-0 kernels against the FP64 issue limit, measured on this GPU now
    # (outside the timed region): on GB300 one multiply-add per 12 bytes makes
    # FP64 issue as tight a bound as HBM
    fp64 = None
    f0 = prof["l0_fp64"]
    if f0 > 0 and t0 > 0:
        rate = mgdamg.fp64_issue_rate() / 1e9
        a64 = f0 / (t0 * 1e-3) / 1e9
        fp64 = {"achieved": round(a64, 1), "peak": round(rate, 1), "unit": "G FP64 lane-ops/s",
                "frac": round(a64 / rate, 4), "ops": f0,
                "peak_source": "measured in this run (mgd_fp64_issue_rate: independent multiply-add chains, "
                               "every lane active)"}
    level0 = {"kernel": "level-0 l1-Jacobi smoothing + residual (k_pre/k_post)",
              "achieved": round(l0_ach, 1) if l0_ach else None, "peak": peak, "unit": "GB/s",
              "frac": round(l0_ach / peak, 4) if l0_ach else None, "launches": n0, "ms": round(t0, 4),
              "bytes_per_launch": round(by0 / max(n0, 1)), "fp64_issue": fp64,
              "traffic": _traffic_from_profiles("level0", out_workload)}
    nm, tm, bym = prof["mgs"]
    mgs_ach = bym / (tm * 1e-3) / 1e9 if tm > 0 else None
    arnoldi = {"kernel": ARNOLDI_KERNEL, "achieved": round(arn_ach, 1) if arn_ach else None, "peak": peak,
               "unit": "GB/s", "frac": round(arn_ach / peak, 4) if arn_ach else None, "launches": na,
               "ms": round(ta, 4), "bytes_per_launch": round(bya / max(na, 1)),
               "note": "one launch = one orthogonalisation: first dot product, the fused steps, the norm, "
                       "the normalisation"}
    # class 5 brackets the j+1 step launches of each orthogonalisation together:
    # per kernel launch, 32 n algorithmic bytes
    nmk = int(round(bym / (32.0 * sysm.n))) if bym > 0 else 0
    mgs = {"kernel": MGS_KERNEL, "achieved": round(mgs_ach, 1) if mgs_ach else None, "peak": peak, "unit": "GB/s",
           "frac": round(mgs_ach / peak, 4) if mgs_ach else None, "launches": nmk, "ms": round(tm, 4),
           "bytes_per_launch": 32 * sysm.n, "traffic": _traffic_from_profiles("mgs", out_workload),
           "timed_as": f"{nm} bracketed groups (the steps of one orthogonalisation each)",
           "arnoldi_class": arnoldi}
    # the dominant kernel: the larger device time in the profiled step (the
    # fused Gram-Schmidt step launches are timed as one class per orthogonalisation)
    dom, other = (mgs, level0) if tm > t0 else (level0, mgs)
    roof = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["achieved"], "peak": peak, "unit": "GB/s",
            "frac": dom["frac"], "traffic": dom["traffic"], "peak_source": peak_kind,
            "launches": dom["launches"], "ms": dom["ms"], "bytes_per_launch": dom["bytes_per_launch"],
            "sampled": "every launch of the class in the first timed step (CUDA events on the solver's stream)",
            "other_class": other}
    if dom is level0:
        roof["fp64_issue"] = fp64
    vgbs = by1 / (t1 * 1e-3) / 1e9 if t1 > 0 else None
    out = {
        "metric": METRIC,
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
        "config": _config(args, sysm, ws),
        "iters": log["iters"][-1],
        "vcycles_per_solve": vcycles,
        "final_relres": relres,
        "final_error_vs_oracle": err64,
        "setup_ms": round(statistics.median(log["setup_ms"]), 3),
        "solve_ms": round(statistics.median(log["solve_ms"]), 3),
        "vcycle_gbs": round(vgbs, 1) if vgbs else None,
        "vcycle_frac": round(vgbs / peak, 4) if vgbs else None,
        "precond_gbs_back_to_back": round(pby / (pms * 1e-3) / 1e9, 1) if pms > 0 else None,
        "precond_frac_back_to_back": round(pby / (pms * 1e-3) / 1e9 / peak, 4) if pms > 0 else None,
        "precond_ms_per_apply": round(pms, 4),
        "mixed": mixed,
        "roofline": roof,
        "e2e": {"value": round(statistics.median(e2e_ms) / 1e3, 6) if e2e_ms else None, "unit": "s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "path": "mgd_setup_host (page-locked host CSR arrays) + mgd_solve_host (host b, host x)",
                "parts_ms_median": ({"setup_host_call": round(statistics.median(p[0] for p in e2e_parts), 3),
                                     "setup_inside": round(statistics.median(p[1] for p in e2e_parts), 3),
                                     "solve_host_call": round(statistics.median(p[2] for p in e2e_parts), 3),
                                     "solve_inside": round(statistics.median(p[3] for p in e2e_parts), 3),
                                     "h2d_csr_copies": round(statistics.median(p[4] for p in e2e_parts), 3),
                                     "release_previous_setup": round(statistics.median(p[5] for p in e2e_parts),
                                                                     3)}
                                    if e2e_parts else None)},
        "gpu_launches": launches,
        "clocks": clk,
        "stats": dict({k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()},
                      per_level_per_apply=per_level),
        "variants": variants,
    }
    if args.adjoint:
        out["adjoint"] = adj
        out["config"]["step"] = "device setup + solve + transposed solve + value gradient"
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, sysm, rec, log["iters"][-1])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _default_interp(config):
    return 1 if config == 1 else 0


def _variants(args):
    """(name, config, preconditioner, solver options) of the context runs."""
    k, c, i = args.kind, args.config, args.interp
    v = [(f"{k}_fp64_per_operator_launches", c, k, dict(interp_type=i)),
         (f"{k}_fp32_vcycle_per_operator_launches", c, k, dict(precision=1, interp_type=i))]
    if c == 3:
        v += [("schur1_fp64_batched_graph", 3, "schur1", dict(batched=1, use_graph=1)),
              ("monolithic_amg_fp32_vcycle_cf_gauss_seidel", 3, "amg",
               dict(precision=1, smoother=1, batched=1, use_graph=1)),
              ("G1_1024x1024_schur1_exti_fp64_batched_graph", 1, "schur1",
               dict(interp_type=1, batched=1, use_graph=1)),
              ("G1_1024x1024_schur1_exti_fp32_vcycle_batched_graph", 1, "schur1",
               dict(precision=1, interp_type=1, batched=1, use_graph=1)),
              ("G1_1024x1024_monolithic_amg_exti_cf_gauss_seidel", 1, "amg",
               dict(interp_type=1, smoother=1, batched=1, use_graph=1))]
    elif c == 1:
        v += [("monolithic_amg_fp64_classical_interp_l1jacobi", 1, "amg", dict(batched=1, use_graph=1)),
              ("monolithic_amg_fp64_exti_cf_gauss_seidel", 1, "amg",
               dict(smoother=1, batched=1, use_graph=1, interp_type=1)),
              (f"{k}_fp64_option3_inner_1e-2", 1, k, dict(inner_mode=1, batched=1, use_graph=1, interp_type=i)),
              (f"{k}_fp64_vcycles_3_1_1", 1, k, dict(nvcyc_group=3, batched=1, use_graph=1, interp_type=i))]
    return v


def _config(args, sysm, ws):
    from paper_2002_04958_gb300 import inputs
    default = args.kind == KINDS_OF.get(args.config) and args.interp == _default_interp(args.config)
    return {"workload": inputs.PRESET_NAMES[args.config] if default else
            f"{inputs.PRESET_NAMES[args.config]}[{args.kind},interp{args.interp}]",
            "G": sysm.G, "grid": list(sysm.dims), "n": sysm.n, "nnz": sysm.nnz,
            "precond": args.kind, "krylov": "FGMRES(30), right preconditioned", "tol": args.tol,
            "interpolation": "extended+i" if args.interp else "classical modified",
            "inverses": ("option #3: V-cycles to 1e-2 for the Schur-type inverses" if args.inner else
                         "option #2: V-cycles per group/E/I inverse " + args.nvcyc.replace(",", "/")),
            "smoother": "Gauss-Seidel in C/F order (multicolour)" if args.smoother else "l1-Jacobi",
            "aggressive_levels": args.agg,
            "precision": "FP64 everywhere" if args.precision == 0 else "FP32 V-cycles, FP64 Krylov",
            "step": "device setup + solve", "parallelism": f"replicas{ws}",
            "launch": ("batched per-level launches" if args.batched else "per-operator launches") +
                      (", preconditioner replayed from a CUDA graph" if args.graph else ""),
            "l2": _l2_note(sysm)}


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


def _traffic_from_profiles(name, workload):
    """DRAM bytes per launch of kernel class `name` ("level0", "mgs") on this
    workload from the committed ncu summary, when it was taken on this workload
    from the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(name)
    if not d or d.get("kernel_source_sha256") != kernel_source_sha256(name) or d.get("workload") != workload:
        return None
    return d.get("traffic_bytes_per_launch")


# source of each kernel class: (file, first marker, end marker); with markers,
# only the text from the first marker up to the end marker is hashed (the
# kernels of the class and their launcher), else the whole file
TRAFFIC_SOURCES = {
    "level0": (("vcycle_kernels.cu", None, None), ("row_dot.cuh", None, None)),
    "mgs": (("solve_kernels.cu", "constexpr int kMgsU", "// v = w / ||w||: one reciprocal per block"),),
}


def kernel_source_sha256(name="level0"):
    """Hash of the source of a kernel class (the code its traffic was measured
    on); None when a marker of the class's source region is missing."""
    import hashlib
    h = hashlib.sha256()
    for fn, first, end in TRAFFIC_SOURCES[name]:
        with open(os.path.join(ROOT, "paper_2002_04958_gb300", "csrc", fn), "rb") as f:
            text = f.read()
        if first is not None:
            i = text.find(first.encode())
            j = text.find(end.encode(), i) if i >= 0 else -1
            if j < 0:
                return None
            text = text[i:j]
        h.update(text)
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


def _oracle_iterations(args, rec):
    """Iteration count of the oracle's full solve: the stored one when the
    workload has a golden record, else --full-iters (None: unknown)."""
    if rec is not None:
        return rec["iterations"]
    return args.full_iters


def _cpu_iters(args):
    if args.cpu_iters is not None:
        return args.cpu_iters
    return 2 if args.config == 3 else 1000


def cpu_baseline(args, sysm, rec, gpu_iters):
    """The FP64 oracle on the same workload, single-threaded C on one host core.

    A full oracle setup, then FGMRES from x = 0: to convergence when that fits
    the sample budget (config 1: about half a minute), else a few iterations
    scaled linearly to the iteration count of the stored oracle solve.  Linear
    scaling under-counts the Gram-Schmidt work, which grows with the Krylov
    depth, so the scaled figure is a lower bound on the oracle's time."""
    from oracle import oracle as orc
    orc.build()
    A = orc.csr_of_system(sysm)
    t0 = time.perf_counter()
    M = orc.Block(A, sysm.G, sysm.N, args.kind, orc.opts(**_oracle_opts(args)))
    t1 = time.perf_counter()
    budget_its = _cpu_iters(args)
    x, it, rr, st, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=budget_its)
    t2 = time.perf_counter()
    full = st == 0
    solve = t2 - t1
    target = _oracle_iterations(args, rec) or gpu_iters
    if not full:   # scale the sampled iterations to the iteration count of the solve
        solve = solve * target / max(it, 1)
    out = {"value": round((t1 - t0) + solve, 4), "unit": "s", "cores": 1, "kind": "oracle",
           "sample": (f"full oracle setup + FGMRES solve of the same system ({it} iterations)" if full else
                      f"full oracle setup + {it} FGMRES iterations, solve time scaled linearly to the "
                      f"{target} iterations of the stored oracle solve (a lower bound: Gram-Schmidt work "
                      f"grows with the Krylov depth)"),
           "setup_s": round(t1 - t0, 4), "iters": it, "converged": full, "extrapolated": not full,
           "host": _host_cpu()}
    if not full and args.config == 3 and not args.no_full_oracle:
        # one complete oracle solve, not extrapolated, on the one-group workload
        # (about half a minute), beside the GPU variant of that workload
        from paper_2002_04958_gb300 import inputs
        s1 = inputs.preset(1)
        A1 = orc.csr_of_system(s1)
        t0 = time.perf_counter()
        M1 = orc.Block(A1, s1.G, s1.N, "schur1", orc.opts(interp_type=1))
        t1 = time.perf_counter()
        _, it1, rr1, st1, _ = orc.fgmres(A1, s1.b, M1, tol=args.tol, maxit=1000)
        t2 = time.perf_counter()
        out["full_solve_one_group_workload"] = {
            "workload": inputs.PRESET_NAMES[1], "precond": "schur1", "interpolation": "extended+i",
            "value": round(t2 - t0, 4), "unit": "s", "setup_s": round(t1 - t0, 4), "solve_s": round(t2 - t1, 4),
            "iters": it1, "relres": rr1, "converged": st1 == 0, "extrapolated": False, "cores": 1}
    return out


def run_reference(args):
    """The oracle as the reference arm: one full oracle setup (timed once), then
    per step a bounded sample of the solve -- `--ref-iters` FGMRES iterations
    from x = 0 -- scaled linearly to the iteration count of the full solve;
    value = setup time + the median scaled solve time."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2002_04958_gb300 import inputs
    orc.build()
    sysm = inputs.preset(args.config)
    rec = _golden(args.config) if args.kind == KINDS_OF.get(args.config) and args.interp == _default_interp(
        args.config) else None
    A = orc.csr_of_system(sysm)
    t0 = time.perf_counter()
    M = orc.Block(A, sysm.G, sysm.N, args.kind, orc.opts(**_oracle_opts(args)))
    setup_s = time.perf_counter() - t0
    k = args.ref_iters if args.ref_iters is not None else (2 if args.config == 3 else 4)

    def step():
        t1 = time.perf_counter()
        x, it, rr, st, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=k)
        return time.perf_counter() - t1, it, st

    for _ in range(args.warmup):
        step()
    samples = [step() for _ in range(args.steps)]
    full_its = _oracle_iterations(args, rec)
    if full_its is None:   # one full oracle solve (outside the samples) gives the iteration count
        _, full_its, _, _, _ = orc.fgmres(A, sysm.b, M, tol=args.tol, maxit=args.max_it)
    vals = [setup_s + so * full_its / max(it, 1) for so, it, st in samples]
    v = statistics.median(vals)
    out = {
        "metric": METRIC,
        "value": round(v, 4), "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(v * 1e3, 2), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": _config(args, sysm, ws),
        "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"one full oracle setup ({setup_s:.2f} s, timed once), then per step "
                                   f"{k} FGMRES iterations from x = 0, solve time scaled linearly to the "
                                   f"{full_its} iterations of the full oracle solve (a lower bound: "
                                   f"Gram-Schmidt work grows with the Krylov depth)",
                         "setup_s": round(setup_s, 4),
                         "step_s_median": round(statistics.median(so for so, _, _ in samples), 4),
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
    ap.add_argument("--kind", default=None, help="preconditioner (default: the workload's)")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--batched", type=int, default=1)
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--cpu-iters", type=int, default=None,
                    help="oracle FGMRES iterations of the cpu_baseline sample (default: a full solve, 2 on config 3)")
    ap.add_argument("--ref-iters", type=int, default=None,
                    help="oracle FGMRES iterations per reference step (default 2 on config 3, else 4)")
    ap.add_argument("--full-iters", type=int, default=None)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-V-cycle form")
    ap.add_argument("--no-full-oracle", action="store_true",
                    help="cpu_baseline without the complete oracle solve of the one-group workload")
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
    if args.kind is None:
        args.kind = KINDS_OF.get(args.config, "amg")
    if args.interp is None:
        args.interp = _default_interp(args.config) if args.kind == KINDS_OF.get(args.config) else 0
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
