"""Preconditioner / V-cycle micro-benchmark.

Sets up one workload once, then applies the preconditioner R times and reports
the algorithmic HBM traffic of the V-cycle kernels against their device time
(CUDA events around each launch).  Also the driver for kernel profiles: with
--no-autotune the first k_pre launch after setup is the level-0 pre-smoothing
+ residual kernel of the first operator.

    python -m paper_2002_04958_gb300.kernel_bench --config 1 --kind amg --applies 5
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--dims", default=None, help="grid of the workload, e.g. 64,64,64 (default: the workload's)")
    ap.add_argument("--kind", default="amg")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--batched", type=int, default=0)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--applies", type=int, default=5)
    ap.add_argument("--timing", type=int, default=1, help="0: no CUDA events (for profiler runs)")
    ap.add_argument("--solve", action="store_true", help="also time one full solve by kernel class")
    ap.add_argument("--interp", type=int, default=0)
    ap.add_argument("--inner", type=int, default=0, help="1: option #3 inverses")
    args = ap.parse_args()

    import torch

    from paper_2002_04958_gb300 import inputs, mgdamg
    from paper_2002_04958_gb300.build import build
    build()
    s = inputs.preset(args.config, dims=[int(t) for t in args.dims.split(",")] if args.dims else None)
    slv = mgdamg.Solver(precision=args.precision, batched=args.batched, use_graph=args.graph,
                        autotune=0 if args.no_autotune else 1, interp_type=args.interp,
                        inner_mode=args.inner)
    slv.setup_system(s, args.kind)
    v = torch.from_numpy(s.b).cuda()
    if args.timing:
        slv.profile(-1)
    for _ in range(args.applies):
        slv.precond_apply(v)
    torch.cuda.synchronize()
    out = {"workload": inputs.PRESET_NAMES[args.config], "dims": list(s.dims), "kind": args.kind, "n": s.n,
           "applies": args.applies}
    if args.timing:
        for cls, name in [(0, "level0_smoothing"), (1, "vcycle_all"), (4, "block_updates")]:
            nl, ms, by = slv.profile_read(cls)
            out[name] = {"launches": nl, "ms": round(ms, 4), "GB": round(by / 1e9, 4),
                         "GBps": round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None}
        per = {}
        for lvl in range(40):
            row = []
            for ph in range(4):
                nl, ms, by = slv.profile_read(16 + 4 * lvl + ph)
                row.append(round(ms / max(args.applies, 1) * 1e3, 1))
            nl, ms, by = slv.profile_read(400 + lvl)
            row.append(round(ms / max(args.applies, 1) * 1e3, 1))
            if any(row):
                per[lvl] = row
        nl, ms, by = slv.profile_read(15)
        out["per_level_us_per_apply"] = {"columns": ["pre", "restrict", "prolong", "post", "coarse"], **per,
                                         "fused_tail": round(ms / max(args.applies, 1) * 1e3, 1)}
        slv.profile(0)
    if args.solve and not args.timing:
        slv.solve(v, tol=1e-8, allow_noconv=True)
    if args.solve and args.timing:
        import time
        slv.profile(-1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, it, rr, rc = slv.solve(v, tol=1e-8, allow_noconv=True)
        wall = (time.perf_counter() - t0) * 1e3
        cls = {}
        for k, name in [(0, "vcycle_level0"), (1, "vcycle_all"), (2, "spmv"), (3, "arnoldi"), (4, "block_updates")]:
            nl, ms, by = slv.profile_read(k)
            cls[name] = {"launches": nl, "ms": round(ms, 3), "GBps": round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None}
        busy = sum(cls[k]["ms"] for k in ["vcycle_all", "spmv", "arnoldi", "block_updates"])
        out["solve"] = {"iters": it, "wall_ms": round(wall, 3), "kernel_ms": round(busy, 3),
                        "idle_ms": round(wall - busy, 3), "classes": cls}
        slv.profile(0)
    st = slv.stats()
    out["setup_ms"] = round(st["setup_ms"], 3)
    out["setup_phases_ms"] = slv.setup_phases()
    # a second setup of the same system (autotune decisions cached)
    slv.setup_system(s, args.kind)
    out["setup2_ms"] = round(slv.stats()["setup_ms"], 3)
    out["setup2_phases_ms"] = slv.setup_phases()
    out["plan"] = slv.plan()
    out["vcycle_bytes_per_apply"] = st["vcycle_bytes"]
    out["levels"] = st["max_levels_used"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
