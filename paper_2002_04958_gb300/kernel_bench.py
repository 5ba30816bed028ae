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
    ap.add_argument("--kind", default="amg")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--batched", type=int, default=0)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--applies", type=int, default=5)
    ap.add_argument("--timing", type=int, default=1, help="0: no CUDA events (for profiler runs)")
    args = ap.parse_args()

    import torch

    from paper_2002_04958_gb300 import inputs, mgdamg
    from paper_2002_04958_gb300.build import build
    build()
    s = inputs.preset(args.config)
    slv = mgdamg.Solver(precision=args.precision, batched=args.batched, use_graph=args.graph,
                        autotune=0 if args.no_autotune else 1)
    slv.setup_system(s, args.kind)
    v = torch.from_numpy(s.b).cuda()
    if args.timing:
        slv.profile(-1)
    for _ in range(args.applies):
        slv.precond_apply(v)
    torch.cuda.synchronize()
    out = {"workload": inputs.PRESET_NAMES[args.config], "kind": args.kind, "n": s.n, "applies": args.applies}
    if args.timing:
        for cls, name in [(0, "level0_smoothing"), (1, "vcycle_all"), (4, "block_updates")]:
            nl, ms, by = slv.profile_read(cls)
            out[name] = {"launches": nl, "ms": round(ms, 4), "GB": round(by / 1e9, 4),
                         "GBps": round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None}
        slv.profile(0)
    st = slv.stats()
    out["vcycle_bytes_per_apply"] = st["vcycle_bytes"]
    out["levels"] = st["max_levels_used"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
