"""Writes oracle_options_fullsize.json: the FP64 oracle's FGMRES(30) solves (tol
1e-8, zero initial guess) of full-size workloads with the options beside the
default path:

  * the one-group 1024 x 1024 system, Schur1 with extended+i interpolation and
    option #3 inverses (V-cycles to 1e-2, Section 4), and with option #4 for
    C_E (Section 3.5, three steps of the recurrence);
  * the same system with the electron energy diffusing (Eq. 2.1 as printed),
    Schur1 with extended+i interpolation;
  * the 20-group 256 x 256 system, monolithic AMG with the C/F Gauss-Seidel
    smoother (Section 3.1).

For each: iterations, final relative residual, norms, the V-cycle count of
every inverse, and 256 seeded solution entries (the largest included).  It
calls only the oracle (a few minutes on one host core).

    python tests/golden/make_oracle_options_fullsize.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc                   # noqa: E402
from paper_2002_04958_gb300 import inputs as I     # noqa: E402

OUT = os.path.join(HERE, "oracle_options_fullsize.json")
N_SAMPLES = 256

CASES = {
    "G1_1024x1024_schur1_exti_option3": (1, "schur1", dict(interp_type=1, inner_mode=1)),
    "G1_1024x1024_schur1_exti_option4_k3": (1, "schur1", dict(interp_type=1, opt4_steps=3)),
    "G1_1024x1024_diffuseE_schur1_exti": (5, "schur1", dict(interp_type=1)),
    "G20_256x256_amg_cf_gauss_seidel": (2, "amg", dict(smoother=1)),
}


def main():
    out = {}
    for name, (cfg, kind, o) in CASES.items():
        s = I.preset(cfg)
        Ao = orc.csr_of_system(s)
        t0 = time.perf_counter()
        ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(**o))
        xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
        t1 = time.perf_counter()
        assert sto == 0, (name, sto)
        cycles = {}
        for op in range(7):
            for comp in range(s.nc):
                c = ob.cycles(op, comp)
                if c:
                    cycles[f"{op},{comp}"] = int(c)
        rng = np.random.default_rng(23)
        idx = np.sort(np.concatenate([rng.choice(s.n, N_SAMPLES - 1, replace=False), [int(np.argmax(np.abs(xo)))]]))
        out[name] = {
            "workload": I.PRESET_NAMES[cfg], "preset": cfg, "n": int(s.n), "nnz": int(s.nnz), "precond": kind,
            "options": o, "tol": 1e-8, "iterations": int(ito), "relres": float(rro),
            "x_norm2": float(np.linalg.norm(xo)), "x_max_abs": float(np.abs(xo).max()),
            "cycles": cycles,
            "sample_index": [int(i) for i in idx], "sample_x": [float(xo[i]) for i in idx],
        }
        print(name, ito, rro, f"{t1 - t0:.1f} s", flush=True)
    out["written_by"] = "python tests/golden/make_oracle_options_fullsize.py"
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
