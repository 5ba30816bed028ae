"""Writes oracle_fgmres_G1_1024x1024_schur1_exti.json: the FP64 oracle's
right-preconditioned FGMRES(30) with the Schur1 block preconditioner
(Section 3.4, one V(1,1) classical-AMG cycle per inverse, PMIS coarsening with
extended+i interpolation) on the one-group 1024 x 1024 system with the
circular inclusion (3,145,728 unknowns), tol 1e-8, zero initial guess -- the
benchmark's one-group workload.

It calls only the oracle (about half a minute on one host core).  The GPU
full-size test checks its iteration count, residual and solution against
these figures.

    python tests/golden/make_oracle_fgmres_G1_1024x1024.py
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

OUT = os.path.join(HERE, "oracle_fgmres_G1_1024x1024_schur1_exti.json")
N_SAMPLES = 256


def main():
    s = I.preset(1)
    Ao = orc.csr_of_system(s)
    t0 = time.perf_counter()
    ob = orc.Block(Ao, s.G, s.N, "schur1", orc.opts(interp_type=1))
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    t1 = time.perf_counter()
    assert sto == 0
    rng = np.random.default_rng(11)
    idx = np.sort(np.concatenate([rng.choice(s.n, N_SAMPLES - 1, replace=False), [int(np.argmax(np.abs(xo)))]]))
    rec = {
        "workload": I.PRESET_NAMES[1], "n": int(s.n), "nnz": int(s.nnz), "tol": 1e-8,
        "precond": "schur1", "interpolation": "extended+i",
        "iterations": int(ito), "relres": float(rro),
        "x_norm2": float(np.linalg.norm(xo)), "x_max_abs": float(np.abs(xo).max()),
        "sample_index": [int(i) for i in idx],
        "sample_x": [float(xo[i]) for i in idx],
        "written_by": "python tests/golden/make_oracle_fgmres_G1_1024x1024.py",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(OUT, ito, rro, f"{t1 - t0:.1f} s")


if __name__ == "__main__":
    main()
