"""Writes oracle_fgmres_G20_96x96x96_schur2.json: the FP64 oracle's
right-preconditioned FGMRES(30) with the Schur2 block preconditioner
(Section 3.2, V(1,1) classical AMG per diagonal block) on the 20-group
96 x 96 x 96 system (19,464,192 unknowns), tol 1e-8, zero initial guess.

It calls only the oracle (about four minutes on one host core); the GPU
full-size test compares its own solve against the stored figures, because the
oracle's solve is too slow to repeat inside the test.

    python tests/golden/make_oracle_fgmres_G20_96x96x96.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc                   # noqa: E402
from paper_2002_04958_gb300 import inputs as I     # noqa: E402

OUT = os.path.join(HERE, "oracle_fgmres_G20_96x96x96_schur2.json")
N_SAMPLES = 256


def main():
    s = I.preset(3)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "schur2")
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert sto == 0
    rng = np.random.default_rng(3)
    idx = np.sort(np.concatenate([rng.choice(s.n, N_SAMPLES - 1, replace=False), [int(np.argmax(np.abs(xo)))]]))
    rec = {
        "workload": I.PRESET_NAMES[3], "n": int(s.n), "nnz": int(s.nnz), "tol": 1e-8,
        "iterations": int(ito), "relres": float(rro),
        "x_norm2": float(np.linalg.norm(xo)), "x_max_abs": float(np.abs(xo).max()),
        "sample_index": [int(i) for i in idx],
        "sample_x": [float(xo[i]) for i in idx],
        "written_by": "python tests/golden/make_oracle_fgmres_G20_96x96x96.py",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(OUT, ito, rro)


if __name__ == "__main__":
    main()
