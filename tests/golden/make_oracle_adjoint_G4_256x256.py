"""Writes oracle_adjoint_G4_256x256_amg.json: the FP64 oracle's forward and
adjoint solves on the four-group 256 x 256 system (393,216 unknowns, 2,354,176
nonzeros) with the monolithic classical-AMG preconditioner (one V(1,1) cycle,
l1-Jacobi smoothing, classical modified interpolation) inside right-
preconditioned FGMRES(30):

  * x = A^-1 b to 1e-8 (the iteration count the GPU must match) and to 1e-13;
  * the loss L = ||x||^2 of the 1e-13 solution, lambda = A^-T (2 x) to 1e-13
    (FGMRES preconditioned by the transposed V-cycle), and the value gradient
    dL/dA_ij = -lambda_i x_j over A's pattern (dL/db = lambda);
  * seeded samples of x, lambda and the gradient, their norms and largest
    entries.

It calls only the oracle (a few minutes on one host core); the GPU adjoint
test compares against these figures.

    python tests/golden/make_oracle_adjoint_G4_256x256.py
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

OUT = os.path.join(HERE, "oracle_adjoint_G4_256x256_amg.json")
N_SAMPLES = 256


def _samples(rng, v):
    idx = np.sort(np.concatenate([rng.choice(v.size, N_SAMPLES - 1, replace=False), [int(np.argmax(np.abs(v)))]]))
    return [int(i) for i in idx], [float(v[i]) for i in idx]


def main():
    s = I.preset(4)
    Ao = orc.csr_of_system(s)
    t0 = time.perf_counter()
    M = orc.Block(Ao, s.G, s.N, "amg")
    x8, it8, rr8, st8, _ = orc.fgmres(Ao, s.b, M, tol=1e-8)
    assert st8 == 0
    x, it, rr, st, _ = orc.fgmres(Ao, s.b, M, tol=1e-13, maxit=6000)
    assert st == 0
    lam, itT, rrT, stT, _ = orc.fgmres(Ao, 2.0 * x, M, tol=1e-13, maxit=6000, transpose=True)
    assert stT == 0
    g = orc.grad_vals(Ao, x, lam)
    t1 = time.perf_counter()
    rng = np.random.default_rng(17)
    xi, xs = _samples(rng, x)
    li, ls = _samples(rng, lam)
    gi, gs = _samples(rng, g)
    rec = {
        "workload": I.PRESET_NAMES[4], "n": int(s.n), "nnz": int(s.nnz), "precond": "amg",
        "iterations_tol_1e-8": int(it8), "relres_tol_1e-8": float(rr8),
        "iterations_tol_1e-13": int(it), "relres_tol_1e-13": float(rr),
        "iterations_transpose_tol_1e-13": int(itT), "relres_transpose_tol_1e-13": float(rrT),
        "loss": float(np.dot(x, x)),
        "x_norm2": float(np.linalg.norm(x)), "x_max_abs": float(np.abs(x).max()),
        "lambda_norm2": float(np.linalg.norm(lam)), "lambda_max_abs": float(np.abs(lam).max()),
        "grad_norm2": float(np.linalg.norm(g)), "grad_max_abs": float(np.abs(g).max()),
        "x_index": xi, "x_sample": xs, "lambda_index": li, "lambda_sample": ls,
        "grad_index": gi, "grad_sample": gs,
        "written_by": "python tests/golden/make_oracle_adjoint_G4_256x256.py",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(OUT, it8, it, itT, f"{t1 - t0:.1f} s")


if __name__ == "__main__":
    main()
