"""Shared comparison of a GPU solution with the oracle's (test helper)."""
import numpy as np


def assert_x_close(xg, xo, rel=1e-10):
    """Relative 2-norm error and worst element both within `rel`: the
    element bound is |xg_i - xo_i| <= rel * max_k |xo_k| for every i."""
    xg = np.asarray(xg)
    xo = np.asarray(xo)
    assert xg.shape == xo.shape
    e2 = np.linalg.norm(xg - xo)
    assert e2 <= rel * np.linalg.norm(xo), ("2-norm", e2 / np.linalg.norm(xo))
    emax = np.abs(xg - xo).max() if xo.size else 0.0
    assert emax <= rel * np.abs(xo).max(), ("max-abs", emax / np.abs(xo).max(), int(np.argmax(np.abs(xg - xo))))
