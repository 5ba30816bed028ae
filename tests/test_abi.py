"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/mgdamg.h (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2002_04958_gb300 import build
    return build.build()


def _declared():
    with open(os.path.join(ROOT, "include", "mgdamg.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgd_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    names = _declared()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lib, nm), nm
    from paper_2002_04958_gb300 import mgdamg
    assert sorted(mgdamg.ENTRY_POINTS) == names


def test_opts_defaults_and_struct_layout(built):
    from paper_2002_04958_gb300 import mgdamg
    o = mgdamg.default_opts()
    assert o.theta_str == 0.25 and o.max_coarse == 100 and o.max_levels == 25
    assert o.theta_wd == 0.9 and o.theta_wc == 1e-2 and o.sigma_wc == 0.5 and o.inner_tol == 1e-2
    assert o.restart == 30 and o.nvcyc_group == 1 and o.precision == 0
    assert o.inner_mode == 0 and o.inner_maxit == 100
    # the ctypes mirror has the C struct's size: the library writes every field
    assert C.sizeof(mgdamg.MgdOpts) == 152 and C.sizeof(mgdamg.MgdStats) == 112
    assert o.opt4_steps == 0
    assert mgdamg.lib().mgd_kernel_launches() >= 0
    assert mgdamg.lib().mgd_opts_default(None) == 1


def test_no_cpu_fallback(built):
    import torch
    from paper_2002_04958_gb300 import mgdamg
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        mgdamg.Solver()


def test_struct_layout_matches_c_compiler(tmp_path):
    """Sizes and field offsets of the ctypes mirrors, as gcc lays out the header's structs."""
    import shutil
    import subprocess
    from paper_2002_04958_gb300 import mgdamg
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    fields = [f for f, _ in mgdamg.MgdOpts._fields_]
    sfields = [f for f, _ in mgdamg.MgdStats._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mgdamg.h"', 'int main(void) {',
             '  printf("%zu %zu\\n", sizeof(mgd_opts), sizeof(mgd_stats));']
    lines += [f'  printf("%zu\\n", offsetof(mgd_opts, {f}));' for f in fields]
    lines += [f'  printf("%zu\\n", offsetof(mgd_stats, {f}));' for f in sfields]
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == C.sizeof(mgdamg.MgdOpts) and vals[1] == C.sizeof(mgdamg.MgdStats)
    offs = vals[2:]
    for k, f in enumerate(fields):
        assert offs[k] == getattr(mgdamg.MgdOpts, f).offset, f
    for k, f in enumerate(sfields):
        assert offs[len(fields) + k] == getattr(mgdamg.MgdStats, f).offset, f


def test_relres_noalloc_binding_rejects_bad_arguments():
    """The allocation-free residual reads raw pointers without device-side
    checks; the binding rejects, before any library call, the mistakes that
    would make it read out of bounds."""
    torch = pytest.importorskip("torch")
    from paper_2002_04958_gb300 import mgdamg
    n = 8
    rp = torch.arange(n + 1, dtype=torch.int32)
    ci = torch.arange(n, dtype=torch.int32)
    v = torch.ones(n, dtype=torch.float64)
    b = torch.ones(n, dtype=torch.float64)
    x = torch.ones(n, dtype=torch.float64)
    out = torch.zeros(3, dtype=torch.float64)
    f = mgdamg.relres_noalloc
    with pytest.raises(TypeError, match="rowptr must be torch.int32"):
        f(rp.to(torch.int64), ci, v, b, x, out)          # torch.from_numpy of an int64 index array
    with pytest.raises(TypeError, match="col must be torch.int32"):
        f(rp, ci.to(torch.int64), v, b, x, out)
    with pytest.raises(TypeError, match="val must be torch.float64"):
        f(rp, ci, v.float(), b, x, out)
    with pytest.raises(TypeError, match="must be a torch.Tensor"):
        f(rp, ci, v, b.numpy(), x, out)
    with pytest.raises(ValueError, match="contiguous"):
        f(rp, ci, v, torch.ones(2 * n, dtype=torch.float64)[::2], x, out)
    with pytest.raises(ValueError, match="b and x need n"):
        f(rp, ci, v, b, torch.ones(n + 1, dtype=torch.float64), out)
    with pytest.raises(ValueError, match="out needs 3"):
        f(rp, ci, v, b, x, torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="outside"):
        f(torch.zeros(1, dtype=torch.int32), ci, v, b[:0], x[:0], out)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        f(rp, ci, v, b, x, out)                           # all host tensors
