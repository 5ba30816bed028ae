"""mgd_relres_noalloc: the residual check for callers that cannot allocate
device memory (an application allocator that owns the device, a fixed,
audited memory footprint).  Its result must equal the true relative
residual that mgd_solve reports, call after call, although its work space is
a fixed array inside the library instead of cudaMalloc'd memory.

Named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


def test_noalloc_relres_matches_solve_twice(lib):
    s = I.make_system(4, (61, 53), multigroup=True)       # n = 19398 (ragged)
    assert s.n <= lib.NOALLOC_MAX_N
    slv = lib.Solver().setup_system(s, "schur2")
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0
    dev = x.device
    rp = torch.from_numpy(s.rowptr).to(dev)
    ci = torch.from_numpy(s.col).to(dev)
    va = torch.from_numpy(s.val).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    outs = []
    for _ in range(2):
        out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
        assert lib.relres_noalloc(rp, ci, va, b, x, out) == 0
        outs.append(out.cpu().numpy())
    for o in outs:
        assert o[2] == pytest.approx(rr, rel=1e-10)
        assert o[1] == pytest.approx(np.linalg.norm(s.b), rel=1e-12)
        assert o[0] == pytest.approx(o[2] * o[1], rel=1e-14)
    assert np.array_equal(outs[0], outs[1])
    # the property the entry point exists for: after the first call on this
    # device (which may load the module), calls allocate no device memory
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    alloc0 = torch.cuda.memory_allocated(dev)
    out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
    for _ in range(5):
        assert lib.relres_noalloc(rp, ci, va, b, x, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert out[2].item() == pytest.approx(rr, rel=1e-10)
    # a different input right after: nothing of the previous call leaks in
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    assert lib.relres_noalloc(rp, ci, va, b, torch.zeros_like(x), out) == 0
    assert out[2].item() == pytest.approx(1.0, rel=1e-14)


def test_noalloc_rejects_oversize(lib):
    n = lib.NOALLOC_MAX_N + 1
    dev = torch.device("cuda")
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    v = torch.zeros(1, dtype=torch.float64, device=dev)
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    # the binding refuses before the call; the library itself refuses too
    with pytest.raises(ValueError, match="outside"):
        lib.relres_noalloc(rp, ci, v, b, b, out)
    import ctypes as C
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.lib().mgd_relres_noalloc(n, p(rp), p(ci), p(v), p(b), p(b), p(out),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
