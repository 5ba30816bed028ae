"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bar (FP64 mode): C/F splittings, coarse patterns, interpolation and coarse
values bit-exact (the setup kernels round every step as the oracle does);
FGMRES iteration counts equal; solution values within 1e-10 relative.
FP32 V-cycle mode: iteration counts within +-1 of the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KIND_NAMES = ["amg", "pctl", "schur1", "schur2", "bd", "blt"]

CASES = [
    # (G, dims, multigroup, inclusion) -- ragged sizes that span many 256-row tiles
    (1, (45, 37), False, False),
    (1, (40, 40), False, True),
    (4, (29, 23), True, False),
    (20, (13, 11), True, False),
    (2, (9, 8, 7), True, False),
]


def _system(case, seed=0):
    G, dims, mg, inc = case
    return I.make_system(G, dims, seed=seed, multigroup=mg, inclusion=inc)


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


def _oracle_hierarchy(orc, ob, kind, op_kind, comp):
    if kind == "amg":
        return ob.amg(orc.OP_MONO, 0)
    return ob.amg(op_kind, comp)


def _compare_hierarchy(slv, op, oh):
    info = slv.op_info(op)
    assert info["nlevels"] == oh.nlevels, (info, oh.nlevels)
    assert bool(info["coarse_lu"]) == oh.coarse_is_lu
    for l in range(oh.nlevels):
        g = slv.level(op, l)
        rp, ci, v = oh.A(l).arrays()
        assert np.array_equal(g["rp"], rp), f"level {l} rowptr"
        assert np.array_equal(g["ci"], ci), f"level {l} columns"
        assert np.array_equal(g["v"], v), f"level {l} values differ (max {abs(g['v'] - v).max():.3e})"
        if l < oh.nlevels - 1:
            assert np.array_equal(g["cf"], oh.CF(l)), f"level {l} C/F"
            prp, pci, pv = oh.P(l).arrays()
            assert np.array_equal(g["prp"], prp) and np.array_equal(g["pci"], pci), f"level {l} P pattern"
            assert np.array_equal(g["pv"], pv), f"level {l} P values"


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"G{c[0]}_{'x'.join(map(str, c[1]))}{'_inc' if c[3] else ''}")
@pytest.mark.parametrize("kind", KIND_NAMES)
def test_setup_bit_exact(gpu, orc, case, kind):
    s = _system(case)
    slv = gpu.Solver().setup_system(s, kind)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind)
    st = slv.stats()
    ops = [slv.op_info(k) for k in range(st["n_ops"])]
    for k, info in enumerate(ops):
        if kind == "pctl" and info["kind"] == 5:
            continue  # A_c depends on the iterative p_a: compared by value below
        if info["use_jacobi"]:
            continue
        oh = _oracle_hierarchy(orc, ob, kind, info["kind"], info["comp"])
        _compare_hierarchy(slv, k, oh)
    if kind == "pctl":
        for a in range(s.nc):
            if a == s.G:
                continue
            pg = slv.block_vector(0, a)
            po = ob.vec(0, a)
            assert np.allclose(pg, po, rtol=1e-10, atol=1e-12 * abs(po).max())


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"G{c[0]}_{'x'.join(map(str, c[1]))}{'_inc' if c[3] else ''}")
@pytest.mark.parametrize("kind", KIND_NAMES)
def test_solve_parity_fp64(gpu, orc, case, kind):
    s = _system(case)
    slv = gpu.Solver().setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind), tol=1e-8, maxit=1000)
    assert sto == 0 and rc == 0
    assert it == ito, (it, ito)
    xg = x.cpu().numpy()
    assert_x_close(xg, xo)
    # independent residual check in FP64 on the host
    A = s.scipy()
    assert np.linalg.norm(s.b - A @ xg) <= 1e-8 * np.linalg.norm(s.b) * (1 + 1e-6)


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4]], ids=["G1", "G4", "G2_3d"])
@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "pctl"])
def test_exti_setup_bit_exact_and_solve(gpu, orc, case, kind):
    # extended+i interpolation: hierarchies bit-exact, iteration counts equal
    s = _system(case)
    slv = gpu.Solver(interp_type=1).setup_system(s, kind)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(interp_type=1))
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        if info["use_jacobi"] or (kind == "pctl" and info["kind"] == 5):
            continue
        _compare_hierarchy(slv, k, _oracle_hierarchy(orc, ob, kind, info["kind"], info["comp"]))
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert rc == 0 and sto == 0 and it == ito
    assert_x_close(x.cpu().numpy(), xo)


@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "bd"])
def test_precond_apply_matches_oracle(gpu, orc, kind):
    s = _system(CASES[2])
    slv = gpu.Solver().setup_system(s, kind)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(s.n)
    z = slv.precond_apply(torch.from_numpy(v)).cpu().numpy()
    Ao = orc.csr_of_system(s)
    zo = orc.Block(Ao, s.G, s.N, kind).apply(v)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "bd", "pctl"])
def test_fp32_vcycle_iterations(gpu, orc, kind):
    s = _system(CASES[2])
    slv = gpu.Solver(precision=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    _, ito, _, _, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind), tol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    xg = x.cpu().numpy()
    assert np.linalg.norm(s.b - s.scipy() @ xg) <= 1.0000001e-8 * np.linalg.norm(s.b)


@pytest.mark.parametrize("kind", ["bd", "schur2", "schur1", "blt"])
def test_batched_and_graph_identical(gpu, kind):
    s = _system(CASES[3])
    b = torch.from_numpy(s.b)
    ref = gpu.Solver(autotune=0).setup_system(s, kind)
    xr, itr, _, _ = ref.solve(b)
    for opts in [dict(batched=1), dict(use_graph=1), dict(batched=1, use_graph=1),
                 dict(batched=1, use_graph=1, pdl=0), dict(pdl=0)]:
        slv = gpu.Solver(autotune=0, **opts).setup_system(s, kind)
        x, it, _, _ = slv.solve(b)
        assert it == itr
        assert torch.equal(x, xr), opts


@pytest.mark.parametrize("kind,prec", [("amg", 0), ("schur1", 0), ("schur2", 1), ("bd", 0)])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[4]], ids=["G1", "G20", "G2_3d"])
def test_fused_coarse_levels(gpu, orc, kind, prec, case):
    # every level below level 0 in the cluster kernel vs per-level launches
    s = _system(case)
    v = torch.from_numpy(np.random.default_rng(7).standard_normal(s.n))
    ref = gpu.Solver(autotune=0, precision=prec, fuse_rows=-1, batched=1).setup_system(s, kind)
    fus = gpu.Solver(autotune=0, precision=prec, fuse_rows=1 << 30, batched=1, use_graph=1).setup_system(s, kind)
    assert all(b["tail"] == 1 for b in fus.plan() if b["depth"] > 1)
    z0 = ref.precond_apply(v).cpu().numpy()
    z1 = fus.precond_apply(v).cpu().numpy()
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.linalg.norm(z1 - z0) <= tol * np.linalg.norm(z0)
    if prec == 0:
        Ao = orc.csr_of_system(s)
        zo = orc.Block(Ao, s.G, s.N, kind).apply(v.numpy())
        assert np.linalg.norm(z1 - zo) <= 1e-12 * np.linalg.norm(zo)
    x1, it1, rr1, _ = fus.solve(torch.from_numpy(s.b))
    x0, it0, rr0, _ = ref.solve(torch.from_numpy(s.b))
    assert abs(it1 - it0) <= (0 if prec == 0 else 1) and rr1 <= 1e-8


def test_fused_coarse_levels_transposed(gpu):
    s = _system(CASES[2])
    ref = gpu.Solver(autotune=0, keep_transpose=1, fuse_rows=-1).setup_system(s, "amg")
    fus = gpu.Solver(autotune=0, keep_transpose=1, fuse_rows=1 << 30).setup_system(s, "amg")
    g = torch.from_numpy(np.random.default_rng(8).standard_normal(s.n))
    l0, it0, _ = ref.solve_transpose(g)
    l1, it1, _ = fus.solve_transpose(g)
    assert it0 == it1
    assert torch.linalg.vector_norm(l1 - l0) <= 1e-10 * torch.linalg.vector_norm(l0)


def test_adaptive_drops_match_oracle(gpu, orc):
    s = _system(CASES[2])
    for kind in ["schur1", "schur2", "pctl"]:
        slv = gpu.Solver(adaptive=1).setup_system(s, kind)
        Ao = orc.csr_of_system(s)
        ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(adaptive=1))
        for a in range(s.nc):
            for b in range(s.nc):
                assert slv.coupling_dropped(a, b) == ob.dropped(a, b)
        x, it, rr, rc = slv.solve(torch.from_numpy(s.b), allow_noconv=True)
        _, ito, _, _, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
        assert it == ito


def test_edge_cases(gpu):
    from paper_2002_04958_gb300.mgdamg import MgdError
    s = I.make_system(1, (1, 1))   # one cell: coarsest immediately
    slv = gpu.Solver().setup_system(s, "amg")
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b))
    assert it == 1 and rr <= 1e-12
    s = I.make_system(1, (7, 5))
    slv = gpu.Solver().setup_system(s, "schur1")
    x, it, rr, rc = slv.solve(torch.zeros(s.n, dtype=torch.float64))
    assert it == 0 and not x.any()
    x, it, rr, rc = gpu.Solver(max_it=2).setup_system(s, "amg").solve(torch.from_numpy(s.b), tol=1e-14,
                                                                        allow_noconv=True)
    assert rc == 2 and it == 2
    # invalid inputs are rejected before any kernel touches them
    bad = s.col.copy()
    r0 = s.rowptr[5]
    bad[r0], bad[r0 + 1] = bad[r0 + 1], bad[r0]
    with pytest.raises(MgdError) as e:
        gpu.Solver().setup(s.G, s.N, torch.from_numpy(s.rowptr), torch.from_numpy(bad), torch.from_numpy(s.val),
                           "amg")
    assert e.value.code == 1
    badv = s.val.copy()
    d = [p for p in range(s.rowptr[3], s.rowptr[4]) if s.col[p] == 3][0]
    badv[d] = -1.0
    with pytest.raises(MgdError):
        gpu.Solver().setup(s.G, s.N, torch.from_numpy(s.rowptr), torch.from_numpy(s.col), torch.from_numpy(badv),
                           "amg")
    badc = s.col.copy()
    row = 2 * s.N   # first ion row: its coupling must sit in cell 0
    p = [q for q in range(s.rowptr[row], s.rowptr[row + 1]) if s.col[q] // s.N == 1][0]
    badc[p] = s.N + 1
    badc_sorted = badc  # still sorted within the row (E block precedes the I block)
    with pytest.raises(MgdError):
        gpu.Solver().setup(s.G, s.N, torch.from_numpy(s.rowptr), torch.from_numpy(badc_sorted),
                           torch.from_numpy(s.val), "bd")
    # row pointers: last entry short of nnz, and a decreasing pair (every
    # entry the validation reads stays inside the arrays)
    for k in ["short", "decreasing"]:
        badr = s.rowptr.copy()
        if k == "short":
            badr[-1] -= 1
        else:
            badr[5], badr[6] = badr[6], badr[5]
        with pytest.raises(MgdError) as e:
            gpu.Solver().setup(s.G, s.N, torch.from_numpy(badr), torch.from_numpy(s.col), torch.from_numpy(s.val),
                               "amg")
        assert e.value.code == 1 and "row pointer" in str(e.value), k


@pytest.mark.parametrize("kind", ["amg", "schur2"])
def test_setup_from_host_buffers(gpu, kind):
    # mgd_setup_host (chunked copies over several streams) sets up exactly what
    # mgd_setup does from device arrays: same hierarchy, same solution bits;
    # pageable numpy arrays and page-locked tensors both work
    s = _system(CASES[3])
    dev = gpu.Solver().setup_system(s, kind)
    xd, itd, _, _ = dev.solve(torch.from_numpy(s.b))
    for pinned in (False, True):
        if pinned:
            rp, ci, va = (torch.from_numpy(a).pin_memory() for a in (s.rowptr, s.col, s.val))
        else:
            rp, ci, va = s.rowptr, s.col, s.val
        hs = gpu.Solver().setup_host(s.G, s.N, rp, ci, va, kind)
        xh, ith, _, _ = hs.solve(torch.from_numpy(s.b))
        assert ith == itd and torch.equal(xh, xd)
        for k in range(dev.stats()["n_ops"]):
            a, b = dev.level(k, 0), hs.level(k, 0)
            assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["ci"], b["ci"])
    with pytest.raises(gpu.MgdError) as e:
        gpu.Solver().setup_host(s.G, s.N + 1, s.rowptr, s.col, s.val, kind)
    assert e.value.code == 1


def test_solve_host_buffers(gpu, orc):
    s = _system(CASES[0])
    slv = gpu.Solver().setup_system(s, "schur2")
    x, it, rr = slv.solve_host(s.b)
    xd, itd, _, _ = slv.solve(torch.from_numpy(s.b))
    assert it == itd and np.array_equal(x, xd.cpu().numpy())


@pytest.mark.parametrize("smoother", [0, 1], ids=["l1jacobi", "cf_gauss_seidel"])
def test_adjoint_gradient(gpu, orc, smoother):
    s = I.make_system(4, (12, 10), multigroup=True)
    slv = gpu.Solver(keep_transpose=1, smoother=smoother).setup_system(s, "amg")
    vals = torch.from_numpy(s.val).cuda().requires_grad_(True)
    b = torch.from_numpy(s.b).cuda().requires_grad_(True)
    x = gpu.mgd_solve(vals, b, slv, 1e-13)
    loss = (x * x).sum()
    loss.backward()
    # oracle gradient
    Ao = orc.csr_of_system(s)
    M = orc.Block(Ao, s.G, s.N, "amg", orc.opts(smoother=smoother))
    xo, *_ = orc.fgmres(Ao, s.b, M, tol=1e-14, maxit=2000)
    lo, *_ = orc.fgmres(Ao, 2 * xo, M, tol=1e-14, maxit=2000, transpose=True)
    go = orc.grad_vals(Ao, xo, lo)
    gv = vals.grad.cpu().numpy()
    assert np.linalg.norm(gv - go) <= 1e-8 * np.linalg.norm(go)
    assert np.linalg.norm(b.grad.cpu().numpy() - lo) <= 1e-8 * np.linalg.norm(lo)
    # central differences on relative perturbations of the values
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(s.nnz)
        d /= np.linalg.norm(d)
        dv = torch.from_numpy(s.val * d).cuda()
        lp = gpu.mgd_solve(vals.detach() + h * dv, b.detach(), slv, 1e-13)
        lm = gpu.mgd_solve(vals.detach() - h * dv, b.detach(), slv, 1e-13)
        fd = ((lp * lp).sum() - (lm * lm).sum()).item() / (2 * h)
        an = (vals.grad * dv).sum().item()
        assert fd == pytest.approx(an, rel=1e-5)


@pytest.mark.parametrize("kind", ["amg", "bd"])
@pytest.mark.parametrize("batched", [0, 1])
def test_fp32_vcycle_transposed_solve(gpu, orc, kind, batched):
    # A^T lam = g with the transposed FP32 V-cycles (the FP32 copies of A^T and
    # of A^T D^-1): iterations within one of the FP64 oracle's transposed
    # solve, the true transposed residual below the tolerance
    s = I.make_system(4, (23, 19), multigroup=True)
    slv = gpu.Solver(keep_transpose=1, precision=1, batched=batched, use_graph=batched).setup_system(s, kind)
    g = np.random.default_rng(3).standard_normal(s.n)
    lam, it, rr = slv.solve_transpose(torch.from_numpy(g), tol=1e-8)
    Ao = orc.csr_of_system(s)
    lo, ito, *_ = orc.fgmres(Ao, g, orc.Block(Ao, s.G, s.N, kind), tol=1e-8, transpose=True)
    assert abs(it - ito) <= 1, (it, ito)
    lg = lam.cpu().numpy()
    assert np.linalg.norm(g - s.scipy().T @ lg) <= 1.0000001e-8 * np.linalg.norm(g)
    # both residuals are below 1e-8 ||g|| and cond(A) is about 4.5e3 here
    assert np.linalg.norm(lg - lo) <= 2e-4 * np.linalg.norm(lo)


@pytest.mark.parametrize("kind", ["amg", "schur1", "bd"])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[4]], ids=["G1", "G20", "G2_3d"])
def test_resident_arnoldi_matches_streaming(gpu, orc, kind, case):
    # the cooperative orthogonalisation (w in shared memory) and the streaming
    # kernels run the same modified Gram-Schmidt: same iterations, same x to rounding
    s = _system(case)
    b = torch.from_numpy(s.b)
    xs, its, _, _ = gpu.Solver(arnoldi_resident=0).setup_system(s, kind).solve(b, tol=1e-8)
    slv = gpu.Solver(arnoldi_resident=1).setup_system(s, kind)
    xr, itr, rr, rc = slv.solve(b, tol=1e-8)
    assert rc == 0 and itr == its
    assert torch.linalg.vector_norm(xr - xs) <= 1e-10 * torch.linalg.vector_norm(xs)
    Ao = orc.csr_of_system(s)
    _, ito, _, _, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind), tol=1e-8)
    assert itr == ito
    x2, it2, _, _ = slv.solve(b, tol=1e-8)      # run to run: the same bits
    assert it2 == itr and torch.equal(x2, xr)


@pytest.mark.parametrize("opts", [dict(), dict(batched=1, use_graph=1)], ids=["eager", "graph"])
def test_precond_bench_matches_apply(gpu, opts):
    s = _system(CASES[3])
    slv = gpu.Solver(**opts).setup_system(s, "bd")
    v = torch.from_numpy(np.random.default_rng(9).standard_normal(s.n))
    z = slv.precond_apply(v)
    ms, by = slv.precond_bench(v, 20)
    assert ms > 0 and by == pytest.approx(slv.stats()["precond_bytes"])
    z2 = slv.precond_apply(v)   # the repeated applies left the solver as it was
    assert torch.equal(z, z2)
    with pytest.raises(gpu.MgdError):
        slv.precond_bench(v, 0)


_PLAN_SCRIPT = """
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2002_04958_gb300 import inputs, mgdamg
s = inputs.make_system(2, (37, 29), multigroup=True)
slv = mgdamg.Solver(autotune=1, batched=1, use_graph=1).setup_system(s, "schur2")
print(json.dumps(slv.plan()))
"""


def test_tune_cache_file(gpu, tmp_path):
    # autotuner decisions written by one process are read back by another,
    # which then runs the same plan; lines that do not parse are skipped
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.txt"
    env = dict(os.environ, MGD_TUNE_CACHE=str(path))

    def run():
        p = subprocess.run([sys.executable, "-c", _PLAN_SCRIPT, root], env=env, capture_output=True, text=True,
                           timeout=600)
        assert p.returncode == 0, p.stderr[-2000:]
        return json.loads(p.stdout.strip().splitlines()[-1])

    first = run()
    lines = path.read_text().splitlines()
    assert lines and all(len(ln.split("|")) == 6 for ln in lines)
    path.write_text("not a cache line\n" + "\n".join(lines) + "\n")
    second = run()
    assert second == first


_LAYOUT_SCRIPT = """
import hashlib, json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_2002_04958_gb300 import inputs, mgdamg
out = {}
for name, G, dims, kind, prec in [("G20_schur2", 20, (37, 29), "schur2", 0), ("G20_bd", 20, (37, 29), "bd", 0),
                                  ("G2_3d_amg", 2, (13, 11, 9), "amg", 0), ("G20_schur2_fp32", 20, (37, 29), "schur2", 1),
                                  ("G4_bd_fp32", 4, (41, 23), "bd", 1)]:
    s = inputs.make_system(G, dims, multigroup=True)
    trans = kind in ("amg", "bd")  # the transposed solve takes AMG or BD
    slv = mgdamg.Solver(autotune=1, batched=1, use_graph=1, keep_transpose=int(trans),
                        precision=prec).setup_system(s, kind)
    b = torch.from_numpy(s.b)
    x, it, rr, rc = slv.solve(b)
    lam, itT, _ = slv.solve_transpose(b) if trans else (x, 0, 0.0)   # raises unless it converged
    rcT = 0
    out[name] = dict(plan=slv.plan(), it=it, itT=itT, rc=[rc, rcT],
                     x=hashlib.sha256(x.cpu().numpy().tobytes()).hexdigest(),
                     lam=hashlib.sha256(lam.cpu().numpy().tobytes()).hexdigest())
print(json.dumps(out))
"""


def test_transfer_layouts_bit_identical(gpu, tmp_path):
    # the multi-row restriction / prolongation layouts (9, 10) sum each row as
    # the one-thread-per-row layout (1) does: with every level's transfer
    # layouts forced through the tune cache, forward and transposed solves are
    # bitwise identical across the three
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.txt"
    env = dict(os.environ, MGD_TUNE_CACHE=str(path))

    def run():
        p = subprocess.run([sys.executable, "-c", _LAYOUT_SCRIPT, root], env=env, capture_output=True, text=True,
                           timeout=900)
        assert p.returncode == 0, p.stderr[-2000:]
        return json.loads(p.stdout.strip().splitlines()[-1])

    run()   # writes the autotuned entries
    lines = path.read_text().splitlines()
    res = {}
    for f in (1, 9, 10):
        forced = []
        for ln in lines:
            fs = ln.split("|")
            depth = len(fs[1].split())
            fs[2] = fs[3] = " ".join([str(f)] * depth)
            forced.append("|".join(fs))
        path.write_text("\n".join(forced) + "\n")
        res[f] = run()
        for name, r in res[f].items():
            assert r["rc"] == [0, 0], (f, name)
            for batch in r["plan"]:
                for lv in batch["levels"][:-1]:
                    if lv["nsub"]:
                        assert lv["fmtR"] == f and lv["fmtP"] == f, (f, name, lv)
    for f in (9, 10):
        for name in res[1]:
            for k in ("it", "itT", "x", "lam"):
                assert res[f][name][k] == res[1][name][k], (f, name, k)


def test_format_conversions_match_hardware(gpu):
    # the block updates of the FP32-V-cycle form convert on the integer pipe;
    # every binary32 pattern, every binary32 tie and its binary64 neighbours
    assert gpu.check_conversions() == 0


def test_fp64_accounting_and_issue_rate(gpu):
    # the FP64 roofline inputs: a measured device rate and the algorithmic FP64
    # lane operations of the level-0 l1-Jacobi kernels (none in FP32 V-cycles)
    rate = gpu.fp64_issue_rate()
    assert 1e10 < rate < 1e14
    s = _system(CASES[2])
    b = torch.from_numpy(s.b)
    for prec in (0, 1):
        slv = gpu.Solver(precision=prec, batched=1).setup_system(s, "bd")
        slv.profile(1)
        slv.solve(b)
        n0, _, _ = slv.profile_read(0)
        f0 = slv.profile_read_fp64(0)
        slv.profile(0)
        assert n0 > 0
        if prec == 1:
            assert f0 == 0.0
        else:
            # one V-cycle per subsystem and apply: k_pre + k_post at level 0,
            # (nnz + 2 n) lane operations each; a one-level hierarchy with a
            # Jacobi coarsest solve (nnz + 3 n); Jacobi inverses and dense
            # coarsest solves none
            per_apply = 0.0
            for k in range(slv.stats()["n_ops"]):
                info = slv.op_info(k)
                if info["use_jacobi"]:
                    continue
                li = slv.level_info(k, 0)
                if info["nlevels"] > 1:
                    per_apply += 2.0 * (li["nnz"] + 2.0 * li["n"])
                elif not info["coarse_lu"]:
                    per_apply += li["nnz"] + 3.0 * li["n"]
            assert per_apply > 0
            assert f0 == pytest.approx(slv.stats()["last_iters"] * per_apply, rel=1e-12)
