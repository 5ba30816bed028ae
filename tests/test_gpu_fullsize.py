"""Parity at the full workload sizes, in the launch configuration the bench
uses (autotuned layouts): the C/F splittings, interpolation and coarse
operators of every hierarchy bit-exact with the oracle, the FGMRES iteration
count of the FP64 solve equal to the oracle's (configs 2 and 3; for the 3D
system the oracle's solve is stored under golden/), the FP32-V-cycle count
within +-1, and the true residual checked independently on the host."""
import json
import os

import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


def _compare_all_levels(slv, ob, orc, kind, max_level=None):
    st = slv.stats()
    checked = 0
    for k in range(st["n_ops"]):
        info = slv.op_info(k)
        if info["use_jacobi"]:
            continue
        oh = ob.amg(orc.OP_MONO, 0) if kind == "amg" else ob.amg(info["kind"], info["comp"])
        assert info["nlevels"] == oh.nlevels
        L = oh.nlevels if max_level is None else min(oh.nlevels, max_level + 1)
        for l in range(L):
            g = slv.level(k, l)
            rp, ci, v = oh.A(l).arrays()
            assert np.array_equal(g["rp"], rp) and np.array_equal(g["ci"], ci) and np.array_equal(g["v"], v)
            if l < oh.nlevels - 1:
                assert np.array_equal(g["cf"], oh.CF(l))
                prp, pci, pv = oh.P(l).arrays()
                assert np.array_equal(g["prp"], prp) and np.array_equal(g["pci"], pci) and np.array_equal(g["pv"], pv)
            checked += 1
    return checked


def test_config1_full_size_hierarchies_and_residual(gpu, orc):
    s = I.preset(1)                      # 1024 x 1024, 3,145,728 unknowns
    slv = gpu.Solver().setup_system(s, "schur1")
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "schur1")
    assert _compare_all_levels(slv, ob, orc, "schur1") >= 10
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0
    xg = x.cpu().numpy()
    res = np.linalg.norm(s.b - s.scipy() @ xg) / np.linalg.norm(s.b)
    assert res <= 1e-8 * (1 + 1e-6) and res == pytest.approx(rr, rel=1e-6)
    # sampled rows of the preconditioner output against the oracle's full apply
    v = np.random.default_rng(1).standard_normal(s.n)
    z = slv.precond_apply(torch.from_numpy(v)).cpu().numpy()
    zo = ob.apply(v)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)


def _golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def test_config1_bench_workload_schur1_exti(gpu, orc):
    """The one-group benchmark workload as the bench runs it (Schur1, extended+i
    interpolation, batched launches, graph replay, autotuned layouts): every
    hierarchy bit-exact, the FP64 iteration count equal to the stored oracle
    solve's, and the whole solution within 1e-10 of a fresh oracle solve,
    element by element; the FP32-V-cycle form within +-1 iteration, its final
    error against the oracle bounded."""
    rec = _golden("oracle_fgmres_G1_1024x1024_schur1_exti.json")
    s = I.preset(1)
    assert s.n == rec["n"] and s.nnz == rec["nnz"]
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "schur1", orc.opts(interp_type=1))
    slv = gpu.Solver(interp_type=1, batched=1, use_graph=1, autotune=1).setup_system(s, "schur1")
    assert _compare_all_levels(slv, ob, orc, "schur1") >= 10
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0 and it == rec["iterations"], (it, rec["iterations"])
    assert rr == pytest.approx(rec["relres"], rel=1e-5)
    xg = x.cpu().numpy()
    idx = np.asarray(rec["sample_index"])
    assert np.max(np.abs(xg[idx] - np.asarray(rec["sample_x"]))) <= 1e-10 * rec["x_max_abs"]
    assert abs(np.linalg.norm(xg) - rec["x_norm2"]) <= 1e-10 * rec["x_norm2"]
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert sto == 0 and ito == rec["iterations"]
    assert_x_close(xg, xo)
    mixed = gpu.Solver(precision=1, interp_type=1, batched=1, use_graph=1, autotune=1).setup_system(s, "schur1")
    xm, itm, rrm, rcm = mixed.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rcm == 0 and abs(itm - ito) <= 1
    xmn = xm.cpu().numpy()
    assert np.linalg.norm(s.b - s.scipy() @ xmn) <= 1.0000001e-8 * np.linalg.norm(s.b)
    assert np.abs(xmn - xo).max() <= 1e-6 * np.abs(xo).max()


def test_config2_full_size_iterations(gpu, orc):
    s = I.preset(2)                      # G = 20, 256 x 256, 1,441,792 unknowns
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "bd")
    slv = gpu.Solver(batched=1).setup_system(s, "bd")
    assert _compare_all_levels(slv, ob, orc, "bd") >= 22
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert rc == 0 and sto == 0 and it == ito
    xg = x.cpu().numpy()
    assert_x_close(xg, xo)
    mixed = gpu.Solver(precision=1, batched=1, use_graph=1).setup_system(s, "bd")
    xm, itm, rrm, rcm = mixed.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rcm == 0 and abs(itm - ito) <= 1
    assert np.linalg.norm(s.b - s.scipy() @ xm.cpu().numpy()) <= 1.0000001e-8 * np.linalg.norm(s.b)


def test_config3_full_size_hierarchies_iterations_residual(gpu, orc):
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_fgmres_G20_96x96x96_schur2.json")) as f:
        rec = json.load(f)
    s = I.preset(3)                      # G = 20, 96 x 96 x 96, 19,464,192 unknowns
    assert s.n == rec["n"] and s.nnz == rec["nnz"]
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "schur2")
    exact = gpu.Solver(batched=1, use_graph=1, autotune=1).setup_system(s, "schur2")
    assert _compare_all_levels(exact, ob, orc, "schur2") >= 22 * 5
    v = np.random.default_rng(2).standard_normal(s.n)
    z = exact.precond_apply(torch.from_numpy(v)).cpu().numpy()
    zo = ob.apply(v)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    del ob, Ao
    x, it, rr, rc = exact.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0 and it == rec["iterations"] and rr == pytest.approx(rec["relres"], rel=1e-5)
    xg = x.cpu().numpy()
    assert abs(np.linalg.norm(xg) - rec["x_norm2"]) <= 1e-10 * rec["x_norm2"]
    idx = np.asarray(rec["sample_index"])
    assert np.max(np.abs(xg[idx] - np.asarray(rec["sample_x"]))) <= 1e-10 * rec["x_max_abs"]
    assert abs(np.abs(xg).max() - rec["x_max_abs"]) <= 1e-10 * rec["x_max_abs"]
    del exact, x
    # the bench's launch configuration: FP32 V-cycles inside the FP64 FGMRES
    mixed = gpu.Solver(precision=1, batched=1, use_graph=1, autotune=1).setup_system(s, "schur2")
    xm, itm, rrm, rcm = mixed.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rcm == 0 and abs(itm - rec["iterations"]) <= 1
    xmn = xm.cpu().numpy()
    res = np.linalg.norm(s.b - s.scipy() @ xmn) / np.linalg.norm(s.b)
    assert res <= 1.0000001e-8 and res == pytest.approx(rrm, rel=1e-6)
    # final error of the mixed form against the FP64 oracle, on the stored entries
    assert np.max(np.abs(xmn[idx] - np.asarray(rec["sample_x"]))) <= 1e-6 * rec["x_max_abs"]


def test_config4_adjoint_full_size(gpu):
    """The adjoint workload at its stated size: G = 4 on 256 x 256, monolithic
    AMG, L = ||x||^2.  The forward iteration count at 1e-8 equals the stored
    oracle solve's; x, lambda = dL/db and dL/dvals from the torch.autograd
    Function (backward: FGMRES with the transposed V-cycle) match the stored
    oracle values; central differences (h = 1e-6, relative perturbations
    vals (.) (1 +- h d) along 32 seeded unit directions d ~ N(0, 1) / ||.||)
    match the analytic directional derivative to 1e-5."""
    rec = _golden("oracle_adjoint_G4_256x256_amg.json")
    s = I.preset(4)
    assert s.n == rec["n"] and s.nnz == rec["nnz"]
    slv = gpu.Solver(keep_transpose=1, max_it=6000, batched=1, use_graph=1).setup_system(s, "amg")
    x8, it8, rr8, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0 and it8 == rec["iterations_tol_1e-8"], (it8, rec["iterations_tol_1e-8"])
    vals = torch.from_numpy(s.val).cuda().requires_grad_(True)
    b = torch.from_numpy(s.b).cuda().requires_grad_(True)
    x = gpu.mgd_solve(vals, b, slv, 1e-13)
    loss = (x * x).sum()
    loss.backward()
    # at 1e-13, near the attainable accuracy, the count depends on the rounding
    # of the layouts the autotuner picked (CSR with several threads per row sums
    # in another order); the parity bar is the 1e-8 count above
    st = slv.stats()
    assert abs(st["last_iters"] - rec["iterations_transpose_tol_1e-13"]) <= 0.05 * rec["iterations_transpose_tol_1e-13"]
    assert loss.item() == pytest.approx(rec["loss"], rel=1e-9)

    def close(v, idx, smp, vmax, vnorm, rel):
        v = v.detach().cpu().numpy()
        assert np.max(np.abs(v[np.asarray(idx)] - np.asarray(smp))) <= rel * vmax
        assert abs(np.linalg.norm(v) - vnorm) <= rel * vnorm
        assert abs(np.abs(v).max() - vmax) <= rel * vmax

    close(x, rec["x_index"], rec["x_sample"], rec["x_max_abs"], rec["x_norm2"], 1e-9)
    close(b.grad, rec["lambda_index"], rec["lambda_sample"], rec["lambda_max_abs"], rec["lambda_norm2"], 1e-8)
    close(vals.grad, rec["grad_index"], rec["grad_sample"], rec["grad_max_abs"], rec["grad_norm2"], 1e-8)
    # L(+) - L(-) = (x+ - x-) . (x+ + x-).  Along a unit direction the values
    # move by ~1e-9 relative, so L changes by ~1e-12 of itself: two separate
    # solves to 1e-13 would differ by their solve errors more than by that.
    # Instead x- is solved to 1e-13 and the difference from its own system,
    # A+ (x+ - x-) = -(A+ - A-) x-, whose right-hand side is a product with
    # 2 h vals (.) d (no cancellation): x+ = x- + (x+ - x-) then solves
    # A+ x+ = A- x-, i.e. both points see the same right-hand side b - r(x-),
    # which moves L's derivative by a relative kappa * 1e-13 only.
    import scipy.sparse as sp
    fds = gpu.Solver(max_it=6000, batched=1, use_graph=1).setup_system(s, "amg")
    rng = np.random.default_rng(0)
    h = 1e-6
    gv = vals.grad.detach()
    for _ in range(32):
        d = rng.standard_normal(s.nnz)
        d /= np.linalg.norm(d)
        dvn = s.val * d
        dv = torch.from_numpy(dvn).cuda()
        fds.update_values(vals.detach() - h * dv)
        xm, _, _, rcm = fds.solve(b.detach(), tol=1e-13)
        xmn = xm.cpu().numpy()
        rhs = -(sp.csr_matrix((2 * h * dvn, s.col, s.rowptr), shape=(s.n, s.n)) @ xmn)
        fds.update_values(vals.detach() + h * dv)
        dl, _, _, rcd = fds.solve(torch.from_numpy(rhs), tol=1e-10)
        dln = dl.cpu().numpy()
        fd = float(np.dot(dln, 2 * xmn + dln)) / (2 * h)
        an = (gv * dv).sum().item()
        assert fd == pytest.approx(an, rel=1e-5)


@pytest.mark.parametrize("name", ["G1_1024x1024_schur1_exti_option3", "G1_1024x1024_schur1_exti_option4_k3",
                                  "G1_1024x1024_diffuseE_schur1_exti", "G20_256x256_amg_cf_gauss_seidel"])
def test_options_at_full_size(gpu, name):
    """The options beside the default path at their workloads' full sizes, in
    the bench's launch form (batched launches, graph replay, autotuned
    layouts): option #3 and option #4 inverses, E diffusing (Eq. 2.1 as
    printed), the C/F Gauss-Seidel smoother.  FP64 iterations and every
    inverse's V-cycle count equal the stored oracle solve's; the stored
    entries within 1e-10 of max|x|."""
    rec = _golden("oracle_options_fullsize.json")[name]
    s = I.preset(rec["preset"])
    assert s.n == rec["n"] and s.nnz == rec["nnz"]
    slv = gpu.Solver(batched=1, use_graph=1, autotune=1, **rec["options"]).setup_system(s, rec["precond"])
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    assert rc == 0 and it == rec["iterations"], (it, rec["iterations"])
    assert rr == pytest.approx(rec["relres"], rel=1e-4)
    xg = x.cpu().numpy()
    idx = np.asarray(rec["sample_index"])
    assert np.max(np.abs(xg[idx] - np.asarray(rec["sample_x"]))) <= 1e-10 * rec["x_max_abs"]
    assert abs(np.linalg.norm(xg) - rec["x_norm2"]) <= 1e-10 * rec["x_norm2"]
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        key = f"{info['kind']},{info['comp']}"
        assert slv.op_cycles(k) == rec["cycles"].get(key, 0), (key, slv.op_cycles(k), rec["cycles"].get(key))
