"""Section 3.1's smoother on the GPU: Gauss-Seidel in C/F order, run as
multicolour Gauss-Seidel (Jones-Plassmann colouring of the symmetrised graph
of each level, C colours then F colours on the way down, the reverse on the
way up), against the oracle through the C ABI.

Bar (FP64): colourings / sweep orders and hierarchies bit-exact, FGMRES
iteration counts equal, x within 1e-10 relative; transposed cycles for the
adjoint; FP32 V-cycles within +-1 iteration."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "G1": (1, (45, 37), False, False),
    "G1_inc": (1, (40, 40), False, True),
    "G4": (4, (29, 23), True, False),
    "G20": (20, (13, 11), True, False),
    "G2_3d": (2, (9, 8, 7), True, False),
}
GS = dict(smoother=1)


def _system(name):
    G, dims, mg, inc = CASES[name]
    return I.make_system(G, dims, multigroup=mg, inclusion=inc)


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


@pytest.mark.parametrize("case", ["G1_inc", "G4", "G2_3d"])
@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "pctl"])
def test_gs_order_and_hierarchy_bit_exact(gpu, orc, case, kind):
    s = _system(case)
    slv = gpu.Solver(**GS).setup_system(s, kind)
    ob = orc.Block(orc.csr_of_system(s), s.G, s.N, kind, orc.opts(**GS))
    checked = 0
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        if info["use_jacobi"] or (kind == "pctl" and info["kind"] == 5):
            continue
        oh = ob.amg(orc.OP_MONO, 0) if kind == "amg" else ob.amg(info["kind"], info["comp"])
        assert info["nlevels"] == oh.nlevels
        for l in range(oh.nlevels):
            g = slv.level(k, l)
            rp, ci, v = oh.A(l).arrays()
            assert np.array_equal(g["rp"], rp) and np.array_equal(g["ci"], ci) and np.array_equal(g["v"], v)
            gk, gnk = slv.level_keys(k, l)
            ok, onk = oh.key(l)
            assert gnk == onk
            if onk:
                assert np.array_equal(gk, ok), (k, l)
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["amg", "pctl", "schur1", "schur2", "bd", "blt"])
def test_gs_solve_parity_fp64(gpu, orc, case, kind):
    s = _system(case)
    slv = gpu.Solver(**GS).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind, orc.opts(**GS)), tol=1e-8, maxit=1000)
    assert rc == sto == 0 and it == ito, (it, ito)
    assert_x_close(x.cpu().numpy(), xo)


@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "bd"])
def test_gs_precond_apply_matches_oracle(gpu, orc, kind):
    s = _system("G4")
    slv = gpu.Solver(**GS).setup_system(s, kind)
    v = np.random.default_rng(3).standard_normal(s.n)
    z = slv.precond_apply(torch.from_numpy(v)).cpu().numpy()
    zo = orc.Block(orc.csr_of_system(s), s.G, s.N, kind, orc.opts(**GS)).apply(v)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


@pytest.mark.parametrize("kind", ["bd", "schur2", "schur1", "amg"])
def test_gs_batched_graph_fused(gpu, kind):
    s = _system("G20")
    b = torch.from_numpy(s.b)
    ref = gpu.Solver(autotune=0, fuse_rows=-1, **GS).setup_system(s, kind)
    xr, itr, _, _ = ref.solve(b)
    for opts in [dict(batched=1), dict(use_graph=1), dict(batched=1, use_graph=1), dict(batched=1, pdl=0)]:
        slv = gpu.Solver(autotune=0, fuse_rows=-1, **GS, **opts).setup_system(s, kind)
        x, it, _, _ = slv.solve(b)
        assert it == itr and torch.equal(x, xr), opts
    # every level below level 0 in the cluster kernel, and the autotuned plan
    for opts in [dict(fuse_rows=1 << 30, batched=1, use_graph=1), dict(autotune=1, batched=1, use_graph=1)]:
        o = dict(autotune=0, **GS)
        o.update(opts)
        slv = gpu.Solver(**o).setup_system(s, kind)
        x, it, _, _ = slv.solve(b)
        assert it == itr, opts
        assert torch.linalg.vector_norm(x - xr) <= 1e-10 * torch.linalg.vector_norm(xr), opts


@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2", "bd", "pctl"])
def test_gs_fp32_vcycles(gpu, orc, kind):
    s = _system("G4")
    slv = gpu.Solver(precision=1, batched=1, use_graph=1, **GS).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    _, ito, _, _, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind, orc.opts(**GS)), tol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)


@pytest.mark.parametrize("fuse", [-1, 1 << 30])
def test_gs_transposed_cycle_adjoint(gpu, orc, fuse):
    s = _system("G4")
    slv = gpu.Solver(keep_transpose=1, fuse_rows=fuse, autotune=0, **GS).setup_system(s, "amg")
    g = np.random.default_rng(4).standard_normal(s.n)
    lam, it, rr = slv.solve_transpose(torch.from_numpy(g), tol=1e-8)
    Ao = orc.csr_of_system(s)
    lo, ito, _, sto, _ = orc.fgmres(Ao, g, orc.Block(Ao, s.G, s.N, "amg", orc.opts(**GS)), tol=1e-8, transpose=True)
    assert sto == 0 and it == ito
    assert np.linalg.norm(lam.cpu().numpy() - lo) <= 1e-10 * np.linalg.norm(lo)


def test_gs_with_option3_and_three_cycles(gpu, orc):
    s = _system("G4")
    for kind, o in [("schur2", dict(inner_mode=1)), ("bd", dict(nvcyc_group=3))]:
        o = dict(o, **GS)
        slv = gpu.Solver(batched=1, use_graph=1, **o).setup_system(s, kind)
        x, it, _, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
        Ao = orc.csr_of_system(s)
        ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(**o))
        xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
        assert rc == sto == 0 and it == ito
        assert_x_close(x.cpu().numpy(), xo)
        for k in range(slv.stats()["n_ops"]):
            info = slv.op_info(k)
            assert slv.op_cycles(k) == ob.cycles(info["kind"], info["comp"])
