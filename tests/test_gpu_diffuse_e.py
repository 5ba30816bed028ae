"""The second workload family: Eq. 2.1 with the electron energy diffusing
(E gets a stencil, so A_E needs its own multilevel hierarchy and option #1
is no longer exact), with one and with (3, 1, 1) V-cycles per group/E/I
inverse and with option #3.  GPU against the oracle through the C ABI:
hierarchies bit-exact, iteration and V-cycle counts equal, x within 1e-10."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = ["amg", "pctl", "schur1", "schur2", "bd", "blt"]


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


def _sys(name):
    return {"G4": I.make_system(4, (29, 23), multigroup=True, diffuse_E=True),
            "G1_inc": I.make_system(1, (40, 40), inclusion=True, diffuse_E=True),
            "G2_3d": I.make_system(2, (9, 8, 7), multigroup=True, diffuse_E=True),
            "G20": I.make_system(20, (13, 11), multigroup=True, diffuse_E=True)}[name]


def _same_hierarchy(slv, op, oh):
    assert slv.op_info(op)["nlevels"] == oh.nlevels
    for l in range(oh.nlevels):
        g = slv.level(op, l)
        rp, ci, v = oh.A(l).arrays()
        assert np.array_equal(g["rp"], rp) and np.array_equal(g["ci"], ci) and np.array_equal(g["v"], v), l
        if l < oh.nlevels - 1:
            assert np.array_equal(g["cf"], oh.CF(l))
            prp, pci, pv = oh.P(l).arrays()
            assert np.array_equal(g["prp"], prp) and np.array_equal(g["pci"], pci) and np.array_equal(g["pv"], pv)


@pytest.mark.parametrize("case", ["G4", "G1_inc", "G2_3d"])
@pytest.mark.parametrize("kind", KINDS)
def test_diffuse_e_parity_fp64(gpu, orc, case, kind):
    s = _sys(case)
    slv = gpu.Solver().setup_system(s, kind)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind)
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        if info["use_jacobi"] or info["kind"] == 5:
            continue
        oh = ob.amg(orc.OP_MONO, 0) if kind == "amg" else ob.amg(info["kind"], info["comp"])
        _same_hierarchy(slv, k, oh)
    # E really diffuses: its operator is multilevel where the method inverts A_E by AMG
    if kind in ("pctl", "bd", "blt"):
        e = [k for k in range(slv.stats()["n_ops"]) if slv.op_info(k)["kind"] == 0 and slv.op_info(k)["comp"] == s.G]
        assert slv.op_info(e[0])["nlevels"] >= 2
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8, maxit=1000)
    assert rc == sto == 0 and it == ito, (it, ito)
    assert_x_close(x.cpu().numpy(), xo)


@pytest.mark.parametrize("kind", ["schur2", "bd", "blt", "pctl"])
@pytest.mark.parametrize("graph", [0, 1])
def test_diffuse_e_cycles_311(gpu, orc, kind, graph):
    s = _sys("G20")
    o = dict(nvcyc_group=3, nvcyc_E=1, nvcyc_I=1)
    slv = gpu.Solver(batched=graph, use_graph=graph, **o).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(**o))
    xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert rc == sto == 0 and it == ito
    assert_x_close(x.cpu().numpy(), xo)
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        assert slv.op_cycles(k) == ob.cycles(info["kind"], info["comp"]), info


@pytest.mark.parametrize("kind", ["schur1", "schur2", "pctl"])
def test_diffuse_e_option3(gpu, orc, kind):
    s = _sys("G4")
    slv = gpu.Solver(inner_mode=1, batched=1, use_graph=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(inner_mode=1))
    xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert rc == sto == 0 and it == ito
    assert_x_close(x.cpu().numpy(), xo)
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        assert slv.op_cycles(k) == ob.cycles(info["kind"], info["comp"]), info


@pytest.mark.parametrize("kind", ["schur1", "schur2", "bd"])
def test_diffuse_e_fp32(gpu, orc, kind):
    s = _sys("G4")
    slv = gpu.Solver(precision=1, batched=1, use_graph=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    _, ito, _, _, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind), tol=1e-8)
    assert rc == 0 and abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(s.b - s.scipy() @ x.cpu().numpy()) <= 1.0000001e-8 * np.linalg.norm(s.b)
