"""Aggressive coarsening of the finest levels (Section 3.1) on the GPU against
the oracle: a second strength + PMIS pass on the Galerkin operator of the
first pass, P = P1 P2.  Bar: C/F marks, P and every coarse operator
bit-exact; FGMRES iteration counts equal and x within 1e-10 relative."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "G1_inc": (1, (40, 40), False, True),
    "G4": (4, (29, 23), True, False),
    "G2_3d": (2, (9, 8, 7), True, False),
    "G20": (20, (13, 11), True, False),
}


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


@pytest.mark.parametrize("opts", [dict(agg_levels=1), dict(agg_levels=1, interp_type=1),
                                  dict(agg_levels=2, interp_type=1), dict(agg_levels=1, smoother=1)],
                         ids=["agg1", "agg1_exti", "agg2_exti", "agg1_gs"])
@pytest.mark.parametrize("case", ["G1_inc", "G4", "G2_3d"])
@pytest.mark.parametrize("kind", ["amg", "schur1", "schur2"])
def test_aggressive_setup_bit_exact_and_solve(gpu, orc, opts, case, kind):
    s = _system(case)
    slv = gpu.Solver(**opts).setup_system(s, kind)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(**opts))
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        if info["use_jacobi"]:
            continue
        oh = ob.amg(orc.OP_MONO, 0) if kind == "amg" else ob.amg(info["kind"], info["comp"])
        assert info["nlevels"] == oh.nlevels
        for l in range(oh.nlevels):
            g = slv.level(k, l)
            rp, ci, v = oh.A(l).arrays()
            assert np.array_equal(g["rp"], rp) and np.array_equal(g["ci"], ci), (k, l)
            assert np.array_equal(g["v"], v), (k, l)
            if l < oh.nlevels - 1:
                assert np.array_equal(g["cf"], oh.CF(l)), (k, l)
                prp, pci, pv = oh.P(l).arrays()
                assert np.array_equal(g["prp"], prp) and np.array_equal(g["pci"], pci) and np.array_equal(g["pv"], pv)
            if opts.get("smoother"):
                gk, gnk = slv.level_keys(k, l)
                ok, onk = oh.key(l)
                assert gnk == onk and (onk == 0 or np.array_equal(gk, ok))
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8, maxit=1000)
    assert rc == sto and it == ito, (it, ito, rc, sto)
    if rc == 0:
        assert_x_close(x.cpu().numpy(), xo)


@pytest.mark.parametrize("kind", ["bd", "schur2"])
def test_aggressive_batched_graph_fp32(gpu, orc, kind):
    s = _system("G20")
    b = torch.from_numpy(s.b)
    ref = gpu.Solver(agg_levels=1, autotune=0).setup_system(s, kind)
    xr, itr, _, _ = ref.solve(b)
    slv = gpu.Solver(agg_levels=1, autotune=0, batched=1, use_graph=1).setup_system(s, kind)
    x, it, _, _ = slv.solve(b)
    assert it == itr and torch.equal(x, xr)
    slv = gpu.Solver(agg_levels=1, precision=1, batched=1, use_graph=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(b, tol=1e-8, allow_noconv=True)
    assert rc == 0 and abs(it - itr) <= 1
