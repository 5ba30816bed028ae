"""Option #3 inside the preconditioner (Section 3.5; Section 4's 1e-2 inner
accuracy) and several V-cycles per inverse, on the GPU against the oracle.

The inner loop runs on the device: the V-cycle kernels skip operators that
have converged, a control kernel decides after every cycle, and under graph
replay a conditional while node repeats the loop body.  Bar (FP64): FGMRES
iteration counts and every inverse's V-cycle count equal the oracle's, the
solution within 1e-10 relative; eager, batched and graph-replayed runs give
the same bits."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "G4": (4, (29, 23), True, False),
    "G20": (20, (13, 11), True, False),
    "G2_3d": (2, (9, 8, 7), True, False),
    "G1_inc": (1, (40, 40), False, True),
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


def _cycles_match(slv, ob):
    for k in range(slv.stats()["n_ops"]):
        info = slv.op_info(k)
        assert slv.op_cycles(k) == ob.cycles(info["kind"], info["comp"]), (k, info)


@pytest.mark.parametrize("case", ["G4", "G20", "G2_3d", "G1_inc"])
@pytest.mark.parametrize("kind", ["schur1", "schur2", "pctl"])
def test_option3_parity_fp64(gpu, orc, case, kind):
    s = _system(case)
    slv = gpu.Solver(inner_mode=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(inner_mode=1))
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8, maxit=1000)
    assert rc == 0 and sto == 0
    assert it == ito, (it, ito)
    assert_x_close(x.cpu().numpy(), xo)
    _cycles_match(slv, ob)
    # the inner loops really iterate: more V-cycles than one per inverse
    acc = [k for k in range(slv.stats()["n_ops"]) if slv.op_info(k)["kind"] in
           {"schur1": (1, 2), "schur2": (3, 4), "pctl": (0,)}[kind] and not slv.op_info(k)["use_jacobi"]]
    assert max(slv.op_cycles(k) for k in acc) > it


@pytest.mark.parametrize("kind", ["schur1", "schur2", "pctl"])
def test_option3_precond_apply_matches_oracle(gpu, orc, kind):
    s = _system("G4")
    slv = gpu.Solver(inner_mode=1).setup_system(s, kind)
    v = np.random.default_rng(5).standard_normal(s.n)
    z = slv.precond_apply(torch.from_numpy(v)).cpu().numpy()
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(inner_mode=1))
    zo = ob.apply(v)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    _cycles_match(slv, ob)


@pytest.mark.parametrize("kind", ["schur2", "schur1", "pctl"])
def test_option3_eager_batched_graph_identical(gpu, kind):
    s = _system("G20")
    b = torch.from_numpy(s.b)
    ref = gpu.Solver(inner_mode=1, autotune=0).setup_system(s, kind)
    xr, itr, _, _ = ref.solve(b)
    cyc = [ref.op_cycles(k) for k in range(ref.stats()["n_ops"])]
    for opts in [dict(batched=1), dict(use_graph=1), dict(batched=1, use_graph=1),
                 dict(batched=1, use_graph=1, pdl=0)]:
        o = dict(inner_mode=1, autotune=0)
        o.update(opts)
        slv = gpu.Solver(**o).setup_system(s, kind)
        x, it, _, _ = slv.solve(b)
        assert it == itr, opts
        assert torch.equal(x, xr), opts
        assert [slv.op_cycles(k) for k in range(slv.stats()["n_ops"])] == cyc, opts
        # a second solve replays the same loops
        x2, it2, _, _ = slv.solve(b)
        assert it2 == itr and torch.equal(x2, xr), opts
    # autotuned sparse formats sum in another order: same counts, values to rounding
    slv = gpu.Solver(inner_mode=1, autotune=1, batched=1, use_graph=1).setup_system(s, kind)
    x, it, _, _ = slv.solve(b)
    assert it == itr
    assert torch.linalg.vector_norm(x - xr) <= 1e-10 * torch.linalg.vector_norm(xr)


@pytest.mark.parametrize("kind", ["schur1", "schur2", "pctl"])
def test_option3_fp32_vcycles(gpu, orc, kind):
    s = _system("G4")
    slv = gpu.Solver(inner_mode=1, precision=1, batched=1, use_graph=1).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    _, ito, _, _, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind, orc.opts(inner_mode=1)), tol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    xg = x.cpu().numpy()
    assert np.linalg.norm(s.b - s.scipy() @ xg) <= 1.0000001e-8 * np.linalg.norm(s.b)


@pytest.mark.parametrize("kind", ["bd", "blt", "schur2"])
@pytest.mark.parametrize("graph", [0, 1])
def test_three_one_one_cycles(gpu, orc, kind, graph):
    # three V-cycles per group inverse, one for E and I (the radiation-heavy split)
    s = _system("G4")
    o = dict(nvcyc_group=3, nvcyc_E=1, nvcyc_I=1)
    slv = gpu.Solver(batched=graph, use_graph=graph, **o).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(**o))
    xo, ito, _, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8)
    assert rc == 0 and sto == 0 and it == ito
    assert_x_close(x.cpu().numpy(), xo)
    _cycles_match(slv, ob)


def test_three_cycles_transposed_bd(gpu, orc):
    # the transposed apply keeps the fixed cycle counts (plain path)
    s = _system("G4")
    slv = gpu.Solver(nvcyc_group=3, keep_transpose=1).setup_system(s, "bd")
    g = np.random.default_rng(2).standard_normal(s.n)
    lam, it, rr = slv.solve_transpose(torch.from_numpy(g), tol=1e-8)
    lamg = lam.cpu().numpy()
    assert np.linalg.norm(g - s.scipy().T @ lamg) <= 1.0000001e-8 * np.linalg.norm(g)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, "bd", orc.opts(nvcyc_group=3))
    lo, ito, _, sto, _ = orc.fgmres(Ao, g, ob, tol=1e-8, transpose=True)
    assert sto == 0 and it == ito
    _cycles_match(slv, ob)


def test_option3_rejects_bad_options(gpu):
    for bad in [dict(inner_maxit=0), dict(inner_mode=2), dict(inner_tol=-1.0), dict(nvcyc_group=100000)]:
        with pytest.raises(Exception):
            gpu.Solver(**bad)
