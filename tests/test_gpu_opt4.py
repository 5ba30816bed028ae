"""Option #4 (Section 3.5) on the GPU against the oracle: the Schur complement
with a one-block inner inverse (S_I of Schur2, C_E of Schur1) inverted by K
steps of w(k+1) = A_a^-1 (q + D_ab A_b^-1 D_ba w(k)) with V-cycles on the
plain blocks.  Bar (FP64): FGMRES iteration counts and every inverse's
V-cycle count equal the oracle's, the solution within 1e-10 (2-norm and worst
element); the preconditioner output within 1e-11; per-operator, batched and
graph-replayed launches agree to rounding."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I
from parity_checks import assert_x_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "G1_inc": dict(G=1, dims=(40, 40), multigroup=False, inclusion=True),
    "G4": dict(G=4, dims=(29, 23), multigroup=True),
    "G2_3d": dict(G=2, dims=(9, 8, 7), multigroup=True),
    "G3_diffE": dict(G=3, dims=(31, 27), multigroup=True, diffuse_E=True),
}


def _system(name):
    return I.make_system(**CASES[name])


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


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["schur2", "schur1"])
@pytest.mark.parametrize("K", [1, 3])
def test_option4_parity_fp64(gpu, orc, case, kind, K):
    s = _system(case)
    slv = gpu.Solver(opt4_steps=K).setup_system(s, kind)
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-8, allow_noconv=True)
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(opt4_steps=K))
    xo, ito, rro, sto, _ = orc.fgmres(Ao, s.b, ob, tol=1e-8, maxit=1000)
    assert rc == 0 and sto == 0
    assert it == ito, (it, ito)
    assert_x_close(x.cpu().numpy(), xo)
    _cycles_match(slv, ob)
    # the plain block replaced the diagonal approximation
    kinds = {slv.op_info(k)["kind"] for k in range(slv.stats()["n_ops"])}
    assert (4 if kind == "schur2" else 1) not in kinds


@pytest.mark.parametrize("kind", ["schur2", "schur1"])
def test_option4_precond_apply_matches_oracle(gpu, orc, kind):
    s = _system("G3_diffE")
    slv = gpu.Solver(opt4_steps=4).setup_system(s, kind)
    v = np.random.default_rng(7).standard_normal(s.n)
    z = slv.precond_apply(torch.from_numpy(v)).cpu().numpy()
    Ao = orc.csr_of_system(s)
    ob = orc.Block(Ao, s.G, s.N, kind, orc.opts(opt4_steps=4))
    zo = ob.apply(v)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    assert np.abs(z - zo).max() <= 1e-11 * np.abs(zo).max()
    _cycles_match(slv, ob)


@pytest.mark.parametrize("kind", ["schur2", "schur1"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32_vcycle"])
def test_option4_launch_forms_agree(gpu, orc, kind, precision):
    s = _system("G4")
    b = torch.from_numpy(s.b)
    runs = []
    for o in [dict(), dict(batched=1), dict(batched=1, use_graph=1)]:
        slv = gpu.Solver(opt4_steps=3, precision=precision, **o).setup_system(s, kind)
        x, it, rr, rc = slv.solve(b, tol=1e-8)
        assert rc == 0
        runs.append((x.cpu().numpy(), it))
    for x, it in runs[1:]:
        assert abs(it - runs[0][1]) <= (0 if precision == 0 else 1)
        if precision == 0:
            assert_x_close(x, runs[0][0], rel=1e-12)
    Ao = orc.csr_of_system(s)
    xo, ito, *_ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind, orc.opts(opt4_steps=3)), tol=1e-8)
    assert all(abs(it - ito) <= (0 if precision == 0 else 1) for _, it in runs)


def test_option4_rejects_bad_step_count(gpu):
    with pytest.raises(gpu.MgdError) as e:
        gpu.Solver(opt4_steps=-1)
    assert e.value.code == 1
