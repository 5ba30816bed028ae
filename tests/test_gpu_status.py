"""Failure statuses of the C ABI, provoked from the host with inputs that are
valid to read (no device fault is involved): a NaN or an infinity in b or in
the matrix values, a singular coarsest-level matrix, and Arnoldi breakdowns
(Section 2, GMRES(m)) with and without a solution in the Krylov space.  Each
case is also run through the oracle where it defines the outcome."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2002_04958_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENOCONV, EBREAKDOWN, ESINGULAR, ENAN = 2, 3, 4, 5


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2002_04958_gb300 import mgdamg
    return mgdamg


def _setup(gpu, A, G, N, kind="amg", **o):
    A = A.tocsr()
    A.sort_indices()
    return gpu.Solver(**o).setup(G, N, torch.from_numpy(A.indptr.astype(np.int32)),
                                 torch.from_numpy(A.indices.astype(np.int32)), torch.from_numpy(A.data), kind)


@pytest.mark.parametrize("where", ["b_nan", "b_inf"])
@pytest.mark.parametrize("kind", ["amg", "schur1"])
def test_non_finite_right_hand_side(gpu, where, kind):
    s = I.make_system(1, (9, 7))
    slv = gpu.Solver(batched=1, use_graph=1).setup_system(s, kind)
    b = s.b.copy()
    b[17] = np.nan if where == "b_nan" else np.inf
    with pytest.raises(gpu.MgdError) as e:
        slv.solve(torch.from_numpy(b))
    assert e.value.code == ENAN
    # the context stays usable
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b))
    assert rc == 0 and rr <= 1e-8


@pytest.mark.parametrize("what", ["offdiag_nan", "coupling_inf", "diag_nan"])
def test_non_finite_matrix_value(gpu, what):
    s = I.make_system(2, (8, 6), multigroup=True)
    v = s.val.copy()
    row = 5
    ps = list(range(s.rowptr[row], s.rowptr[row + 1]))
    if what == "offdiag_nan":
        p = [q for q in ps if s.col[q] != row and s.col[q] // s.N == 0][0]
        v[p] = np.nan
    elif what == "coupling_inf":
        p = [q for q in ps if s.col[q] // s.N != 0][0]
        v[p] = -np.inf
    else:
        p = [q for q in ps if s.col[q] == row][0]
        v[p] = np.nan
    for kind in ["amg", "schur2"]:
        with pytest.raises(gpu.MgdError) as e:
            gpu.Solver().setup(s.G, s.N, torch.from_numpy(s.rowptr), torch.from_numpy(s.col), torch.from_numpy(v),
                               kind)
        assert e.value.code == ENAN, (what, kind)
    # the same through mgd_update_values on a set-up context
    slv = gpu.Solver().setup_system(s, "amg")
    with pytest.raises(gpu.MgdError) as e:
        slv.update_values(torch.from_numpy(v))
    assert e.value.code == ENAN


def test_singular_coarsest_level(gpu):
    # I_3 (x) [[1, -1], [-1, 1]]: positive diagonal, strong connections, singular;
    # n = 6 <= max_coarse, so level 0 is the coarsest and its elimination meets a zero pivot
    L = sp.kron(sp.eye(3), sp.csr_matrix(np.array([[1.0, -1.0], [-1.0, 1.0]])))
    with pytest.raises(gpu.MgdError) as e:
        _setup(gpu, L, 1, 2)
    assert e.value.code == ESINGULAR


@pytest.mark.parametrize("o", [dict(), dict(batched=1, use_graph=1)], ids=["plain", "batched_graph"])
def test_happy_breakdown_returns_exact_solution(gpu, orc, o):
    # A = 2 I: no strong connections, the only level is solved exactly by the
    # dense inverse, so A M v_0 = v_0 and h_{1,0} = 0 exactly
    n = 6
    A = sp.csr_matrix(2.0 * sp.eye(n))
    slv = _setup(gpu, A, 1, 2, **o)
    b = np.zeros(n)
    b[4] = 1.0
    x, it, rr, rc = slv.solve(torch.from_numpy(b))
    assert rc == 0 and it == 1 and rr == 0.0
    assert np.array_equal(x.cpu().numpy(), b / 2)
    Ao = orc.Csr.from_scipy(A)
    xo, ito, rro, st, _ = orc.fgmres(Ao, b, orc.Block(Ao, 1, 2, "amg"), tol=1e-8)
    assert st == 0 and ito == 1 and np.array_equal(xo, b / 2)


@pytest.mark.parametrize("o", [dict(), dict(batched=1, use_graph=1)], ids=["plain", "batched_graph"])
def test_breakdown_without_solution(gpu, orc, o):
    # singular A = I_3 (x) [[1, 1], [1, 1]]; positive off-diagonals are not strong,
    # so coarsening stalls above max_coarse = 1 and the level is relaxed by two
    # l1-Jacobi sweeps (no elimination): M v_0 = v_0 for the null vector
    # v_0 = (1, -1, 0, ...)/sqrt(2), hence A M v_0 = 0 and the Hessenberg matrix is singular
    n = 6
    S = sp.kron(sp.eye(3), sp.csr_matrix(np.ones((2, 2))))
    slv = _setup(gpu, S, 1, 2, max_coarse=1, **o)
    b = np.zeros(n)
    b[0], b[1] = 1.0, -1.0
    with pytest.raises(gpu.MgdError) as e:
        slv.solve(torch.from_numpy(b))
    assert e.value.code == EBREAKDOWN
    So = orc.Csr.from_scipy(S.tocsr())
    xo, ito, rro, st, _ = orc.fgmres(So, b, orc.Block(So, 1, 2, "amg", orc.opts(max_coarse=1)), tol=1e-8)
    assert st == 2 and ito == 1 and not xo.any()


def test_iteration_cap_keeps_last_iterate(gpu, orc):
    s = I.make_system(1, (9, 7))
    slv = gpu.Solver(max_it=4).setup_system(s, "amg")
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b), tol=1e-14, allow_noconv=True)
    assert rc == ENOCONV and it == 4
    Ao = orc.csr_of_system(s)
    xo, ito, rro, st, _ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, "amg"), tol=1e-14, maxit=4)
    assert st == 1 and ito == 4
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()


def test_binding_refuses_wrong_lengths(gpu):
    # the library reads these buffers through raw pointers: the binding
    # refuses a short vector before the call
    s = I.make_system(1, (9, 7))
    slv = gpu.Solver().setup_system(s, "amg")
    short = torch.zeros(s.n - 1, dtype=torch.float64)
    for call in (lambda: slv.solve(short), lambda: slv.precond_apply(short),
                 lambda: slv.update_values(torch.zeros(s.nnz - 1, dtype=torch.float64)),
                 lambda: slv.grad_values(short, short), lambda: slv.solve_host(short.numpy())):
        with pytest.raises(ValueError):
            call()
    with pytest.raises(gpu.MgdError):
        gpu.Solver().solve(torch.zeros(4, dtype=torch.float64))
    x, it, rr, rc = slv.solve(torch.from_numpy(s.b))   # the context is unharmed
    assert rc == 0 and rr <= 1e-8
