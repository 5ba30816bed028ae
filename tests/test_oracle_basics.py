"""Pins of the CPU oracle's building blocks against facts fixed outside it:
published generator outputs, library routines, closed forms, hand-worked
values and brute force on tiny inputs (no GPU)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_2002_04958_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLD, name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_reference_values(orc):
    ref = _golden_ints("splitmix64_seed1234567.txt")
    got_c = [orc.lib().or_splitmix64(1234567, i) for i in range(5)]
    z = I._mix64(np.uint64(1234567) + np.arange(1, 6, dtype=np.uint64) * I.GOLDEN)
    assert got_c == ref
    assert [int(v) for v in z] == ref


def test_uniform_streams_agree(orc):
    for seed, stream in [(0, 1000), (7, 1003), (2**63 + 5, 10)]:
        u = I.uniform(seed, stream, 50)
        assert np.all((u >= 0) & (u < 1))
        c = np.array([orc.uniform(seed, stream, i) for i in range(50)])
        assert np.array_equal(u, c)


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("G,dims,mg", [(1, (7, 5), False), (3, (4, 3, 5), True)])
def test_generator_block_structure(G, dims, mg):
    s = I.make_system(G, dims, multigroup=mg)
    N = int(np.prod(dims))
    A = s.scipy().toarray()
    nc = G + 2
    E, Iidx = G, G + 1
    # nnz: per diffusing block N + 2*sum_axes (N/n_ax)*(n_ax-1); E diagonal; 2N per coupling pair
    faces = sum(N // d * (d - 1) for d in dims)
    ndiff = G + 1
    assert s.nnz == ndiff * (N + 2 * faces) + N + 2 * N * (G + 1)
    for a in range(nc):
        for b in range(nc):
            blk = A[a * N:(a + 1) * N, b * N:(b + 1) * N]
            if a == b:
                continue
            coupled = (a < G and b == E) or (a == E and b < G) or {a, b} == {E, Iidx}
            if coupled:
                assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
                assert np.all(np.diag(blk) < 0)
            else:
                assert np.count_nonzero(blk) == 0
    # D_EI = D_IE (Eq. 2.2) and D_gE != D_Eg
    dEI = np.diag(A[E * N:(E + 1) * N, Iidx * N:(Iidx + 1) * N])
    dIE = np.diag(A[Iidx * N:(Iidx + 1) * N, E * N:(E + 1) * N])
    assert np.array_equal(dEI, dIE)
    assert not np.array_equal(np.diag(A[0:N, E * N:(E + 1) * N]), np.diag(A[E * N:(E + 1) * N, 0:N]))
    # strictly diagonally dominant rows: margin >= mass term 1 (Dirichlet faces add more)
    d = np.diag(A)
    off = np.abs(A).sum(1) - d
    assert np.all(d - off >= 1.0 - 1e-12 * d.max())
    # symmetric diffusion blocks; E has no stencil
    for a in range(nc):
        blk = A[a * N:(a + 1) * N, a * N:(a + 1) * N]
        assert np.allclose(blk, blk.T, rtol=0, atol=0)
    AE = A[E * N:(E + 1) * N, E * N:(E + 1) * N]
    assert np.count_nonzero(AE - np.diag(np.diag(AE))) == 0
    assert s.rowptr[-1] == s.nnz
    for r in range(s.n):
        c = s.col[s.rowptr[r]:s.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("preset", [5, 6])
def test_generator_diffuse_e_structure(preset):
    # Eq. 2.1 as printed: E diffuses with the groups' stencil; every other rule unchanged
    s = I.preset(preset, dims=(7, 6))
    G, N = s.G, s.N
    faces = sum(N // d * (d - 1) for d in (7, 6))
    assert s.nnz == (G + 2) * (N + 2 * faces) + 2 * N * (G + 1)
    A = s.scipy().toarray()
    E = G
    AE = A[E * N:(E + 1) * N, E * N:(E + 1) * N]
    A0 = A[:N, :N]
    assert np.array_equal(AE != 0, A0 != 0)
    assert np.array_equal(AE, AE.T)
    d = np.diag(A)
    assert np.all(d - (np.abs(A).sum(1) - d) >= 1.0 - 1e-12 * d.max())
    t = I.preset(preset - 4, dims=(7, 6))   # the same system without E diffusion
    assert np.array_equal(np.delete(A, np.s_[E * N:(E + 1) * N], 0),
                          np.delete(t.scipy().toarray(), np.s_[E * N:(E + 1) * N], 0))


def test_generator_tpfa_values_by_hand():
    # 2x1 grid, one group: cell diffusion k0, k1 -> face T = 2 k0 k1 / (k0+k1),
    # boundary faces 2k (three per cell in 2D with ny=1: left/right ends + bottom + top)
    s = I.make_system(1, (2, 1))
    k0, k1 = I.log_uniform(0, I.STREAM_DIFF + 0, 2, -3.0, 3.0)
    A = s.scipy().toarray()
    T = 2 * k0 * k1 / (k0 + k1)
    cgE = I.log_uniform(0, I.STREAM_C_GE + 0, 2, -2.0, 2.0)
    assert A[0, 1] == pytest.approx(-T, rel=1e-15)
    assert A[0, 0] == pytest.approx(T + 3 * 2 * k0 + cgE[0] + 1.0, rel=1e-14)
    assert A[0, 2 + 0] == pytest.approx(-cgE[0], rel=1e-15)


# ---------------------------------------------------------------- CSR kernels
def _rand_csr(rng, n, m, density):
    M = sp.random(n, m, density=density, random_state=rng, format="csr")
    M.data = rng.standard_normal(M.nnz)
    M.sort_indices()
    return M


def test_spmv_transpose_spgemm_vs_scipy(orc):
    rng = np.random.default_rng(1)
    X = _rand_csr(rng, 40, 30, 0.1)
    Y = _rand_csr(rng, 30, 25, 0.15)
    Xo, Yo = orc.Csr.from_scipy(X), orc.Csr.from_scipy(Y)
    x = rng.standard_normal(30)
    assert np.allclose(orc.spmv(Xo, x), X @ x, rtol=1e-14, atol=1e-14)
    assert abs(orc.transpose(Xo).scipy() - X.T).max() == 0
    Z = orc.spgemm(Xo, Yo).scipy()
    assert np.allclose(Z.toarray(), (X @ Y).toarray(), rtol=1e-13, atol=1e-14)
    # structural pattern: every (i,j) reachable through some k is stored
    pat = ((abs(X) > 0).astype(int) @ (abs(Y) > 0).astype(int)).tocsr()
    assert Z.nnz == pat.nnz


def test_dense_lu_vs_numpy(orc):
    rng = np.random.default_rng(2)
    for n in [1, 5, 37, 100]:
        a = rng.standard_normal((n, n)) + 0.1 * np.eye(n)
        b = rng.standard_normal(n)
        st, lu, piv = orc.lu_factor(a)
        assert st == 0
        x = orc.lu_solve(lu, piv, b)
        assert np.allclose(x, np.linalg.solve(a, b), rtol=1e-9, atol=1e-11)
        xt = orc.lu_solve(lu, piv, b, transpose=True)
        assert np.allclose(xt, np.linalg.solve(a.T, b), rtol=1e-9, atol=1e-11)
    st, _, _ = orc.lu_factor(np.zeros((3, 3)))
    assert st != 0


# ---------------------------------------------------------------- strength
def test_strength_hand_example(orc):
    # row 0: a = [4, -1, -0.2, -0.3]: max(-a_0k) = 1, threshold 0.25 ->
    #   -1 strong, -0.2 weak, -0.3 strong.  row 1: positive off-diagonals only
    #   -> no strong connections.  row 2: diagonal only.  row 3: [-2 (col0), 5, -0.5 (col 2)]
    #   max 2, thr 0.5 -> col0 strong, col2 strong (equality counts).
    A = sp.csr_matrix(np.array([[4, -1, -0.2, -0.3],
                                [0.5, 3, 0.1, 0],
                                [0, 0, 2, 0],
                                [-2, 0, -0.5, 5.0]]))
    A.sort_indices()
    S = orc.strength(orc.Csr.from_scipy(A))
    expect = [0, 1, 0, 1,   0, 0, 0,   0,   1, 1, 0]
    assert S.tolist() == expect


def test_strength_brute_force(orc):
    rng = np.random.default_rng(3)
    for trial in range(5):
        n = 60
        A = _rand_csr(rng, n, n, 0.1) + sp.eye(n) * 5
        A = A.tocsr()
        A.sort_indices()
        S = orc.strength(orc.Csr.from_scipy(A), 0.25)
        k = 0
        for i in range(n):
            cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
            vals = A.data[A.indptr[i]:A.indptr[i + 1]]
            off = [-v for c, v in zip(cols, vals) if c != i]
            mx = max(off) if off else 0.0
            for c, v in zip(cols, vals):
                assert S[k] == int(c != i and mx > 0 and -v >= 0.25 * mx)
                k += 1


# ---------------------------------------------------------------- PMIS
def _pmis_naive(n, S_pairs, w):
    """Independent brute-force restatement on a dense strength matrix."""
    Sm = np.zeros((n, n), bool)
    for i, j in S_pairs:
        Sm[i, j] = True
    nbr = Sm | Sm.T
    cf = np.zeros(n, int)
    for i in range(n):
        if not Sm[i].any() and not Sm[:, i].any():
            cf[i] = -1
        elif w[i] < 1:
            cf[i] = -1
    while (cf == 0).any():
        und = cf == 0
        newc = []
        for i in np.flatnonzero(und):
            js = np.flatnonzero(nbr[i] & und)
            if all((w[i], i) > (w[j], j) for j in js):
                newc.append(i)
        cf[newc] = 1
        for i in np.flatnonzero(cf == 0):
            if (Sm[i] & (cf == 1)).any():
                cf[i] = -1
    return cf


def test_pmis_brute_force_and_invariants(orc):
    rng = np.random.default_rng(4)
    for trial in range(6):
        n = int(rng.integers(20, 150))
        A = _rand_csr(rng, n, n, 4.0 / n)
        A = (A - sp.diags(A.diagonal()) - sp.random(n, n, 0.02, random_state=rng) + sp.eye(n) * 10).tocsr()
        A.sort_indices()
        Ao = orc.Csr.from_scipy(A)
        S = orc.strength(Ao)
        nc, CF = orc.pmis(Ao, S, seed=trial, level=trial % 3)
        rows = np.repeat(np.arange(n), np.diff(A.indptr))
        pairs = [(int(r), int(c)) for r, c, s in zip(rows, A.indices, S) if s]
        cnt = np.zeros(n)
        for _, j in pairs:
            cnt[j] += 1
        w = cnt + np.array([orc.uniform(trial, 1000 + trial % 3, i) for i in range(n)])
        ref = _pmis_naive(n, pairs, w)
        assert np.array_equal(CF.astype(int), ref)
        assert nc == int((CF == 1).sum())
        # invariants: total; F points that influence someone have a strong C neighbour
        assert set(np.unique(CF)) <= {-1, 1}
        Sm = np.zeros((n, n), bool)
        for i, j in pairs:
            Sm[i, j] = True
        for i in range(n):
            if CF[i] == -1 and Sm[:, i].any():
                assert (Sm[i] & (CF == 1)).any()
            if CF[i] == 1:   # no C point depends strongly on a C point of larger weight
                for j in np.flatnonzero(Sm[i] & (CF == 1)):
                    assert (w[i], i) > (w[j], j)


def test_pmis_ties_larger_index_wins(orc):
    # path graph 0-1-2-3-4 (tridiagonal Poisson), all weights equal 2:
    # round 1: only point 4 beats all its undecided neighbours -> C; 3 -> F.
    # round 2: 2 beats 1 -> C; 1 -> F.  round 3: 0 has no undecided neighbour -> C.
    A = _tridiag(5)
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    nc, CF = orc.pmis_weights(Ao, S, np.full(5, 2.0))
    assert CF.tolist() == [1, -1, 1, -1, 1] and nc == 3
    # a weight below 1 makes point 1 F before the rounds; round 1: 0 (no
    # undecided neighbour) and 4 -> C, 3 -> F; round 2: 2 -> C
    nc, CF = orc.pmis_weights(Ao, S, np.array([2.0, 0.5, 2.0, 2.0, 2.0]))
    assert CF.tolist() == [1, -1, 1, -1, 1]


# ---------------------------------------------------------------- interpolation
def _tridiag(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def test_interp_1d_poisson_closed_form(orc):
    n = 15
    A = _tridiag(n)
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    CF = np.where(np.arange(n) % 2 == 1, 1, -1).astype(np.int8)   # C = odd points (7 of them)
    P = orc.interp(Ao, S, CF).scipy().toarray()
    nc = 7
    Pref = np.zeros((n, nc))
    for c in range(nc):
        Pref[2 * c + 1, c] = 1.0
        Pref[2 * c, c] = 0.5
        Pref[2 * c + 2, c] = 0.5
    assert np.array_equal(P, Pref)
    Ac = orc.rap(Ao, orc.interp(Ao, S, CF)).scipy().toarray()
    assert np.array_equal(Ac, 0.5 * _tridiag(nc).toarray())


def test_interp_hand_strong_f_neighbour(orc):
    # 1-D chain 0-1-2-3 with C = {0, 3}, F = {1, 2}; Poisson row stencil [-1 2 -1]
    # plus a weak connection.  Row 1: C_1={0}, strong F nbr 2 whose connections
    # into C_1 are none (a_20 = 0) -> lumped to the diagonal:
    #   w_10 = -(-1) / (2 + (-1)) = 1.
    A = sp.csr_matrix(np.array([[2, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 2.0]]))
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    CF = np.array([1, -1, -1, 1], np.int8)
    P = orc.interp(Ao, S, CF).scipy().toarray()
    assert np.array_equal(P, np.array([[1, 0], [1, 0], [0, 1], [0, 1.0]]))
    # 2-D: F point with a strong F neighbour that does connect into C_i.
    # Matrix rows: i=0 (F): a00=4, a01=-1 (C), a02=-1 (F), a03=-0.1 (weak C)
    #              k=2 (F): a21=-2 (C, in C_0), a20=-1, a22=5, a23=-1 (C, not in C_0)
    # C_0 = {1}; F_0 = {2}; W_0 = {3};  abar_21 = -2 -> denom = -2
    #   w_01 = -( -1 + (-1)(-2)/(-2) ) / (4 + (-0.1)) = -(-2)/3.9 = 2/3.9
    M = np.array([[4, -1, -1, -0.1],
                  [0, 1, 0, 0],
                  [-1, -2, 5, -1],
                  [0, 0, 0, 1.0]])
    A = sp.csr_matrix(M)
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    CF = np.array([-1, 1, -1, 1], np.int8)
    P = orc.interp(Ao, S, CF).scipy().toarray()
    assert P[0, 0] == pytest.approx(2 / 3.9, rel=1e-15)
    assert P[0, 1] == 0.0


def test_interp_reproduces_constants_on_zero_row_sums(orc):
    # graph Laplacian of a 2-D grid (zero row sums, Neumann): P 1 = 1 on
    # every F row with a nonempty interpolation set
    nx = 12
    T = sp.diags([-np.ones(nx - 1), -np.ones(nx - 1)], [-1, 1])
    L1 = sp.diags(np.asarray(-T.sum(1)).ravel()) + T
    A = (sp.kron(L1, sp.eye(nx)) + sp.kron(sp.eye(nx), L1)).tocsr()
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    nc, CF = orc.pmis(Ao, S, seed=3)
    P = orc.interp(Ao, S, CF).scipy()
    rows = np.diff(P.indptr) > 0
    s = np.asarray(P.sum(1)).ravel()
    assert rows.sum() > nc
    assert np.allclose(s[rows], 1.0, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- RAP
def test_rap_matches_dense_and_is_symmetric(orc):
    s = I.make_system(1, (9, 7))
    N = s.N
    A = s.scipy()[2 * N:, 2 * N:].tocsr()     # the ion block: symmetric SPD stencil
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    _, CF = orc.pmis(Ao, S)
    Po = orc.interp(Ao, S, CF)
    Ac = orc.rap(Ao, Po).scipy().toarray()
    P = Po.scipy().toarray()
    ref = P.T @ A.toarray() @ P
    assert np.allclose(Ac, ref, rtol=1e-13, atol=1e-13 * abs(ref).max())
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-14 * abs(Ac).max())


# ---------------------------------------------------------------- extended+i interpolation
def test_exti_reduces_to_classical_without_distance_two(orc):
    # 1-D Poisson with C = odd points: no F point has a strong F neighbour, so
    # the interpolatory sets are the direct C neighbours and w = 1/2, 1/2
    n = 15
    A = _tridiag(n)
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    CF = np.where(np.arange(n) % 2 == 1, 1, -1).astype(np.int8)
    assert np.array_equal(orc.interp_exti(Ao, S, CF).scipy().toarray(), orc.interp(Ao, S, CF).scipy().toarray())


def test_exti_hand_distance_two(orc):
    # chain 0(C) - 1(F) - 2(F) - 3(C), Poisson rows [-1 2 -1] (ends with 2 on the diagonal)
    # F point 1: C^_1 = {0} u {3} (3 is a strong C neighbour of its strong F neighbour 2)
    #   k = 2: d_2 = abar_21 (l = i) + abar_23 = -1 + -1 = -2
    #   num_0 = a_10 = -1; num_3 = 0 + a_12 abar_23 / d_2 = (-1)(-1)/(-2) = -1/2
    #   a~_11 = 2 + a_12 abar_21 / d_2 = 2 + (-1)(-1)/(-2) = 3/2
    #   w_10 = 1/(3/2) = 2/3, w_13 = (1/2)/(3/2) = 1/3   (linear interpolation)
    A = sp.csr_matrix(np.array([[2, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 2.0]]))
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    CF = np.array([1, -1, -1, 1], np.int8)
    P = orc.interp_exti(Ao, S, CF).scipy().toarray()
    assert np.allclose(P, np.array([[1, 0], [2 / 3, 1 / 3], [1 / 3, 2 / 3], [0, 1.0]]), rtol=1e-15, atol=0)


def test_exti_reproduces_constants_and_galerkin(orc):
    nx = 14
    T = sp.diags([-np.ones(nx - 1), -np.ones(nx - 1)], [-1, 1])
    L1 = sp.diags(np.asarray(-T.sum(1)).ravel()) + T
    A = (sp.kron(L1, sp.eye(nx)) + sp.kron(sp.eye(nx), L1)).tocsr()
    A.sort_indices()
    Ao = orc.Csr.from_scipy(A)
    S = orc.strength(Ao)
    nc, CF = orc.pmis(Ao, S, seed=5)
    Pe = orc.interp_exti(Ao, S, CF)
    P = Pe.scipy()
    rows = np.diff(P.indptr) > 0
    assert np.allclose(np.asarray(P.sum(1)).ravel()[rows], 1.0, rtol=0, atol=1e-13)
    # at least as many interpolation entries as the classical formula, and no empty F rows here
    Pc = orc.interp(Ao, S, CF).scipy()
    assert P.nnz >= Pc.nnz and rows.sum() >= (np.diff(Pc.indptr) > 0).sum()
    Pd = P.toarray()
    Ac = orc.rap(Ao, Pe).scipy().toarray()
    assert np.allclose(Ac, Pd.T @ A.toarray() @ Pd, rtol=0, atol=1e-12 * abs(Ac).max())


# ---------------------------------------------------------------- Gauss-Seidel order (smoother 1)
def _greedy_by_weight(adj, w):
    """Sequential greedy colouring, points taken by decreasing weight (ties: larger
    index first): the colouring Jones-Plassmann rounds produce on a symmetric graph."""
    n = len(adj)
    order = sorted(range(n), key=lambda i: (w[i], i), reverse=True)
    col = [-1] * n
    for i in order:
        used = {col[j] for j in adj[i] if col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


@pytest.mark.parametrize("n,density,sym,seed", [(60, 0.05, True, 1), (150, 0.03, True, 2), (120, 0.04, False, 3),
                                                (40, 0.5, True, 4)])
def test_colouring_is_greedy_by_weight_and_proper(orc, n, density, sym, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    if sym:
        M = M + M.T
    M = (M + sp.eye(n)).tocsr()
    M.sort_indices()
    level = seed % 3
    nc, col = orc.colour(orc.Csr.from_scipy(M), seed=7, level=level)
    Ms = ((M + M.T) != 0).tolil()
    adj = [[j for j in Ms.rows[i] if j != i] for i in range(n)]
    w = I.uniform(7, 2000 + level, n)
    assert list(col) == _greedy_by_weight(adj, w)
    assert nc == col.max() + 1
    for i in range(n):
        assert all(col[i] != col[j] for j in adj[i])


def _dense_m_matrix(n, seed):
    rng = np.random.default_rng(seed)
    B = -rng.uniform(0.5, 1.0, (n, n))
    A = (B + B.T) / 2
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, -A.sum(1) + 1.0)
    return A


def test_gs_vcycle_is_triangular_solves_on_a_complete_graph(orc):
    # every point its own colour: the C/F-ordered multicolour sweeps become
    # plain forward (down) and backward (up) Gauss-Seidel in the sweep order
    n = 130
    A = _dense_m_matrix(n, 5)
    As = sp.csr_matrix(A)
    As.sort_indices()
    h = orc.Amg(orc.Csr.from_scipy(As), orc.opts(smoother=1, max_levels=2))
    assert h.nlevels == 2 and h.coarse_is_lu
    key, nk = h.key(0)
    CF = h.CF(0)
    assert nk == n and sorted(key) == list(range(n))
    assert key[CF == 1].max() < key[CF == -1].min()        # C points are swept first
    perm = np.argsort(key)
    Ap = A[np.ix_(perm, perm)]
    b = np.random.default_rng(6).standard_normal(n)
    x = np.zeros(n)
    x[perm] = sla.solve_triangular(np.tril(Ap), b[perm], lower=True)
    r = b - A @ x
    P = h.P(0).scipy().toarray()
    Ac = h.A(1).scipy().toarray()
    x = x + P @ np.linalg.solve(Ac, P.T @ r)
    rp = (b - A @ x)[perm]
    x[perm] = x[perm] + sla.solve_triangular(np.triu(Ap), rp, lower=False)
    assert np.allclose(h.vcycle(b), x, rtol=1e-12, atol=1e-12 * abs(x).max())


def test_gs_vcycle_symmetric_and_adjoint(orc):
    # mirrored sweep orders make the cycle symmetric on a symmetric operator;
    # the transposed cycle is the adjoint on a nonsymmetric one
    rng = np.random.default_rng(9)
    T = sp.diags([-np.ones(29), 2 * np.ones(30), -np.ones(29)], [-1, 0, 1])
    A = (sp.kron(T, sp.eye(30)) + sp.kron(sp.eye(30), T)).tocsr()
    A.sort_indices()
    h = orc.Amg(orc.Csr.from_scipy(A), orc.opts(smoother=1, max_coarse=20))
    assert h.nlevels >= 3
    u, v = rng.standard_normal(900), rng.standard_normal(900)
    assert abs(h.vcycle(u) @ v - u @ h.vcycle(v)) <= 1e-13 * np.linalg.norm(u) * np.linalg.norm(v) * 10
    s = I.make_system(2, (12, 10), multigroup=True)
    hm = orc.Amg(orc.csr_of_system(s), orc.opts(smoother=1, max_coarse=20))
    u, v = rng.standard_normal(s.n), rng.standard_normal(s.n)
    lhs, rhs = hm.vcycle(u) @ v, u @ hm.vcycle(v, transpose=True)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(u) * np.linalg.norm(v) * 10
    assert abs(hm.vcycle(u) @ v - u @ hm.vcycle(v)) > 1e-8 * np.linalg.norm(u) * np.linalg.norm(v)


def test_gs_keys_on_a_hierarchy(orc):
    s = I.make_system(1, (24, 20), inclusion=True)
    h = orc.Amg(orc.csr_of_system(s), orc.opts(smoother=1))
    for l in range(h.nlevels - 1):
        key, nk = h.key(l)
        CF = h.CF(l)
        assert set(key) == set(range(nk))                   # no empty sweep
        assert key[CF == 1].max() < key[CF == -1].min()
        A = h.A(l).scipy().tocoo()
        off = A.row != A.col
        assert np.all(key[A.row[off]] != key[A.col[off]])    # a sweep's points are uncoupled
    assert h.key(h.nlevels - 1)[0] is None
