"""Pins of the oracle's option #4 (Section 3.5): the Schur complement whose
inner inverse is a single block -- S_I = A_I - D_IE A_E^-1 D_EI in Schur2,
C_E = A_E - D_EI A_I^-1 D_IE in Schur1 -- is inverted by K steps of
    w^(0) = 0,  w^(k+1) = A_a^-1 (q + D_ab A_b^-1 D_ba w^(k)).

With exact block inverses supplied through the oracle's callback, K steps
equal the truncated Neumann series sum_{k<K} (A_a^-1 D_ab A_b^-1 D_ba)^k A_a^-1,
built here with dense numpy matrices and plugged into the paper's own stage
list of Schur2 (Section 3.4's three steps) and Schur1 (its five steps); for
large K the preconditioner equals the one with the exact Schur complement
(the fixed point solves S w = q).  Inverse counts follow from the step
lists; with real V-cycles FGMRES converges to the dense solution."""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I


def _parts(s):
    A = s.scipy().toarray()
    N, G = s.N, s.G

    def blk(a, b):
        return A[a * N:(a + 1) * N, b * N:(b + 1) * N]

    def dg(a, b):
        return np.diag(np.diag(blk(a, b)))

    return A, blk, dg


def _cb_from(ops):
    def cb(op, comp, rhs):
        return np.linalg.solve(ops[(op, comp)], rhs)
    return cb


def _precond_matrix(apply, n):
    return np.column_stack([apply(np.eye(n)[:, k]) for k in range(n)])


def _neumann(Aa, Dab, Ab, Dba, K):
    inv = np.linalg.inv
    T = inv(Aa) @ Dab @ inv(Ab) @ Dba
    L = np.zeros_like(Aa)
    P = inv(Aa)
    for _ in range(K):
        L = L + P
        P = T @ P
    return L


def _schur2_ref(s, SI_inv, Sg_inv):
    """Section 3.4's Schur2 steps with given S_I^-1 and S_g^-1 (dense)."""
    A, blk, dg = _parts(s)
    N, G = s.N, s.G
    E, Ii = G, G + 1
    AEi = np.linalg.inv(blk(E, E))

    def apply(v):
        z = np.zeros_like(v)
        b = lambda a: v[a * N:(a + 1) * N]
        wEs = AEi @ b(E)
        for g in range(G):
            z[g * N:(g + 1) * N] = Sg_inv[g] @ (b(g) - dg(g, E) @ wEs)
        wI = SI_inv @ (b(Ii) - dg(Ii, E) @ wEs)
        z[Ii * N:(Ii + 1) * N] = wI
        acc = dg(E, Ii) @ wI
        for g in range(G):
            acc = acc + dg(E, g) @ z[g * N:(g + 1) * N]
        z[E * N:(E + 1) * N] = wEs - AEi @ acc
        return z
    return apply


def _schur1_ref(s, CE_inv, Cg_inv):
    """Section 3.4's Schur1 steps with given C_E^-1 and C_g^-1 (dense)."""
    A, blk, dg = _parts(s)
    N, G = s.N, s.G
    E, Ii = G, G + 1
    AIi = np.linalg.inv(blk(Ii, Ii))

    def apply(v):
        z = np.zeros_like(v)
        b = lambda a: v[a * N:(a + 1) * N]
        wIs = AIi @ b(Ii)
        wEs = CE_inv @ (b(E) - dg(E, Ii) @ wIs)
        for g in range(G):
            z[g * N:(g + 1) * N] = Cg_inv[g] @ (b(g) - dg(g, E) @ wEs)
        acc = np.zeros(N)
        for g in range(G):
            acc = acc + dg(E, g) @ z[g * N:(g + 1) * N]
        wE = wEs - CE_inv @ acc
        z[E * N:(E + 1) * N] = wE
        z[Ii * N:(Ii + 1) * N] = wIs - AIi @ (dg(Ii, E) @ wE)
        return z
    return apply


def _ops_schur2(s):
    A, blk, dg = _parts(s)
    G = s.G
    E, Ii = G, G + 1
    inv = np.linalg.inv
    ops = {(0, a): blk(a, a) for a in range(s.nc)}
    Sg = {g: blk(g, g) - dg(g, E) @ inv(blk(E, E)) @ dg(E, g) for g in range(G)}
    for g in range(G):
        ops[(3, g)] = Sg[g]
    return ops, Sg


@pytest.mark.parametrize("K", [1, 2, 5])
def test_schur2_option4_is_truncated_neumann_series(orc, K):
    s = I.make_system(3, (4, 3), multigroup=True, diffuse_E=True, seed=2)
    A, blk, dg = _parts(s)
    G = s.G
    E, Ii = G, G + 1
    ops, Sg = _ops_schur2(s)
    M = orc.Block(orc.csr_of_system(s), s.G, s.N, "schur2", orc.opts(opt4_steps=K))
    got = _precond_matrix(lambda v: M.apply(v, _cb_from(ops)), s.n)
    assert M.ninv == G + 2 * K + 1          # A_E twice, S_g G times, A_I K times, A_E K-1 more
    LK = _neumann(blk(Ii, Ii), dg(Ii, E), blk(E, E), dg(E, Ii), K)
    ref = _precond_matrix(_schur2_ref(s, LK, [np.linalg.inv(Sg[g]) for g in range(G)]), s.n)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    if K > 1:   # the series really moved: K steps differ from one step
        L1 = _neumann(blk(Ii, Ii), dg(Ii, E), blk(E, E), dg(E, Ii), 1)
        ref1 = _precond_matrix(_schur2_ref(s, L1, [np.linalg.inv(Sg[g]) for g in range(G)]), s.n)
        assert np.abs(ref1 - ref).max() > 1e-6 * np.abs(ref).max()


def test_schur2_option4_converges_to_exact_schur_complement(orc):
    s = I.make_system(2, (4, 3), multigroup=True, diffuse_E=True, seed=4)
    A, blk, dg = _parts(s)
    G = s.G
    E, Ii = G, G + 1
    ops, Sg = _ops_schur2(s)
    T = np.linalg.inv(blk(Ii, Ii)) @ dg(Ii, E) @ np.linalg.inv(blk(E, E)) @ dg(E, Ii)
    rho = max(abs(np.linalg.eigvals(T)))
    assert rho < 1                          # the recurrence contracts on these systems
    K = int(np.ceil(np.log(1e-16) / np.log(rho))) + 5
    M = orc.Block(orc.csr_of_system(s), s.G, s.N, "schur2", orc.opts(opt4_steps=K))
    got = _precond_matrix(lambda v: M.apply(v, _cb_from(ops)), s.n)
    SI = blk(Ii, Ii) - dg(Ii, E) @ np.linalg.inv(blk(E, E)) @ dg(E, Ii)
    ref = _precond_matrix(_schur2_ref(s, np.linalg.inv(SI), [np.linalg.inv(Sg[g]) for g in range(G)]), s.n)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    # and then the Schur2 error identity of Section 3.4 holds with this S_I
    Mm = np.linalg.inv(got)
    N = s.N
    AEi = np.linalg.inv(blk(E, E))
    Err = np.zeros_like(A)
    idx = list(range(G)) + [Ii]
    for i in idx:
        for j in idx:
            if i != j:
                Err[i * N:(i + 1) * N, j * N:(j + 1) * N] = -dg(i, E) @ AEi @ dg(E, j)
    assert np.allclose(A - Mm, Err, rtol=0, atol=1e-9 * abs(A).max())


@pytest.mark.parametrize("K", [1, 3])
def test_schur1_option4_for_c_e(orc, K):
    s = I.make_system(3, (4, 3), multigroup=True, diffuse_E=True, seed=6)
    A, blk, dg = _parts(s)
    G = s.G
    E, Ii = G, G + 1
    inv = np.linalg.inv
    ops = {(0, a): blk(a, a) for a in range(s.nc)}
    # C_g keeps its operator; here C_g = A_g - D_gE C_E^-1 D_Eg with the exact C_E
    CE = blk(E, E) - dg(E, Ii) @ inv(blk(Ii, Ii)) @ dg(Ii, E)
    Cg = {g: blk(g, g) - dg(g, E) @ inv(CE) @ dg(E, g) for g in range(G)}
    for g in range(G):
        ops[(2, g)] = Cg[g]
    M = orc.Block(orc.csr_of_system(s), s.G, s.N, "schur1", orc.opts(opt4_steps=K))
    got = _precond_matrix(lambda v: M.apply(v, _cb_from(ops)), s.n)
    assert M.ninv == G + 4 * K              # A_I twice, C_E twice by K + K-1 inverses, C_g G times
    LK = _neumann(blk(E, E), dg(E, Ii), blk(Ii, Ii), dg(Ii, E), K)
    ref = _precond_matrix(_schur1_ref(s, LK, [inv(Cg[g]) for g in range(G)]), s.n)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_option4_operators_and_fgmres(orc):
    """With real V-cycles: option #4 holds hierarchies of the plain blocks A_I
    (Schur2) and A_E (Schur1) instead of S_I-hat / C_E-hat, and FGMRES
    converges to the dense solution."""
    s = I.make_system(2, (8, 8), multigroup=True, diffuse_E=True)
    Ao = orc.csr_of_system(s)
    A, blk, dg = _parts(s)
    xs = np.linalg.solve(A, s.b)
    for kind, op_a, comp, missing in [("schur2", 0, s.G + 1, (4, s.G + 1)), ("schur1", 0, s.G, (1, s.G))]:
        M = orc.Block(Ao, s.G, s.N, kind, orc.opts(opt4_steps=3))
        assert M.amg(*missing) is None
        h = M.amg(op_a, comp)
        assert np.array_equal(h.A(0).scipy().toarray(), blk(comp, comp))
        x, it, rr, st, _ = orc.fgmres(Ao, s.b, M, tol=1e-12, maxit=2000)
        assert st == 0 and np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
        x1, it1, *_ = orc.fgmres(Ao, s.b, orc.Block(Ao, s.G, s.N, kind), tol=1e-12, maxit=2000)
        assert it <= it1 + 2                # at least as good as the diagonal approximation here
