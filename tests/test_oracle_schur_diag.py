"""Pin of the oracle's diagonal Schur-complement approximations (Section 3.5).

Section 3.5 replaces the Schur complements by operators whose correction
touches only the diagonal, because every coupling block D_ab is diagonal
(Eq. 2.2):
    S_g-hat = A_g - D_gE diag(A_E)^-1 D_Eg      (Schur2, each group g)
    S_I-hat = A_I - D_IE diag(A_E)^-1 D_EI      (Schur2)
and, "in exactly the same manner", for Schur1 (Section 3.4)
    C_E-hat = A_E - D_EI diag(A_I)^-1 D_IE
    C_g-hat = A_g - D_gE diag(C_E-hat)^-1 D_Eg  (each group g).

Each operator is rebuilt here with dense numpy matrices from the monolithic
matrix alone (blocks cut out by index, couplings as diagonal matrices, the
products written as the formulas print them) and compared entry by entry with
the level-0 operator of the hierarchy the oracle builds for that inverse.
The mutants below (a flipped sign, one coupling used twice, another group's
coupling, diag(A_E) in place of diag(C_E-hat), the unmodified block) each
differ from the correct operator by far more than the tolerance, so the
comparison would reject an oracle that computed any of them.
"""
import numpy as np
import pytest

from paper_2002_04958_gb300 import inputs as I


def _dense_blocks(s):
    A = s.scipy().toarray()
    N = s.N

    def blk(a, b):
        return A[a * N:(a + 1) * N, b * N:(b + 1) * N]

    def D(a, b):
        M = blk(a, b)
        assert np.count_nonzero(M - np.diag(np.diag(M))) == 0   # Eq. 2.2: couplings are diagonal
        return M

    def dinv(M):
        return np.diag(1.0 / np.diag(M))

    return A, blk, D, dinv


def _expected(s, kind):
    """{(op, comp): dense operator} from the Section 3.4/3.5 formulas."""
    A, blk, D, dinv = _dense_blocks(s)
    G = s.G
    E, Ii = G, G + 1
    out = {}
    if kind == "schur1":
        CE = blk(E, E) - D(E, Ii) @ dinv(blk(Ii, Ii)) @ D(Ii, E)
        out[(1, E)] = CE
        for g in range(G):
            out[(2, g)] = blk(g, g) - D(g, E) @ dinv(CE) @ D(E, g)
    else:
        for g in range(G):
            out[(3, g)] = blk(g, g) - D(g, E) @ dinv(blk(E, E)) @ D(E, g)
        out[(4, Ii)] = blk(Ii, Ii) - D(Ii, E) @ dinv(blk(E, E)) @ D(E, Ii)
    return out


def _mutants(s, kind):
    """Plausible mistakes, keyed like _expected."""
    A, blk, D, dinv = _dense_blocks(s)
    G = s.G
    E, Ii = G, G + 1
    m = []
    if kind == "schur1":
        CE = blk(E, E) - D(E, Ii) @ dinv(blk(Ii, Ii)) @ D(Ii, E)
        m.append(("sign of the E correction", (1, E), blk(E, E) + D(E, Ii) @ dinv(blk(Ii, Ii)) @ D(Ii, E)))
        m.append(("E block unmodified", (1, E), blk(E, E)))
        m.append(("diag(A_I) replaced by diag(A_E)", (1, E), blk(E, E) - D(E, Ii) @ dinv(blk(E, E)) @ D(Ii, E)))
        for g in range(G):
            m.append((f"group {g}: diag(A_E) in place of diag(C_E-hat)", (2, g),
                      blk(g, g) - D(g, E) @ dinv(blk(E, E)) @ D(E, g)))
            m.append((f"group {g}: D_gE used twice", (2, g), blk(g, g) - D(g, E) @ dinv(CE) @ D(g, E)))
            m.append((f"group {g}: D_Eg used twice", (2, g), blk(g, g) - D(E, g) @ dinv(CE) @ D(E, g)))
            m.append((f"group {g}: sign", (2, g), blk(g, g) + D(g, E) @ dinv(CE) @ D(E, g)))
            h = (g + 1) % G
            if h != g:
                m.append((f"group {g}: coupling of group {h}", (2, g),
                          blk(g, g) - D(h, E) @ dinv(CE) @ D(E, h)))
    else:
        AE = blk(E, E)
        for g in range(G):
            m.append((f"group {g}: sign", (3, g), blk(g, g) + D(g, E) @ dinv(AE) @ D(E, g)))
            m.append((f"group {g}: D_gE used twice", (3, g), blk(g, g) - D(g, E) @ dinv(AE) @ D(g, E)))
            m.append((f"group {g}: unmodified", (3, g), blk(g, g)))
        m.append(("I: diag(A_I) in place of diag(A_E)", (4, Ii),
                  blk(Ii, Ii) - D(Ii, E) @ dinv(blk(Ii, Ii)) @ D(E, Ii)))
        m.append(("I: sign", (4, Ii), blk(Ii, Ii) + D(Ii, E) @ dinv(AE) @ D(E, Ii)))
        m.append(("I: unmodified", (4, Ii), blk(Ii, Ii)))
    return m


def _tol(M):
    return 1e-15 * max(abs(M).max(), 1.0) * 4


@pytest.mark.parametrize("kind", ["schur1", "schur2"])
@pytest.mark.parametrize("G,diffuse_E", [(3, True), (3, False), (1, True)])
def test_diagonal_schur_operators_match_section_3_5(orc, kind, G, diffuse_E):
    s = I.make_system(G, (6, 5), multigroup=G > 1, diffuse_E=diffuse_E, seed=3)
    Ao = orc.csr_of_system(s)
    M = orc.Block(Ao, s.G, s.N, kind)
    exp = _expected(s, kind)
    got = {}
    for (op, comp), want in exp.items():
        h = M.amg(op, comp)
        assert h is not None, (op, comp)
        Ag = h.A(0).scipy().toarray()
        got[(op, comp)] = Ag
        # same pattern as the block (only the diagonal changes), same values
        assert Ag.shape == want.shape
        err = abs(Ag - want).max()
        assert err <= _tol(want), (kind, op, comp, err)
        assert np.any(np.diag(Ag) != np.diag(np.asarray(s.scipy().toarray())[comp * s.N:(comp + 1) * s.N,
                                                                                  comp * s.N:(comp + 1) * s.N]))
    # each plausible mistake would have been rejected by the comparison above
    for name, key, mut in _mutants(s, kind):
        gap = abs(mut - exp[key]).max()
        assert gap > 1e3 * _tol(exp[key]), (name, gap)
        assert abs(got[key] - mut).max() > 1e3 * _tol(exp[key]), name


def test_schur1_ce_hat_is_exact_schur_complement_when_a_i_is_diagonal(orc):
    """With A_I diagonal, diag(A_I)^-1 = A_I^-1, so C_E-hat is the exact Schur
    complement A_E - D_EI A_I^-1 D_IE (checked through an exact inverse, not
    through the diagonal formula)."""
    s = I.make_system(2, (5, 4), multigroup=True, diffuse_E=True, seed=5)
    A, blk, D, _ = _dense_blocks(s)
    E, Ii = s.G, s.G + 1
    # make A_I diagonal: drop its off-diagonal stencil entries from the monolithic matrix
    import scipy.sparse as sp
    Am = s.scipy().tolil()
    for k in range(s.N):
        i = Ii * s.N + k
        for j in list(Am.rows[i]):
            if j != i and j // s.N == Ii:
                Am[i, j] = 0.0
    Am = Am.tocsr()
    Am.eliminate_zeros()
    Am.sort_indices()
    from oracle import oracle as orc_mod
    Ao = orc_mod.Csr.from_scipy(Am)
    M = orc.Block(Ao, s.G, s.N, "schur1")
    Ad = Am.toarray()
    blk2 = lambda a, b: Ad[a * s.N:(a + 1) * s.N, b * s.N:(b + 1) * s.N]
    AI = blk2(Ii, Ii)
    assert np.count_nonzero(AI - np.diag(np.diag(AI))) == 0
    exact = blk2(E, E) - blk2(E, Ii) @ np.linalg.inv(AI) @ blk2(Ii, E)
    h = M.amg(1, E)
    if h is None:   # option #1 (Jacobi) when C_E-hat is diagonal; E diffuses here, so it is not
        pytest.fail("C_E-hat has no hierarchy")
    got = h.A(0).scipy().toarray()
    assert abs(got - exact).max() <= 1e-13 * abs(exact).max()
    assert sp.issparse(Am)
