"""Pins of the oracle's extended+i interpolation (Sec. 2.3, the distance-two formula).

Each check compares the oracle with something other than itself: closed-form linear
interpolation on the 1-D Laplacian (which the formula reproduces exactly when every F run
between C points is at most two long), a hand-worked example with weak and positive
couplings, constant preservation on zero-row-sum M-matrices (a consequence of the formula
derived in the docstring), the interpolatory set computed by sparse-matrix algebra, and the
complexities the paper prints for its 7-point Poisson run (Table 2).
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr


def dense_P(rp, ci, v, n, nc):
    P = np.zeros((n, nc))
    for i in range(n):
        P[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return P


@pytest.mark.parametrize("cf", [[1, 0, 0, 1, 0, 1, 0, 0, 1],
                                [0, 1, 0, 0, 1, 0, 0, 1, 0, 1, 0],
                                [1, 0, 1, 0, 0, 1, 0, 0, 1, 0, 1]])
def test_ext_1d_laplacian_is_linear_interpolation(cf):
    """1-D Laplacian (2, -1), every coupling strong, F runs of length <= 2: each F point's
    interpolatory set is its two bracketing C points and the weights are exactly those of
    linear interpolation (e.g. C F F C: 2/3, 1/3).  Ends bracketed on one side take weight 1
    on the one C point that reaches them (the Dirichlet zero does not enter)."""
    n = len(cf)
    A = pr.poisson1d(n)
    S = O.strength(A, 0.25)
    cf = np.array(cf, np.int8)
    rp, ci, v, nc = O.ext_interp(A, S, cf)
    P = dense_P(rp, ci, v, n, nc)
    C = list(np.where(cf)[0])
    coarse = {c: J for J, c in enumerate(C)}
    for i in range(n):
        if cf[i]:
            assert P[i].tolist() == [1.0 if J == coarse[i] else 0.0 for J in range(nc)]
            continue
        left = max([c for c in C if c < i], default=None)
        right = min([c for c in C if c > i], default=None)
        want = np.zeros(nc)
        # the grid extends to virtual Dirichlet points -1 and n (value zero)
        lo = left if left is not None else -1
        hi = right if right is not None else n
        if left is not None:
            want[coarse[left]] = float(Fraction(hi - i, hi - lo))
        if right is not None:
            want[coarse[right]] = float(Fraction(i - lo, hi - lo))
        assert np.allclose(P[i], want, rtol=2e-16, atol=0), (i, P[i], want)


def test_ext_without_strong_f_neighbours():
    """No strong F neighbour: w_ij = -a_ij / (a_ii + sum of the weak couplings outside
    Chat_i), j in C_i^S.  Row 0: a00 = 5; -2 to C point 1 (strong), -0.25 to C point 3
    (weak), +0.5 to F point 4 (weak, positive): Chat_0 = {1}; at = 5 - 0.25 + 0.5 = 5.25;
    w_01 = 2 / 5.25 = 8/21."""
    d = np.diag([5.0, 3.0, 3.0, 3.0, 3.0])
    for j, a in ((1, -2.0), (3, -0.25), (4, 0.5)):
        d[0, j] = d[j, 0] = a
    A = pr.dense_to_csr(d)
    S = O.strength(A, 0.25)
    cf = np.array([0, 1, 0, 1, 0], np.int8)
    rp, ci, v, nc = O.ext_interp(A, S, cf)
    assert list(ci[rp[0]:rp[1]]) == [0]
    assert v[rp[0]] == pytest.approx(8.0 / 21.0, rel=2e-16)


def test_ext_distance_two_hand_example():
    """Row 0 couples strongly to C point 1 (-2) and F point 2 (-1); point 2 couples strongly to
    C point 3 (-1) and to 0.  Chat_0 = {1, 3}.  d_2 = a_20 + a_23 = -2 (l in Chat_0 u {0});
    at = a_00 + a_02 abar_20 / d_2 = 4 + (-1)(-1)/(-2) = 3.5;
    w_01 = -(a_01 + 0) / 3.5 = 4/7;  w_03 = -(0 + a_02 abar_23 / d_2) / 3.5 = -(-0.5)/3.5 = 1/7."""
    d = np.diag([4.0, 4.0, 4.0, 4.0])
    for (i, j, a) in ((0, 1, -2.0), (0, 2, -1.0), (2, 3, -1.0)):
        d[i, j] = d[j, i] = a
    A = pr.dense_to_csr(d)
    S = O.strength(A, 0.25)
    cf = np.array([0, 1, 0, 1], np.int8)
    rp, ci, v, nc = O.ext_interp(A, S, cf)
    assert list(ci[rp[0]:rp[1]]) == [0, 1]
    assert v[rp[0]] == pytest.approx(4.0 / 7.0, rel=2e-16)
    assert v[rp[0] + 1] == pytest.approx(1.0 / 7.0, rel=2e-16)


def _zero_rowsum_m_matrix(n, seed):
    rng = np.random.default_rng(seed)
    d = np.zeros((n, n))
    for i in range(n):
        for j in rng.choice(n, 4, replace=False):
            if i != j:
                d[i, j] = d[j, i] = -rng.uniform(0.05, 1.0)
    np.fill_diagonal(d, -d.sum(axis=1))
    keep = np.diag(d) > 0
    return pr.dense_to_csr(d[np.ix_(keep, keep)])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ext_preserves_constants(seed):
    """Zero row sums and non-positive couplings give sum_j w_ij = 1: with
    d_k = sum_{j in Chat_i} abar_kj + abar_ki, the numerators sum to
    sum_{Chat_i} a_ij + sum_k a_ik - sum_k a_ik abar_ki / d_k = -at."""
    A = _zero_rowsum_m_matrix(120, seed)
    S = O.strength(A, 0.25)
    cf = O.pmis(A, S, seed, 0)
    rp, ci, v, nc = O.ext_interp(A, S, cf)
    checked = 0
    for i in range(A.n):
        if not cf[i] and rp[i + 1] > rp[i]:
            assert abs(v[rp[i]:rp[i + 1]].sum() - 1.0) < 1e-13
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("make", [lambda: pr.poisson3d(7), lambda: pr.diffusion3d(7, 2.0, 5)[0],
                                  lambda: pr.graph_laplacian_spd(300, 6, 0.05, 4)])
def test_ext_interpolatory_set_by_matrix_algebra(make):
    """The pattern of P's F rows is Chat = pattern(S_C + S_F S_C), S_C / S_F the strong
    couplings to C / F points (off-diagonal)."""
    A = make()
    S = O.strength(A, 0.25)
    cf = O.pmis(A, S, 1, 0)
    rp, ci, v, nc = O.ext_interp(A, S, cf)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    strong = S.astype(bool) & (rows != A.col)
    isC = cf[A.col].astype(bool)
    SC = sp.csr_matrix((np.ones(int((strong & isC).sum())), (rows[strong & isC], A.col[strong & isC])), (A.n, A.n))
    SF = sp.csr_matrix((np.ones(int((strong & ~isC).sum())), (rows[strong & ~isC], A.col[strong & ~isC])), (A.n, A.n))
    Chat = (SC + SF @ SC).tocsr()
    Cidx = np.cumsum(cf) - 1
    for i in range(A.n):
        got = ci[rp[i]:rp[i + 1]].tolist()
        if cf[i]:
            assert got == [Cidx[i]]
        else:
            want = sorted(Cidx[np.unique(Chat.indices[Chat.indptr[i]:Chat.indptr[i + 1]])].tolist())
            assert got == want


def test_ext_hierarchy_solves_and_converges_faster():
    p = pr.config2(24)
    its = {}
    for it in ("direct", "ext"):
        h = O.Hierarchy(p.A, interp=it)
        st, x, k, _, _ = h.pcg(p.b, rtol=1e-8)
        assert st == 0
        assert np.linalg.norm(x - p.xstar) <= 1e-6 * np.linalg.norm(p.xstar)
        its[it] = k
    assert its["ext"] < its["direct"]


def test_ext_pcg_matches_dense_solve():
    A = pr.diffusion3d(7, 2.0, 6)[0]
    b = pr.uniform(A.n, 9)
    h = O.Hierarchy(A, seed=2, interp="ext")
    st, x, it, _, _ = h.pcg(b, rtol=1e-12, maxit=200)
    assert st == 0
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_ext_complexities_match_the_papers_poisson_run():
    """Table 2, poi65m (7-point Poisson, theta = 0.25, PMIS, extended+i): C_gd = 1.327,
    C_op = 4.036.  The same set-up on a 40^3 grid lands within a few percent of both."""
    h = O.Hierarchy(pr.poisson3d(40), interp="ext")
    cgd, cop = h.complexities()
    assert abs(cgd - 1.327) <= 0.05 * 1.327
    assert abs(cop - 4.036) <= 0.06 * 4.036


def test_ext_rejects_block_systems():
    A = pr.kron_identity(pr.poisson3d(4), 3)
    with pytest.raises(RuntimeError):
        O.Hierarchy(A, block_size=3, interp="ext")
