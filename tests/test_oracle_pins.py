"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks one oracle function against something other than itself:
published test vectors, closed forms, hand-worked examples, invariants, or a
brute-force dense evaluation of the paper's defining formula.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_dense(d):
    return pr.dense_to_csr(np.asarray(d, dtype=np.float64))


# ---------------------------------------------------------------- RNG ----

def test_splitmix64_published_vector():
    """SplitMix64 seeded with 1234567: first outputs of the published generator."""
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    assert [O.splitmix64(1234567, c) for c in range(1, 6)] == vals


def test_pmis_random_range_and_counter():
    u = [O.pmis_random(7, 0, i) for i in range(1000)]
    assert all(0.0 <= x < 1.0 for x in u)
    assert len(set(u)) == 1000
    # level k uses counter (k << 32) + i + 1
    assert O.pmis_random(7, 3, 5) == (O.splitmix64(7, (3 << 32) + 6) >> 11) * 2.0 ** -53


# ---------------------------------------------------------- generators ----

@pytest.mark.parametrize("N", [1, 2, 5, 64])
def test_poisson2d_nnz_closed_form(N):
    A = pr.poisson2d(N)
    assert A.nnz == pr.nnz_poisson2d(N)
    assert O.check_csr(A) == 0


@pytest.mark.parametrize("N", [1, 3, 8, 32])
def test_poisson3d_nnz_closed_form(N):
    A = pr.poisson3d(N)
    assert A.nnz == pr.nnz_poisson3d(N)
    assert O.check_csr(A) == 0


def test_config_sizes():
    assert pr.nnz_poisson2d(64) == 20224
    assert pr.nnz_poisson3d(128) == 14581760
    assert pr.nnz_poisson3d(256) == 117047296
    assert pr.config1().A.nnz == 20224


def test_diffusion_unit_coefficient_is_poisson():
    k = np.ones((6, 6, 6))
    A = pr.diffusion3d_from_k(k)
    B = pr.poisson3d(6)
    assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)


def test_diffusion_symmetric_spd():
    A, _ = pr.diffusion3d(6, 2.0, 2)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0


# ------------------------------------------------------------ strength ----

def test_strength_hand_example():
    # row 0: diag 4, off-diagonals -1, -0.2, -0.5, +0.3  (theta = 0.25, m = 1)
    d = np.array([[4.0, -1.0, -0.2, -0.5, 0.3],
                  [-1.0, 4.0, 0.0, 0.0, 0.0],
                  [-0.2, 0.0, 4.0, 0.0, 0.0],
                  [-0.5, 0.0, 0.0, 4.0, -2.0],
                  [0.3, 0.0, 0.0, -2.0, 4.0]])
    A = csr_from_dense(d)
    S = O.strength(A, 0.25)
    strong = {(i, int(A.col[p])) for i in range(A.n) for p in range(A.rowptr[i], A.rowptr[i + 1]) if S[p]}
    # row 0: -1 and -0.5 reach 0.25; row 1: its only neighbour; row 2 likewise;
    # row 3: m = 2, threshold 0.5: -0.5 ties exactly (>= keeps it), -2 strong;
    # row 4: +0.3 is never strong, -2 is.
    assert strong == {(0, 1), (0, 3), (1, 0), (2, 0), (3, 0), (3, 4), (4, 3)}


def test_strength_positive_offdiagonals_only():
    A = csr_from_dense([[2.0, 0.5], [0.5, 2.0]])
    assert O.strength(A, 0.25).sum() == 0


def test_strength_constant_coefficient_all_strong():
    for A in (pr.poisson2d(7), pr.poisson3d(5)):
        S = O.strength(A, 0.25)
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        assert np.array_equal(S.astype(bool), rows != A.col)


# ---------------------------------------------------------------- PMIS ----

def _strong_sets(A, S):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    Si = [set() for _ in range(A.n)]
    STi = [set() for _ in range(A.n)]
    for r, c, s in zip(rows, A.col, S):
        if s:
            Si[r].add(int(c))
            STi[int(c)].add(int(r))
    return Si, STi


def check_pmis_invariants(A, S, cf):
    Si, STi = _strong_sets(A, S)
    for i in range(A.n):
        if cf[i]:
            # (i) no two C points are strongly connected both ways, and on a
            # symmetric strength graph not at all.  (With an asymmetric graph a
            # C point may depend on a later C point that it beat earlier: the
            # F step only reaches points that depend on a new C point.)
            assert not any(cf[j] for j in Si[i] & STi[i])
            if all(Si[j] == STi[j] for j in range(A.n)):
                assert not any(cf[j] for j in Si[i] | STi[i])
        else:
            # (ii) an F point influenced nobody or depends on a C point
            assert len(STi[i]) == 0 or any(cf[j] for j in Si[i])


@pytest.mark.parametrize("make", [lambda: pr.poisson1d(50), lambda: pr.poisson2d(17), lambda: pr.poisson3d(7),
                                  lambda: pr.graph_laplacian_spd(200, 6, 0.1, 5),
                                  lambda: pr.diffusion3d(8, 2.0, 3)[0]])
def test_pmis_invariants(make):
    A = make()
    S = O.strength(A, 0.25)
    for seed in (0, 1, 99):
        cf = O.pmis(A, S, seed, 0)
        check_pmis_invariants(A, S, cf)
        assert np.array_equal(cf, O.pmis(A, S, seed, 0))  # (iii) deterministic
    assert not np.array_equal(O.pmis(A, S, 0, 0), O.pmis(A, S, 1, 0))


def test_pmis_1d_small_cases():
    # 1-D Poisson, n = 3: the middle point influences two points, the ends one
    A = pr.poisson1d(3)
    S = O.strength(A, 0.25)
    for seed in range(5):
        assert list(O.pmis(A, S, seed, 0)) == [0, 1, 0]
    # 1-D Poisson: no two adjacent C points; every F point has a C neighbour
    A = pr.poisson1d(101)
    cf = O.pmis(A, O.strength(A, 0.25), 3, 0)
    assert not np.any(cf[:-1] & cf[1:])
    for i in np.where(cf == 0)[0]:
        assert (i > 0 and cf[i - 1]) or (i < 100 and cf[i + 1])


def test_pmis_star_graph():
    # the centre influences 6 leaves (lambda >= 6), each leaf one point
    d = np.eye(7) * 7.0
    d[0, 1:] = d[1:, 0] = -1.0
    A = csr_from_dense(d)
    S = O.strength(A, 0.25)
    for seed in range(4):
        assert list(O.pmis(A, S, seed, 0)) == [1, 0, 0, 0, 0, 0, 0]


def test_pmis_isolated_points_are_fine():
    A = csr_from_dense(np.diag([1.0, 2.0, 3.0]))
    S = O.strength(A, 0.25)
    assert list(O.pmis(A, S, 0, 0)) == [0, 0, 0]


# -------------------------------------------------------- interpolation ----

def alternating_cf(n):
    return np.array([i % 2 for i in range(n)], dtype=np.int8)  # C at odd indices


def test_direct_interp_1d_alternating_halves():
    n = 15
    A = pr.poisson1d(n)
    S = O.strength(A, 0.25)
    rp, ci, v, nc = O.direct_interp(A, S, alternating_cf(n))
    assert nc == 7
    P = np.zeros((n, nc))
    for i in range(n):
        P[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    expect = np.zeros((n, nc))
    for J in range(nc):
        expect[2 * J + 1, J] = 1.0
        expect[2 * J, J] = 0.5
        expect[2 * J + 2, J] = 0.5
    assert np.array_equal(P, expect)


def test_direct_interp_hand_example():
    # row 0: a00 = 5; -2 (C, strong), -1 (F, strong), -0.25 (C, weak), +0.5 (C)
    # S_0 = {1, 2}, P_0 = {1}; sum_N a^- = -3.25, sum_P a^- = -2, alpha = 1.625,
    # no positive entry in P_0 so at = 5 + 0.5 = 5.5;  w_01 = 3.25 / 5.5 = 13/22.
    d = np.diag([5.0, 3.0, 3.0, 3.0, 3.0])
    for j, a in ((1, -2.0), (2, -1.0), (3, -0.25), (4, 0.5)):
        d[0, j] = d[j, 0] = a
    A = csr_from_dense(d)
    S = O.strength(A, 0.25)
    cf = np.array([0, 1, 0, 1, 1], dtype=np.int8)
    rp, ci, v, nc = O.direct_interp(A, S, cf)
    assert nc == 3
    assert list(ci[rp[0]:rp[1]]) == [0]
    assert abs(v[rp[0]] - 13.0 / 22.0) <= 2e-16
    # C rows are unit rows into the ascending coarse numbering
    for i, J in ((1, 0), (3, 1), (4, 2)):
        assert list(ci[rp[i]:rp[i + 1]]) == [J] and v[rp[i]] == 1.0
    # F row 2 depends only on point 0, which is F: empty row
    assert rp[3] - rp[2] == 0


def _zero_rowsum_mixed_sign(n, seed):
    rng = np.random.default_rng(seed)
    d = np.zeros((n, n))
    for i in range(n):
        for j in rng.choice(n, 4, replace=False):
            if i != j:
                w = -rng.uniform(0.2, 1.0) if rng.uniform() < 0.8 else rng.uniform(0.05, 0.3)
                d[i, j] = d[j, i] = w
    np.fill_diagonal(d, 0.0)
    np.fill_diagonal(d, -d.sum(axis=1))
    return d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_direct_interp_preserves_constants(seed):
    """Zero row sum  =>  interpolation weights of an F row sum to one (both branches)."""
    d = _zero_rowsum_mixed_sign(80, seed)
    keep = np.diag(d) > 0
    d = d[np.ix_(keep, keep)]
    A = csr_from_dense(d)
    S = O.strength(A, 0.25)
    cf = O.pmis(A, S, seed, 0)
    rp, ci, v, nc = O.direct_interp(A, S, cf)
    rowsum = np.abs(d.sum(axis=1)) <= 1e-14 * np.abs(d).max()
    checked = 0
    for i in range(A.n):
        if not cf[i] and rp[i + 1] > rp[i] and rowsum[i]:
            assert abs(v[rp[i]:rp[i + 1]].sum() - 1.0) < 1e-13
            checked += 1
    assert checked > 10


# ------------------------------------------------------------- Galerkin ----

def _dense_P(rp, ci, v, n, nc):
    P = np.zeros((n, nc))
    for i in range(n):
        P[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return P


def test_galerkin_1d_alternating_exact():
    n = 31
    A = pr.poisson1d(n)
    rp, ci, v, nc = O.direct_interp(A, O.strength(A, 0.25), alternating_cf(n))
    crp, cci, cv = O.galerkin(A, rp, ci, v, nc)
    Ac = np.zeros((nc, nc))
    for I in range(nc):
        Ac[I, cci[crp[I]:crp[I + 1]]] = cv[crp[I]:crp[I + 1]]
    expect = np.diag(np.ones(nc)) - 0.5 * (np.eye(nc, k=1) + np.eye(nc, k=-1))
    assert np.array_equal(Ac, expect)


@pytest.mark.parametrize("make", [lambda: pr.poisson2d(12), lambda: pr.graph_laplacian_spd(150, 5, 0.2, 1),
                                  lambda: pr.diffusion3d(6, 2.0, 4)[0]])
def test_galerkin_brute_force(make):
    A = make()
    S = O.strength(A, 0.25)
    cf = O.pmis(A, S, 11, 0)
    rp, ci, v, nc = O.direct_interp(A, S, cf)
    crp, cci, cv = O.galerkin(A, rp, ci, v, nc)
    P = _dense_P(rp, ci, v, A.n, nc)
    D = A.to_dense()
    dense = P.T @ D @ P
    pattern = (np.abs(P).T @ (D != 0).astype(float) @ (np.abs(P) > 0).astype(float)) != 0
    got = np.zeros((nc, nc))
    got_pat = np.zeros((nc, nc), bool)
    for I in range(nc):
        cols = cci[crp[I]:crp[I + 1]]
        assert np.all(np.diff(cols) > 0)
        got[I, cols] = cv[crp[I]:crp[I + 1]]
        got_pat[I, cols] = True
    assert np.array_equal(got_pat, pattern)
    scale = np.abs(dense).max()
    assert np.abs(got - dense).max() <= 1e-13 * scale
    # energy identity x_c^T A_c x_c = (P x_c)^T A (P x_c), symmetry, SPD
    rng = np.random.default_rng(0)
    for _ in range(3):
        xc = rng.standard_normal(nc)
        lhs, rhs = xc @ got @ xc, (P @ xc) @ D @ (P @ xc)
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    assert np.abs(got - got.T).max() <= 1e-14 * scale
    assert np.linalg.eigvalsh(got).min() > 0


# ------------------------------------------------- Cholesky / SpMV / Jacobi ----

def test_cholesky_and_solve():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((40, 40))
    M = M @ M.T + 40 * np.eye(40)
    L = O.cholesky(M)
    assert np.allclose(L, np.linalg.cholesky(M), rtol=0, atol=1e-12 * np.abs(L).max())
    y = rng.standard_normal(40)
    assert np.allclose(O.cholesky_solve(L, y), np.linalg.solve(M, y), rtol=1e-12, atol=1e-14)


def test_cholesky_rejects_indefinite():
    with pytest.raises(RuntimeError):
        O.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_spmv_dense():
    A = pr.graph_laplacian_spd(90, 5, 0.3, 2)
    x = np.random.default_rng(1).standard_normal(A.n)
    assert np.allclose(O.spmv(A, x), A.to_dense() @ x, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("k,l", [(1, 1), (3, 5), (9, 9)])
def test_jacobi_on_2d_poisson_eigenvectors(k, l):
    N, omega = 9, 2.0 / 3.0
    A = pr.poisson2d(N)
    xs = np.arange(1, N + 1)
    v = np.outer(np.sin(l * np.pi * xs / (N + 1)), np.sin(k * np.pi * xs / (N + 1))).reshape(-1)
    lam = 4 - 2 * np.cos(k * np.pi / (N + 1)) - 2 * np.cos(l * np.pi / (N + 1))
    s = O.jacobi_sweep(A, omega, np.zeros(A.n), v)
    assert np.allclose(s, (1 - omega * lam / 4) * v, rtol=0, atol=1e-14)


def test_jacobi_on_1d_poisson_eigenvectors():
    n, omega = 20, 2.0 / 3.0
    A = pr.poisson1d(n)
    for k in (1, 7, 20):
        v = np.sin(k * np.pi * np.arange(1, n + 1) / (n + 1))
        lam = 2 - 2 * np.cos(k * np.pi / (n + 1))
        s = O.jacobi_sweep(A, omega, np.zeros(n), v)
        assert np.allclose(s, (1 - omega * lam / 2) * v, rtol=0, atol=1e-14)


# ------------------------------------------------------------- V-cycle ----

def _dense_hierarchy(h):
    As, Ps = [], []
    for k in range(h.nlevels):
        rp, ci, v = h.A(k)
        n = len(rp) - 1
        D = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(rp))
        D[rows, ci] = v
        As.append(D)
        if k < h.nlevels - 1:
            prp, pci, pv = h.P(k)
            nc = h.level_sizes(k + 1)[0]
            Ps.append(_dense_P(prp, pci, pv, n, nc))
    return As, Ps


def _dense_vcycle_operator(A0, Ps, omega, nu1, nu2):
    """B_k = (I - E_k) A_k^{-1},  E_k = S^nu2 (I - P B_{k+1} P^T A_k) S^nu1  (Eq. twoGridOp,
    with the coarse inverse replaced recursively by the coarse V-cycle); A_{k+1} = P^T A_k P."""
    A = A0
    if not Ps:
        return np.linalg.inv(A)
    P = Ps[0]
    Bc = _dense_vcycle_operator(P.T @ A @ P, Ps[1:], omega, nu1, nu2)
    n = A.shape[0]
    S = np.eye(n) - omega * np.diag(1.0 / np.diag(A)) @ A
    E = np.linalg.matrix_power(S, nu2) @ (np.eye(n) - P @ Bc @ P.T @ A) @ np.linalg.matrix_power(S, nu1)
    return (np.eye(n) - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("make,levels,nu", [
    (lambda: pr.poisson1d(31), 2, (1, 1)),
    (lambda: pr.poisson2d(10), 2, (1, 1)),
    (lambda: pr.poisson2d(10), 2, (2, 1)),
    (lambda: pr.graph_laplacian_spd(60, 5, 0.2, 7), 2, (1, 2)),
    (lambda: pr.poisson2d(16), 4, (1, 1)),
    (lambda: pr.diffusion3d(6, 2.0, 8)[0], 3, (1, 1)),
])
def test_vcycle_matches_dense_operator(make, levels, nu):
    A = make()
    omega = 2.0 / 3.0
    h = O.Hierarchy(A, seed=5, max_coarse=4, max_levels=levels, nu1=nu[0], nu2=nu[1])
    assert h.nlevels == levels
    As, Ps = _dense_hierarchy(h)
    B = _dense_vcycle_operator(As[0], Ps, omega, *nu)
    got = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.abs(got - B).max() <= 1e-10 * np.abs(B).max()


def test_vcycle_symmetric_positive():
    A = pr.poisson2d(24)
    h = O.Hierarchy(A, seed=1)
    rng = np.random.default_rng(2)
    for _ in range(4):
        u, w = rng.standard_normal(A.n), rng.standard_normal(A.n)
        a, b = u @ h.vcycle(w), w @ h.vcycle(u)
        assert abs(a - b) <= 1e-12 * abs(a) + 1e-14
        assert u @ h.vcycle(u) > 0


# ----------------------------------------------------------------- PCG ----

@pytest.mark.parametrize("make", [lambda: pr.poisson1d(200), lambda: pr.poisson2d(20),
                                  lambda: pr.graph_laplacian_spd(300, 6, 0.05, 3),
                                  lambda: pr.diffusion3d(7, 2.0, 6)[0]])
@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_matches_dense_solve(make, flexible):
    A = make()
    b = pr.uniform(A.n, 9)
    h = O.Hierarchy(A, seed=2)
    st, x, it, hist, _ = h.pcg(b, rtol=1e-12, maxit=200, flexible=flexible)
    assert st == 0 and it > 0
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert hist[-1] < 1e-12 * np.linalg.norm(b) and hist[0] == pytest.approx(np.linalg.norm(b))
    # the recursive residual tracks the true one
    assert np.linalg.norm(b - A.to_dense() @ x) <= 1e-10 * np.linalg.norm(b)


def test_pcg_a_norm_error_monotone():
    A = pr.diffusion3d(7, 2.0, 1)[0]
    D = A.to_dense()
    b = pr.uniform(A.n, 4)
    xs = np.linalg.solve(D, b)
    h = O.Hierarchy(A, seed=3)
    for precond in (True, False):
        st, x, it, hist, xh = h.pcg(b, rtol=1e-10, maxit=400, precond=precond, keep_iterates=True)
        assert st == 0
        errs = [np.sqrt((xs - xk) @ D @ (xs - xk)) for xk in xh]
        e0 = np.sqrt(xs @ D @ xs)
        errs = [e0] + errs
        for a, c in zip(errs, errs[1:]):
            assert c <= a * (1 + 1e-12) + 1e-14 * e0


def test_cg_finite_termination_in_eigenspace():
    n = 60
    A = pr.poisson1d(n)
    h = O.Hierarchy(A, seed=0)
    idx = [2, 9, 17, 40]
    b = sum(np.sin(k * np.pi * np.arange(1, n + 1) / (n + 1)) for k in idx)
    st, x, it, hist, _ = h.pcg(b, rtol=1e-10, maxit=50, precond=False)
    assert st == 0 and it <= len(idx) + 1


def test_pcg_exact_preconditioner_one_iteration():
    A = pr.poisson2d(8)
    h = O.Hierarchy(A, max_levels=1)
    assert h.nlevels == 1
    st, x, it, hist, _ = h.pcg(pr.uniform(A.n, 1), rtol=1e-10)
    assert st == 0 and it == 1


def test_setup_rejects_indefinite():
    """An indefinite matrix with a positive diagonal fails the dense Cholesky."""
    A = csr_from_dense([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(RuntimeError, match="-2"):
        O.Hierarchy(A, max_levels=1)


def test_check_csr_rejects_malformed():
    A = pr.poisson1d(5)
    bad = pr.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[1], bad.col[2] = bad.col[2], bad.col[1]  # unsorted row
    assert O.check_csr(bad) == O.ERR_ARG
    neg = pr.CSR(A.n, A.rowptr.copy(), A.col.copy(), -A.val)
    assert O.check_csr(neg) == O.ERR_NOT_SPD
    for bad_value in (np.nan, np.inf, -np.inf):  # values must be finite
        v = A.val.copy()
        v[2] = bad_value
        assert O.check_csr(pr.CSR(A.n, A.rowptr.copy(), A.col.copy(), v)) == O.ERR_ARG


# ------------------------------------------------------------ set-up ----

def test_setup_stops_at_max_coarse():
    A = pr.poisson2d(40)
    h = O.Hierarchy(A, seed=0, max_coarse=64)
    sizes = [h.level_sizes(k)[0] for k in range(h.nlevels)]
    assert sizes[-1] <= 64 and all(s > 64 for s in sizes[:-1])
    assert all(b < a for a, b in zip(sizes, sizes[1:]))
    cgd, cop = h.complexities()
    assert cgd == pytest.approx(sum(sizes) / sizes[0])


def test_setup_levels_are_galerkin_products():
    A = pr.poisson2d(20)
    h = O.Hierarchy(A, seed=4)
    As, Ps = _dense_hierarchy(h)
    for k in range(h.nlevels - 1):
        dense = Ps[k].T @ As[k] @ Ps[k]
        assert np.abs(As[k + 1] - dense).max() <= 1e-13 * np.abs(dense).max()
        assert np.linalg.eigvalsh(As[k + 1]).min() > 0
        # C/F of the level is a valid PMIS splitting of its own strength graph
        rp, ci, v = h.A(k)
        Ak = pr.CSR(len(rp) - 1, rp, ci, v)
        check_pmis_invariants(Ak, h.S(k), h.cf(k))
