"""Pins of the oracle's FSAI smoother (Eq. smo: M^-1 = G^T G with G lower triangular, used in
the smoother S = I - omega M^-1 A of Eq. smoother).

Reading: static FSAI on the pattern of lower(A).  Each check compares the oracle with
something other than itself: the Frobenius-norm minimisation that defines FSAI solved by
numpy least squares on the dense Cholesky factor, the inverse Cholesky factor when the
pattern is full, the closed form on diagonal matrices, dense numpy arithmetic for the
smoothing step, and the dense two-grid operator of Eq. twoGridOp for the V-cycle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr


def dense(A):
    return A.to_dense()


def G_dense(G, n):
    rp, ci, v = G
    D = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    D[rows, ci] = v
    return D


def random_spd(n, seed, per_row=4, decades=2.0):
    rng = np.random.default_rng(seed)
    d = np.zeros((n, n))
    for i in range(n):
        for j in rng.choice(n, per_row, replace=False):
            if i != j:
                d[i, j] = d[j, i] = -10.0 ** rng.uniform(-decades, 0.0) * (1 if rng.uniform() < 0.85 else -0.3)
    np.fill_diagonal(d, np.abs(d).sum(axis=1) + rng.uniform(0.05, 1.0, n))
    return pr.dense_to_csr(d)


@pytest.mark.parametrize("make", [lambda: random_spd(40, 1), lambda: random_spd(60, 2, 6),
                                  lambda: pr.poisson2d(7), lambda: pr.diffusion3d(4, 2.0, 3)[0]])
def test_fsai_is_the_frobenius_minimiser(make):
    """Row i of G minimises ||e_i^T - g^T L||_2 over g supported on P_i = {j <= i : a_ij stored}
    (A = L L^T), scaled so that (G A G^T)_ii = 1 (Kolotilina-Yeremin)."""
    A = make()
    D = dense(A)
    L = np.linalg.cholesky(D)
    G = G_dense(O.fsai(A), A.n)
    for i in range(A.n):
        Pi = [j for j in A.col[A.rowptr[i]:A.rowptr[i + 1]] if j <= i]
        e = np.zeros(A.n)
        e[i] = 1.0
        g, *_ = np.linalg.lstsq(L[Pi, :].T, e, rcond=None)
        g = g / np.sqrt(g @ D[np.ix_(Pi, Pi)] @ g)
        row = np.zeros(A.n)
        row[Pi] = g
        assert np.abs(G[i] - row).max() <= 1e-12 * np.abs(row).max()
        assert np.all(G[i, [j for j in range(A.n) if j not in Pi]] == 0.0)


def test_fsai_full_pattern_is_inverse_cholesky():
    """A full lower pattern gives G = L^-1 (the exact inverse factor) and G A G^T = I."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((25, 25))
    d = X @ X.T + 25 * np.eye(25)
    A = pr.dense_to_csr(d)
    G = G_dense(O.fsai(A), 25)
    Li = np.linalg.inv(np.linalg.cholesky(d))
    assert np.abs(G - Li).max() <= 1e-12 * np.abs(Li).max()
    assert np.abs(G @ d @ G.T - np.eye(25)).max() <= 1e-12


def test_fsai_diagonal_matrix():
    a = np.array([4.0, 9.0, 0.25, 2.0])
    A = pr.dense_to_csr(np.diag(a))
    rp, ci, v = O.fsai(A)
    assert list(ci) == [0, 1, 2, 3]
    assert np.array_equal(v, 1.0 / np.sqrt(a))


@pytest.mark.parametrize("make", [lambda: pr.poisson3d(6), lambda: random_spd(80, 5),
                                  lambda: pr.graph_laplacian_spd(120, 6, 0.1, 2)])
def test_fsai_unit_diagonal_and_lower_pattern(make):
    A = make()
    D = dense(A)
    rp, ci, v = O.fsai(A)
    G = G_dense((rp, ci, v), A.n)
    assert np.allclose(np.diag(G @ D @ G.T), 1.0, rtol=0, atol=1e-14)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    lower = A.col <= rows
    assert len(ci) == lower.sum() and np.array_equal(ci, A.col[lower])
    # the last entry of every row is its diagonal, and it is positive
    assert np.all(ci[rp[1:] - 1] == np.arange(A.n)) and np.all(v[rp[1:] - 1] > 0)


def test_fsai_sweep_dense():
    A = random_spd(50, 7)
    D = dense(A)
    G = O.fsai(A)
    Gd = G_dense(G, A.n)
    rng = np.random.default_rng(1)
    y, s = rng.standard_normal(A.n), rng.standard_normal(A.n)
    got = O.fsai_sweep(A, G, 0.8, y, s)
    want = s + 0.8 * Gd.T @ (Gd @ (y - D @ s))
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def _dense_hierarchy(h):
    As, Ps, Gs = [], [], []
    for k in range(h.nlevels):
        rp, ci, v = h.A(k)
        n = len(rp) - 1
        As.append(G_dense((rp, ci, v), n))
        if k < h.nlevels - 1:
            prp, pci, pv = h.P(k)
            nc = h.level_sizes(k + 1)[0]
            P = np.zeros((n, nc))
            P[np.repeat(np.arange(n), np.diff(prp)), pci] = pv
            Ps.append(P)
            Gs.append(G_dense(h.G(k), n))
    return As, Ps, Gs


def _dense_vcycle_fsai(As, Ps, Gs, omega, nu1, nu2):
    """B_k = (I - E_k) A_k^-1 with E_k = S^nu2 (I - P B_{k+1} P^T A_k) S^nu1 (Eq. twoGridOp),
    S = I - omega G^T G A (Eq. smoother with Eq. smo); G_k is the FSAI factor of the oracle's
    own A_k, pinned above."""
    A = As[0]
    if not Ps:
        return np.linalg.inv(A)
    P = Ps[0]
    Bc = _dense_vcycle_fsai(As[1:], Ps[1:], Gs[1:], omega, nu1, nu2)
    n = A.shape[0]
    S = np.eye(n) - omega * Gs[0].T @ Gs[0] @ A
    E = np.linalg.matrix_power(S, nu2) @ (np.eye(n) - P @ Bc @ P.T @ A) @ np.linalg.matrix_power(S, nu1)
    return (np.eye(n) - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("make,levels,nu", [
    (lambda: pr.poisson2d(10), 2, (1, 1)),
    (lambda: pr.poisson2d(16), 4, (1, 1)),
    (lambda: pr.diffusion3d(6, 2.0, 8)[0], 3, (2, 1)),
    (lambda: random_spd(70, 3), 3, (1, 2)),
])
def test_fsai_vcycle_matches_dense_operator(make, levels, nu):
    A = make()
    h = O.Hierarchy(A, seed=5, max_coarse=4, max_levels=levels, nu1=nu[0], nu2=nu[1], smoother="fsai", omega=1.0)
    assert h.nlevels == levels
    As, Ps, Gs = _dense_hierarchy(h)
    # each level's G is the FSAI factor of that level's operator
    for k, Gk in enumerate(Gs):
        assert np.array_equal(Gk, G_dense(O.fsai(pr.dense_to_csr(As[k])), As[k].shape[0]))
    B = _dense_vcycle_fsai(As, Ps, Gs, 1.0, *nu)
    got = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.abs(got - B).max() <= 1e-10 * np.abs(B).max()
    if nu[0] == nu[1]:  # G^T G is symmetric, so S is A-self-adjoint and V(nu, nu) is a symmetric preconditioner
        assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()


@pytest.mark.parametrize("make", [lambda: pr.poisson2d(20), lambda: pr.diffusion3d(7, 2.0, 6)[0]])
def test_fsai_pcg_matches_dense_solve(make):
    A = make()
    b = pr.uniform(A.n, 9)
    h = O.Hierarchy(A, seed=2, smoother="fsai", omega=1.0)
    st, x, it, hist, _ = h.pcg(b, rtol=1e-12, maxit=200)
    assert st == 0
    xd = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_fsai_smoother_spectrum_and_fewer_iterations():
    """omega rho(G^T G A) < 2 at omega = 1 on 3-D Poisson (the condition that follows Eq.
    smoother), and the FSAI V-cycle needs fewer PCG iterations than damped Jacobi."""
    A = pr.poisson3d(10)
    G = G_dense(O.fsai(A), A.n)
    lmax = np.linalg.eigvalsh(G @ dense(A) @ G.T).max()
    assert 1.0 < lmax < 2.0
    p = pr.config2(24)
    its = {}
    for sm, om in (("jacobi", 2.0 / 3.0), ("fsai", 1.0)):
        st, _, it, _, _ = O.Hierarchy(p.A, smoother=sm, omega=om).pcg(p.b, rtol=1e-8)
        assert st == 0
        its[sm] = it
    assert its["fsai"] < its["jacobi"]
