"""Pins of the oracle's systems variant (nodal block strength, node PMIS, unknown-wise
direct interpolation) against hand-worked values, exact invariances and reductions to the
scalar method."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr


def _dense_csr(d):
    """CSR of d keeping every entry of the nonzero bs x bs blocks (explicit zeros)."""
    return pr.dense_to_csr(np.asarray(d, dtype=np.float64))


def _hand_blocks():
    """Three nodes, two unknowns each.  ||A_00|| = ||A_11|| = 5, ||A_22|| = 10,
    ||A_01|| = 1, ||A_12|| = 5, no coupling 0-2:  s_01 = 1/5, s_12 = 5/sqrt(50) = 1/sqrt(2)."""
    d = np.zeros((6, 6))
    d[0:2, 0:2] = np.diag([3.0, 4.0])
    d[2:4, 2:4] = np.diag([3.0, 4.0])
    d[4:6, 4:6] = np.diag([6.0, 8.0])
    d[0:2, 2:4] = [[-1.0, 0.0], [0.0, 0.0]]
    d[2:4, 4:6] = [[0.0, -3.0], [-4.0, 0.0]]
    d[2:4, 0:2] = d[0:2, 2:4].T
    d[4:6, 2:4] = d[2:4, 4:6].T
    A = pr.dense_to_csr(d)
    # dense_to_csr drops zeros off the diagonal: put the explicit zeros of the blocks back
    mask = np.zeros((6, 6), bool)
    for I, J in [(0, 0), (1, 1), (2, 2), (0, 1), (1, 0), (1, 2), (2, 1)]:
        mask[2 * I:2 * I + 2, 2 * J:2 * J + 2] = True
    cols = np.broadcast_to(np.arange(6), (6, 6))
    return pr._finish(6, cols, d, mask), d


@pytest.mark.parametrize("theta,strong1", [(0.25, {0, 2}), (0.5, {2})])
def test_block_strength_hand_example(theta, strong1):
    A, _ = _hand_blocks()
    Nrp, Nci, SN, S = O.block_strength(A, 2, theta)
    assert list(Nrp) == [0, 2, 5, 7] and list(Nci) == [0, 1, 0, 1, 2, 1, 2]
    strong = {I: {int(Nci[e]) for e in range(Nrp[I], Nrp[I + 1]) if SN[e]} for I in range(3)}
    assert strong[0] == {1} and strong[2] == {1} and strong[1] == strong1
    # unknown-wise: a row is strongly influenced only by its own component of strong nodes
    for i in range(6):
        for p in range(A.rowptr[i], A.rowptr[i + 1]):
            j = A.col[p]
            want = j % 2 == i % 2 and j // 2 != i // 2 and (j // 2) in strong[i // 2]
            assert S[p] == want


def test_block_strength_power_of_two_node_scaling_invariant():
    """s_IJ is invariant under A -> D A D with D = d_I I on node I; with powers of two the
    scaling is exact in floating point, so the strong sets are identical."""
    A = pr.elasticity3d(3)
    rng = np.random.default_rng(5)
    nn = A.n // 3
    dI = 2.0 ** rng.integers(-6, 7, size=nn)
    dvec = np.repeat(dI, 3)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    B = pr.CSR(A.n, A.rowptr, A.col, A.val * dvec[rows] * dvec[A.col])
    for theta in (0.25, 0.5, 0.8):
        a = O.block_strength(A, 3, theta)
        b = O.block_strength(B, 3, theta)
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    # an unscaled measure (row maximum of raw block norms) would change: the scaling is not trivial
    assert dI.max() / dI.min() >= 2 ** 8


@pytest.mark.parametrize("full", [True, False])
def test_block_hierarchy_of_kron_is_kron_of_scalar(full):
    """A (x) I_3 with equal-magnitude neighbours: nodal strength equals the scalar strength, so
    the first coarsening of the systems variant is the scalar one applied per component: C/F
    repeated per node, P = P_s (x) I_3, A_1 = A_1,s (x) I_3 (values equal; the full-block form
    keeps zero blocks)."""
    As = pr.poisson2d(14)
    A = pr.kron_identity(As, 3, full_blocks=full)
    hs = O.Hierarchy(As, seed=3, max_levels=2)
    hb = O.Hierarchy(A, seed=3, max_levels=2, block_size=3)
    assert hs.nlevels == 2 and hb.nlevels == 2
    assert np.array_equal(hb.cf(0), np.repeat(hs.cf(0), 3))
    for get in ("P", "A"):
        ks = 0 if get == "P" else 1
        rp_s, ci_s, v_s = getattr(hs, get)(ks)
        rp_b, ci_b, v_b = getattr(hb, get)(ks)
        nrow = len(rp_s) - 1
        ncol = int(ci_s.max()) + 1
        Ds = np.zeros((nrow, ncol))
        for i in range(nrow):
            Ds[i, ci_s[rp_s[i]:rp_s[i + 1]]] = v_s[rp_s[i]:rp_s[i + 1]]
        Db = np.zeros((3 * nrow, 3 * ncol))
        for i in range(3 * nrow):
            Db[i, ci_b[rp_b[i]:rp_b[i + 1]]] = v_b[rp_b[i]:rp_b[i + 1]]
        assert np.array_equal(Db, np.kron(Ds, np.eye(3))), get


def test_block_setup_elasticity_invariants():
    """Q1 elasticity: node-level PMIS invariants, every unknown of a node shares its label,
    unknown-wise P (no cross-component weights), translations reproduced on rows whose
    same-component sum vanishes, and SPD Galerkin levels equal to the dense P^T A P."""
    A = pr.elasticity3d(5)
    h = O.Hierarchy(A, seed=1, block_size=3, omega=0.5)
    assert h.nlevels >= 2
    checked = 0
    for k in range(h.nlevels - 1):
        rp, ci, v = h.A(k)
        n = len(rp) - 1
        Ak = pr.CSR(n, rp, ci, v)
        cf = h.cf(k)
        assert np.array_equal(cf.reshape(-1, 3), np.repeat(cf[::3, None], 3, axis=1))
        Nrp, Nci, SN, S = O.block_strength(Ak, 3, 0.25)
        cfn = cf[::3]
        for I in range(n // 3):
            nb = Nci[Nrp[I]:Nrp[I + 1]]
            sI = nb[SN[Nrp[I]:Nrp[I + 1]] == 1]
            if cfn[I]:
                assert not np.any(cfn[sI])  # no strong C-C connection
        prp, pci, pv = h.P(k)
        for i in range(n):
            cols = pci[prp[i]:prp[i + 1]]
            assert np.all(cols % 3 == i % 3)
        # translation along each axis: same-component sums vanish on interior rows
        Dk = Ak.to_dense()
        for i in range(n):
            if cf[i] or prp[i + 1] == prp[i]:
                continue
            same = Dk[i, (np.arange(n) % 3) == (i % 3)]
            wsum = pv[prp[i]:prp[i + 1]].sum()
            if abs(same.sum()) <= 1e-12 * np.abs(same).max():
                sel = S[Ak.rowptr[i]:Ak.rowptr[i + 1]].astype(bool) & (cf[Ak.col[Ak.rowptr[i]:Ak.rowptr[i + 1]]] == 1)
                pvals = Ak.val[Ak.rowptr[i]:Ak.rowptr[i + 1]][sel]
                # a negative interpolatory coupling: either both branches scale to the full row
                # sums, or the positive couplings are lumped into the diagonal; both give sum 1
                if np.any(pvals < 0):
                    assert abs(wsum - 1.0) < 1e-12
                    checked += 1
        P = np.zeros((n, int(pci.max()) + 1))
        for i in range(n):
            P[i, pci[prp[i]:prp[i + 1]]] = pv[prp[i]:prp[i + 1]]
        crp, cci, cv = h.A(k + 1)
        nc = len(crp) - 1
        Ac = np.zeros((nc, nc))
        for I in range(nc):
            Ac[I, cci[crp[I]:crp[I + 1]]] = cv[crp[I]:crp[I + 1]]
        ref = P.T @ Dk @ P
        assert np.abs(Ac - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.linalg.eigvalsh(0.5 * (Ac + Ac.T)).min() > 0
        assert nc % 3 == 0
    assert checked > 100


def test_block_pcg_elasticity_matches_dense_solve():
    A = pr.elasticity3d(4, E=(1.0, 1e3), layer=2)
    b = np.random.default_rng(3).uniform(-1.0, 1.0, A.n)
    h = O.Hierarchy(A, seed=0, block_size=3, omega=0.5)
    st, x, it, hist, _ = h.pcg(b, rtol=1e-12, maxit=2000)
    assert st == 0
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_elasticity_generator_closed_forms():
    for ne in (2, 3, 5):
        A = pr.elasticity3d(ne)
        assert A.n == 3 * (ne + 1) ** 2 * ne and A.nnz == pr.nnz_elasticity3d(ne)
    assert pr.nnz_elasticity3d(64) == 63_695_790 and 3 * 65 * 65 * 64 == 811_200
    K = pr.q1_hex_stiffness(0.3)
    ev = np.linalg.eigvalsh(K)
    assert np.array_equal(K, K.T) and np.sum(np.abs(ev) < 1e-12) == 6 and ev.min() > -1e-12
    # rigid translations are in the null space of the element matrix
    for c in range(3):
        u = np.zeros(24)
        u[c::3] = 1.0
        assert np.abs(K @ u).max() < 1e-13
    A = pr.elasticity3d(3)
    D = A.to_dense()
    assert np.array_equal(D, D.T) and np.linalg.eigvalsh(D).min() > 0
