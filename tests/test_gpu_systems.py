"""GPU parity of the systems variant (block_size 3: nodal block strength, PMIS on the node
graph, unknown-wise direct interpolation) against the CPU oracle.

Bars: C/F splittings and the patterns of P and A_c bit-exact; values 1e-12 relative to the
row's largest entry (expected bitwise); FP64 PCG with the oracle's iteration count and x
within 1e-9; FP32 V-cycle batches within 1e-6 of the oracle's x.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2102_07417_gb300 import amg  # noqa: E402
from paper_2102_07417_gb300 import problems as pr  # noqa: E402

from test_gpu_parity import assert_same_hierarchy, bitwise_equal_hierarchy, dev  # noqa: E402

SYSTEMS = {
    "elasticity_6": lambda: pr.elasticity3d(6),
    "elasticity_10_layers": lambda: pr.elasticity3d(10, layer=2),
    "kron_poisson3d_10": lambda: pr.kron_identity(pr.poisson3d(10), 3),
    "kron_diffusion3d_8": lambda: pr.kron_identity(pr.diffusion3d(8, 2.0, 1)[0], 3),
}
OMEGA = 0.5  # omega * rho(D^-1 A) < 2 for Q1 elasticity (rho ~ 3.09)


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("seed", [0, 5])
def test_block_hierarchy_bit_exact(name, seed):
    A = SYSTEMS[name]()
    ho = O.Hierarchy(A, seed=seed, block_size=3, omega=OMEGA)
    hg = amg.Hierarchy(A, seed=seed, block_size=3, omega=OMEGA)
    assert ho.nlevels >= 2
    assert_same_hierarchy(hg, ho)
    assert bitwise_equal_hierarchy(hg, ho)


def test_block_large_sell_path_fp64_pcg():
    """45,000 unknowns (the solve kernels run on the sliced-ELLPACK copies): bit-exact hierarchy
    and the oracle's iteration count.

    The stopping rule of Sec. 4 is a threshold test on the recursive residual.  This run takes
    368 iterations and the oracle's final residual is 0.987 of the threshold (the residual falls
    ~23% per iteration there), so a preconditioner equal to the oracle's in exact arithmetic but
    rounded differently (the dense operator that replaces the levels of <= 1024 rows) can cross
    it one iteration later.  The bar: the same count, or one more only when the oracle's final
    residual lies within 5% of the threshold; x within 1e-9 of the oracle's when the counts
    agree, else within 1e-6 (the solution bar of the method's accuracy target) with a true
    residual below 1.05 rtol."""
    A = pr.elasticity3d(24, layer=8)
    ho = O.Hierarchy(A, seed=0, block_size=3, omega=OMEGA)
    hg = amg.Hierarchy(A, seed=0, block_size=3, omega=OMEGA)
    assert_same_hierarchy(hg, ho)
    b = pr.uniform(A.n, 3)
    sto, xo, ito, hist_o, _ = ho.pcg(b, rtol=1e-8, maxit=3000)
    x, it, st, _ = hg.solve(dev(b), rtol=1e-8, maxit=3000)
    assert st == sto == 0
    tol = 1e-8 * np.linalg.norm(b)
    near = hist_o[ito] > 0.95 * tol
    assert it == ito or (near and it == ito + 1), (it, ito, hist_o[ito] / tol)
    xg = x.cpu().numpy()
    if it == ito:
        assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    else:
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
        assert np.linalg.norm(b - A.matvec(xg)) <= 1.05 * tol


def test_block_batch_fp32_16_rhs():
    """Sixteen right-hand sides in one batched FP32 V-cycle under the FP64 flexible PCG."""
    A = pr.elasticity3d(8, layer=2)
    rng = np.random.Generator(np.random.PCG64(3))
    Bm = rng.uniform(-1.0, 1.0, size=(A.n, 16))
    hg = amg.Hierarchy(A, seed=0, block_size=3, omega=OMEGA, precision=amg.PREC_FP32)
    X, iters, stats, st, _ = hg.solve_batch(dev(Bm), rtol=1e-8, maxit=2000)
    assert st == amg.AMG_OK
    Xg = X.cpu().numpy()
    ho = O.Hierarchy(A, seed=0, block_size=3, omega=OMEGA)
    for j in (0, 5, 15):
        _, xo, ito, _, _ = ho.pcg(Bm[:, j], rtol=1e-8, maxit=2000)
        assert np.linalg.norm(Xg[:, j] - xo) <= 1e-6 * np.linalg.norm(xo)
        # the FP32 V-cycle costs iterations on this ill-conditioned operator (E jumps 1e3 between
        # layers): at most 1.5x the FP64 oracle's count
        assert ito - 3 <= iters[j] <= 1.5 * ito
        assert np.linalg.norm(Bm[:, j] - A.matvec(Xg[:, j])) < 1e-7 * np.linalg.norm(Bm[:, j])


def test_block_size_needs_full_blocks():
    A = pr.kron_identity(pr.poisson2d(8), 3, full_blocks=False)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(A, block_size=3)
    assert e.value.code == amg.AMG_ERR_INVALID_ARG
    B = pr.poisson2d(8)  # 64 unknowns: not a multiple of 3
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(B, block_size=3)
    assert e.value.code == amg.AMG_ERR_INVALID_ARG


def test_config4_full_size():
    """64^3 Q1 elasticity (811,200 unknowns, 63.7M nonzeros), 16 right-hand sides in one batched
    FP32 V-cycle under the FP64 flexible PCG.  The hierarchy is checked against the oracle's
    systems set-up at full size (~8 s on one host core): every level's node labels, P and A_k
    bit-exact.  The oracle's solve (~3400 iterations per column) is too slow here, so the solve is
    checked by properties: every column converges; its true residual, from an FP64 product through
    amg_spmv, is within 10x of rtol; node labels are shared by a node's unknowns; and sampled rows
    of the level-1 operator equal the brute-force sum over R_I and A P."""
    A, Bm = pr.config4()
    ho = O.Hierarchy(A, seed=0, block_size=3, omega=OMEGA)
    h64 = amg.Hierarchy(A, seed=0, block_size=3, omega=OMEGA)
    assert_same_hierarchy(h64, ho)
    assert bitwise_equal_hierarchy(h64, ho)
    h64.close()
    del ho
    hg = amg.Hierarchy(A, seed=0, block_size=3, omega=OMEGA, precision=amg.PREC_FP32)
    B = dev(Bm)
    X, iters, stats, st, _ = hg.solve_batch(B, rtol=1e-8, maxit=5000)
    assert st == amg.AMG_OK and min(iters) > 0
    for j in range(16):
        x = X[:, j].contiguous()
        r = B[:, j] - hg.spmv(0, x)
        assert float(torch.linalg.norm(r) / torch.linalg.norm(B[:, j])) < 1e-7
    e0, e1 = hg.export(0), hg.export(1)
    cf = e0["cf"]
    assert np.array_equal(cf.reshape(-1, 3), np.repeat(cf[::3, None], 3, axis=1))
    arp, aci, av = e0["A"]
    prp, pci, pv = e0["P"]
    crp, cci, cv = e1["A"]
    nc = len(crp) - 1
    assert nc % 3 == 0
    import scipy.sparse as sp
    P = sp.csr_matrix((pv, pci, prp), shape=(A.n, nc))
    R = P.T.tocsr()
    rng = np.random.default_rng(0)
    for I in rng.choice(nc, 20, replace=False):
        acc = {}
        for q in range(R.indptr[I], R.indptr[I + 1]):
            i, rv = R.indices[q], R.data[q]
            for t in range(arp[i], arp[i + 1]):
                j, a = aci[t], av[t]
                for u in range(prp[j], prp[j + 1]):
                    acc[pci[u]] = acc.get(pci[u], 0.0) + rv * a * pv[u]
        cols = np.array(sorted(acc))
        assert np.array_equal(cci[crp[I]:crp[I + 1]], cols)
        ref = np.array([acc[c] for c in cols])
        got = cv[crp[I]:crp[I + 1]]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
