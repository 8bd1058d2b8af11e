"""GPU parity of extended+i interpolation (Sec. 2.3, the distance-two formula) against the
CPU oracle, through the C ABI.

Bars: C/F splittings and the patterns of P and every A_k bit-exact; values bitwise equal
(the set-up evaluates the formula in the oracle's order, no FMA contraction; the test also
allows 1e-12 of the row's largest entry); PCG in FP64 with the oracle's iteration count and x
within 1e-9 of the oracle's; with the FSAI smoother as well; FP32 V-cycle modes to rtol 1e-8
with x within 1e-6.
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

CASES = {
    "poisson2d_48": lambda: pr.poisson2d(48),
    "poisson3d_20": lambda: pr.poisson3d(20),
    "diffusion3d_18": lambda: pr.diffusion3d(18, 2.0, 2)[0],
    "graph_laplacian_900": lambda: pr.graph_laplacian_spd(900, 7, 0.05, 3),
    "poisson1d_301": lambda: pr.poisson1d(301),
    "graph_hubs_4000": lambda: pr.graph_with_hubs(4000, 6, 3, 1200, 0.05, 8),
    "isolated_points": lambda: pr.dense_to_csr(np.diag(np.arange(1.0, 40.0))),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("seed", [0, 13])
def test_ext_hierarchy_bit_exact(name, seed):
    A = CASES[name]()
    ho = O.Hierarchy(A, seed=seed, interp="ext")
    hg = amg.Hierarchy(A, seed=seed, interp=amg.INTERP_EXT)
    assert_same_hierarchy(hg, ho)
    assert bitwise_equal_hierarchy(hg, ho)
    cgd, cop = ho.complexities()
    inf = hg.info()
    assert inf["cgd"] == pytest.approx(cgd, rel=1e-15) and inf["cop"] == pytest.approx(cop, rel=1e-15)


def test_ext_hierarchy_config2_full_size():
    """128^3 Poisson with extended+i: every level bit-exact against the oracle."""
    p = pr.config2()
    ho = O.Hierarchy(p.A, seed=0, interp="ext")
    hg = amg.Hierarchy(p.A, seed=0, interp=amg.INTERP_EXT)
    assert_same_hierarchy(hg, ho)
    assert bitwise_equal_hierarchy(hg, ho)


@pytest.mark.parametrize("name", ["poisson3d_20", "diffusion3d_18", "graph_laplacian_900"])
@pytest.mark.parametrize("smoother", ["jacobi", "fsai"])
def test_ext_pcg_fp64_parity(name, smoother):
    A = CASES[name]()
    om = 1.0 if smoother == "fsai" else 2.0 / 3.0
    ho = O.Hierarchy(A, seed=1, interp="ext", smoother=smoother, omega=om)
    hg = amg.Hierarchy(A, seed=1, interp=amg.INTERP_EXT, omega=om,
                       smoother=amg.SMOOTH_FSAI if smoother == "fsai" else amg.SMOOTH_JACOBI)
    b = pr.uniform(A.n, 4)
    sto, xo, ito, hist_o, _ = ho.pcg(b, rtol=1e-8, maxit=500)
    x, it, st, hist = hg.solve(dev(b), rtol=1e-8, maxit=500, hist=True)
    assert st == sto == 0 and it == ito
    assert np.abs(hist - hist_o).max() <= 1e-6 * hist_o[0]
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["poisson3d_20", "graph_hubs_4000"])
def test_ext_fsai_factors_match_oracle(name):
    """FSAI factors on the denser extended+i hierarchies: poisson3d_20's levels hold rows of every
    size bin of the GPU factor kernels (up to ~100 lower entries, a block per row in shared
    memory), the hub graph rows too long for shared memory (a warp per row in global scratch).
    Pattern exact, values within 1e-12 of the row's largest entry."""
    A = CASES[name]()
    ho = O.Hierarchy(A, seed=0, interp="ext", smoother="fsai", omega=1.0)
    hg = amg.Hierarchy(A, seed=0, interp=amg.INTERP_EXT, smoother=amg.SMOOTH_FSAI, omega=1.0)
    assert_same_hierarchy(hg, ho)
    for k in range(ho.nlevels - 1):
        gr, gc, gv = hg.export_fsai(k)
        orp, oci, ov = ho.G(k)
        assert np.array_equal(gr, orp) and np.array_equal(gc, oci), f"G_{k} pattern"
        scale = np.maximum.reduceat(np.abs(ov), orp[:-1])
        rows = np.repeat(np.arange(len(orp) - 1), np.diff(orp))
        assert np.all(np.abs(gv - ov) <= 1e-12 * scale[rows]), f"G_{k} values"


def test_ext_large_sell_levels_and_fp32():
    """262,144 rows (the solve kernels on sliced-ELLPACK copies): FP64 with the oracle's count,
    FP32 V-cycle within 1e-6 of the oracle's x."""
    A = pr.diffusion3d(64, 2.0, 5)[0]
    ho = O.Hierarchy(A, seed=0, interp="ext")
    b = pr.uniform(A.n, 2)
    sto, xo, ito, _, _ = ho.pcg(b, rtol=1e-8, maxit=500)
    for prec in (amg.PREC_FP64, amg.PREC_FP32):
        hg = amg.Hierarchy(A, seed=0, interp=amg.INTERP_EXT, precision=prec)
        x, it, st, _ = hg.solve(dev(b), rtol=1e-8, maxit=500)
        assert st == sto == 0
        if prec == amg.PREC_FP64:
            assert it == ito
            assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        else:
            assert it <= 1.2 * ito + 1
            assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_ext_batch_matches_single_solves():
    A = CASES["poisson3d_20"]()
    hg = amg.Hierarchy(A, seed=0, interp=amg.INTERP_EXT)
    rng = np.random.default_rng(1)
    B = rng.uniform(-1.0, 1.0, (A.n, 4))
    X, iters, stats, st, _ = hg.solve_batch(dev(B), rtol=1e-8)
    assert st == 0
    for j in range(4):
        x, it, s1, _ = hg.solve(dev(B[:, j].copy()), rtol=1e-8)
        assert it == iters[j]
        assert np.linalg.norm(X[:, j].cpu().numpy() - x.cpu().numpy()) <= 1e-9 * np.linalg.norm(x.cpu().numpy())


def test_ext_needs_scalar_problems():
    A = pr.kron_identity(pr.poisson3d(5), 3)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy(A, block_size=3, interp=amg.INTERP_EXT)
    assert e.value.code == amg.AMG_ERR_INVALID_ARG
