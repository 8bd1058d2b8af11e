"""GPU parity of the FSAI smoother (Sec. 2.1, Eq. smo: M^-1 = G^T G, G lower triangular on the
static pattern of lower(A_k)) against the CPU oracle, through the C ABI.

Bars: the hierarchy (C/F, P, A_k) is the Jacobi one, bit-exact; G_k's pattern exact and its
values within 1e-12 of the row's largest entry (the GPU solves each local system through its
Cholesky factor as g = L^-T e_last, the oracle solves it and rescales: the same numbers up to
rounding); V-cycle FP64 within 1e-10 of max |z| (G's rounding propagated through the cycle);
FP32 within 1e-5; PCG FP64 with the oracle's iteration count and x within 1e-9; FP32 modes to
rtol 1e-8 with x within 1e-6 of the oracle's.
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
    "poisson2d_40": lambda: pr.poisson2d(40),
    "poisson3d_20": lambda: pr.poisson3d(20),
    "diffusion3d_16": lambda: pr.diffusion3d(16, 2.0, 2)[0],
    "graph_hubs_3000": lambda: pr.graph_with_hubs(3000, 6, 3, 900, 0.05, 8),
}


def pair(A, nu=(1, 1), precision=amg.PREC_FP64, seed=0):
    ho = O.Hierarchy(A, seed=seed, nu1=nu[0], nu2=nu[1], smoother="fsai", omega=1.0)
    hg = amg.Hierarchy(A, seed=seed, nu1=nu[0], nu2=nu[1], smoother=amg.SMOOTH_FSAI, omega=1.0, precision=precision)
    return ho, hg


@pytest.mark.parametrize("name", list(CASES))
def test_fsai_factors_match_oracle(name):
    A = CASES[name]()
    ho, hg = pair(A)
    assert_same_hierarchy(hg, ho)
    assert bitwise_equal_hierarchy(hg, ho)
    for k in range(ho.nlevels - 1):
        gr, gc, gv = hg.export_fsai(k)
        orp, oci, ov = ho.G(k)
        assert np.array_equal(gr, orp) and np.array_equal(gc, oci), f"G_{k} pattern"
        scale = np.maximum.reduceat(np.abs(ov), orp[:-1])
        rows = np.repeat(np.arange(len(orp) - 1), np.diff(orp))
        assert np.all(np.abs(gv - ov) <= 1e-12 * scale[rows]), f"G_{k} values"
    assert hg.export_fsai(ho.nlevels - 1) is None


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (0, 2), (1, 0)])
def test_fsai_vcycle_fp64_parity(name, nu):
    A = CASES[name]()
    ho, hg = pair(A, nu)
    y = pr.uniform(A.n, 5)
    zo = ho.vcycle(y)
    zg = hg.vcycle(dev(y)).cpu().numpy()
    assert np.abs(zg - zo).max() <= 1e-10 * np.abs(zo).max()


@pytest.mark.parametrize("prec,tol", [(amg.PREC_FP32, 1e-5), (amg.PREC_FP32_BF16PR, 2e-2)])
def test_fsai_vcycle_reduced_precision(prec, tol):
    A = CASES["diffusion3d_16"]()
    ho, hg = pair(A, precision=prec)
    y = pr.uniform(A.n, 6)
    zo = ho.vcycle(y)
    zg = hg.vcycle(dev(y)).cpu().numpy()
    assert np.abs(zg - zo).max() <= tol * np.abs(zo).max()


@pytest.mark.parametrize("name", list(CASES))
def test_fsai_pcg_fp64_parity(name):
    A = CASES[name]()
    ho, hg = pair(A)
    b = pr.uniform(A.n, 7)
    sto, xo, ito, hist_o, _ = ho.pcg(b, rtol=1e-8, maxit=500)
    x, it, st, hist = hg.solve(dev(b), rtol=1e-8, maxit=500, hist=True)
    assert st == sto == 0 and it == ito
    assert np.abs(hist - hist_o).max() <= 1e-6 * hist_o[0]
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)


def test_fsai_pcg_large_sell_levels():
    """262,144 rows: level 0's A, G and omega G^T run on their sliced-ELLPACK copies."""
    A = pr.diffusion3d(64, 2.0, 4)[0]
    ho, hg = pair(A)
    b = pr.uniform(A.n, 8)
    sto, xo, ito, _, _ = ho.pcg(b, rtol=1e-8, maxit=500)
    x, it, st, _ = hg.solve(dev(b), rtol=1e-8, maxit=500)
    assert st == sto == 0 and it == ito
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


@pytest.mark.parametrize("prec", [amg.PREC_FP32, amg.PREC_FP32_BF16PR])
def test_fsai_pcg_mixed_precision(prec):
    p = pr.config2(48)
    ho, hg = pair(p.A, precision=prec)
    sto, xo, ito, _, _ = ho.pcg(p.b, rtol=1e-8, maxit=500)
    x, it, st, _ = hg.solve(dev(p.b), rtol=1e-8, maxit=500)
    assert st == sto == 0 and it <= 1.2 * ito + 1
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_fsai_fewer_iterations_than_jacobi():
    p = pr.config2(64)
    hj = amg.Hierarchy(p.A, seed=0)
    hf = amg.Hierarchy(p.A, seed=0, smoother=amg.SMOOTH_FSAI)
    _, itj, stj, _ = hj.solve(dev(p.b), rtol=1e-8)
    x, itf, stf, _ = hf.solve(dev(p.b), rtol=1e-8)
    assert stj == stf == 0 and itf < itj
    assert np.linalg.norm(x.cpu().numpy() - p.xstar) <= 1e-6 * np.linalg.norm(p.xstar)


def test_fsai_batched_paths_are_rejected():
    A = pr.poisson2d(20)
    hg = amg.Hierarchy(A, smoother=amg.SMOOTH_FSAI)
    with pytest.raises(amg.AmgError) as e:
        hg.solve_batch(dev(np.ones((A.n, 2))))
    assert e.value.code == amg.AMG_ERR_UNSUPPORTED
    with pytest.raises(amg.AmgError) as e:
        hg.slots(2)
    assert e.value.code == amg.AMG_ERR_UNSUPPORTED
