"""The set-up kernels take some FP64 decisions on bit patterns with integer
instructions (GB300's FP64 pipe is narrow).  These CPU tests restate those
rules in numpy, independently of the kernels, and check that they decide
exactly as the oracle's FP64 comparisons do, on values chosen to break a wrong
argument: signed zeros, subnormals, equal magnitudes, a threshold that
underflows to zero, huge magnitudes.

- Strength (Eq. cla read as Ruge-Stueben): m_i = max_{k != i} -a_ik > 0 iff
  some off-diagonal is negative, m_i is then the largest magnitude among the
  negative entries (non-negative doubles order as their bit patterns), and
  -a_ij >= thr_i = theta m_i iff a_ij < 0 with |a_ij| >= thr_i as bit patterns
  when thr_i > 0, iff a_ij <= 0 when thr_i = +0.
- PMIS measures lambda_i = |S_i^T| + u_i >= 0 compare as signed 64-bit
  integers exactly as the doubles do.
- The interpolation's sign classes (v < 0, v > 0, neither for +-0).
"""
import numpy as np

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr

MAG = np.uint64(0x7FFFFFFFFFFFFFFF)


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.int64)


def strength_bits(A, theta):
    """The bit-pattern form of the strength rule (a restatement, not the kernel)."""
    S = np.zeros(A.nnz, dtype=np.uint8)
    for i in range(A.n):
        b, e = A.rowptr[i], A.rowptr[i + 1]
        cols, vals = A.col[b:e], A.val[b:e]
        vb = bits(vals)
        off = cols != i
        neg = (vb < 0) & off
        mk = np.uint64(0)
        if neg.any():
            mk = (vb[neg].view(np.uint64) & MAG).max()
        if mk == 0:
            continue
        m = np.array([mk], dtype=np.uint64).view(np.float64)[0]
        thr = np.float64(theta) * m
        tb = np.uint64(bits(thr))
        mags = vb.view(np.uint64) & MAG
        if tb == 0:
            strong = (vb < 0) | (vb == 0)
        else:
            strong = (vb < 0) & (mags >= tb)
        S[b:e] = (strong & off).astype(np.uint8)
    return S


def _adversarial_matrix(n, seed):
    """Symmetric-pattern matrices whose off-diagonal values include signed
    zeros, subnormals, repeated magnitudes, positive entries and values large
    enough or small enough that theta * m_i underflows."""
    rng = np.random.default_rng(seed)
    special = np.array([0.0, -0.0, -5e-324, 5e-324, -1e-310, -1.0, -1.0, -0.25, 0.5, -4.0, 2.0,
                        -1e300, -3e-323, -2.5, -2.5, 7.0, -1e-320])
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i), cols.append(i), vals.append(10.0 + rng.uniform())
        for j in rng.choice(n, size=rng.integers(2, 7), replace=False):
            if j == i:
                continue
            v = special[rng.integers(len(special))] if rng.uniform() < 0.6 else -rng.uniform(0.01, 3.0)
            rows += [i, j]
            cols += [j, i]
            vals += [v, v]
    D = {}
    for r, c, v in zip(rows, cols, vals):
        D[(r, c)] = v  # later duplicates overwrite: pattern stays symmetric
    rp = np.zeros(n + 1, dtype=np.int32)
    keys = sorted(D)
    for r, _ in keys:
        rp[r + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([c for _, c in keys], dtype=np.int32)
    v = np.array([D[k] for k in keys], dtype=np.float64)
    return pr.CSR(n, rp, ci, v)


def test_strength_bit_rule_equals_fp64_rule_on_adversarial_values():
    for seed in range(6):
        A = _adversarial_matrix(120, seed)
        for theta in (0.25, 0.5, 1.0, 1e-300):
            assert np.array_equal(strength_bits(A, theta), O.strength(A, theta)), (seed, theta)


def test_strength_threshold_underflow_row():
    """A row whose only negative off-diagonal is the smallest subnormal: theta m_i
    rounds to +0, so -a_ij >= +0 holds for the subnormal, +0 and -0 entries and
    not for the positive one (the thr = +0 branch of the bit rule)."""
    d = np.eye(5)
    for j, v in ((1, -5e-324), (2, 0.0), (3, -0.0), (4, 1e-320)):
        d[0, j] = d[j, 0] = v
    rp, ci, vals = [0], [], []
    for i in range(5):
        for j in range(5):
            if i == j or (i == 0 or j == 0):  # keep explicit zeros in row/column 0
                ci.append(j)
                vals.append(d[i, j])
        rp.append(len(ci))
    A = pr.CSR(5, np.array(rp, np.int32), np.array(ci, np.int32), np.array(vals))
    So = O.strength(A, 0.25)
    assert list(So[:5]) == [0, 1, 1, 1, 0]  # row 0: columns 0..4
    assert np.array_equal(strength_bits(A, 0.25), So)


def test_strength_bit_rule_equals_fp64_rule_on_problem_matrices():
    for A in (pr.poisson2d(12), pr.diffusion3d(6, 2.0, 4)[0], pr.graph_laplacian_spd(200, 6, 0.3, 2)):
        assert np.array_equal(strength_bits(A, 0.25), O.strength(A, 0.25))


def test_pmis_measures_order_as_int64():
    rng = np.random.default_rng(3)
    cnt = rng.integers(0, 40, size=4000).astype(np.float64)
    u = rng.integers(0, 2**53, size=4000, dtype=np.uint64).astype(np.float64) * 2.0 ** -53
    lam = np.concatenate([cnt + u, [0.0, 1.0, 1.0, np.nextafter(1.0, 2.0), 39.999999999999, 5e-324]])
    k = bits(lam)
    a, b = np.meshgrid(np.arange(len(lam)), np.arange(len(lam)), indexing="ij")
    sel = (a[:, :50].ravel(), b[:, :50].ravel())  # every value against 50 others
    assert np.array_equal(lam[sel[0]] > lam[sel[1]], k[sel[0]] > k[sel[1]])
    assert np.array_equal(lam[sel[0]] == lam[sel[1]], k[sel[0]] == k[sel[1]])


def test_sign_class_matches_fp64_comparisons():
    vals = np.array([0.0, -0.0, 5e-324, -5e-324, 1.0, -1.0, np.inf, -np.inf, np.nan, -np.nan, 1e308, -1e-310])
    vb = bits(vals)
    mag = vb.view(np.uint64) & MAG
    ok = (mag != 0) & (mag <= np.uint64(0x7FF0000000000000))
    cls = np.where(ok, np.where(vb < 0, -1, 1), 0)
    with np.errstate(invalid="ignore"):
        ref = np.where(vals < 0.0, -1, np.where(vals > 0.0, 1, 0))
    assert np.array_equal(cls, ref)
