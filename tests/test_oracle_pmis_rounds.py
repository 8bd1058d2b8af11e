"""Pins of the oracle's PMIS round rule (Sec. 2.2, PMIS of De Sterck, Yang & Heys).

The paper cites PMIS without pseudocode, so the rule the oracle follows is a
reading: measures lambda_i = |S_i^T| + u_i; points with lambda_i < 1 start as
F; in synchronous rounds (decisions use the state at the round's start) an
undecided point becomes C when it beats every undecided j in S_i u S_i^T
(larger lambda, equal lambdas broken by the larger index), then every
undecided point whose S_i holds a new C point becomes F.

Invariants such as independence and F coverage hold for any maximal
independent set, and on a symmetric strength graph every variant of the rule
gives the same split, so they cannot tell the rule from a misreading.  The
cases below use asymmetric strength graphs and measures set by hand, and state
the expected split after every round, worked out by hand in each docstring.
Each plausible misreading is then planted in a copy of the oracle's source,
compiled on the CPU, and must fail at least one case.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_07417_gb300 import problems as pr

U_, F_, C_ = -1, 0, 1


def strength_case(S):
    """CSR with the pattern of S + S^T + I and the per-entry strength mask S."""
    S = np.asarray(S, dtype=np.uint8)
    n = S.shape[0]
    d = np.eye(n) * 4.0 - ((S + S.T) > 0)
    A = pr.dense_to_csr(d)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    mask = S[rows, A.col].astype(np.uint8)
    return A, mask


# Each case: strength matrix S (S[i][j] = 1: j in S_i, i depends strongly on j),
# measures lambda, and the state after rounds 0, 1, 2, ... (-1 undecided, 0 F, 1 C).
CASES = {
    "new_c_points_keep_competing": dict(
        S=[[0, 0, 0],
           [0, 0, 1],
           [1, 0, 0]],
        lam=[1.5, 0.75, 1.125],
        rounds=[[U_, F_, U_],
                [C_, F_, F_]],
        why="""S_1 = {2}, S_2 = {0}; S_0^T = {2}, S_2^T = {1}, S_1^T = {} (lambda_1 < 1: F).
        Round 1: point 0 meets only 2 (1.125 < 1.5) and becomes C; point 2 meets
        0 (1.5 > 1.125), still undecided at the round's start, so it is not C.
        Then 2 depends on the new C point 0 (0 in S_2) and becomes F.
        A reading where 0 stops competing as soon as it is C (asynchronous,
        in-place rounds) makes 2 C as well: [1, 0, 1]."""),
    "neighbourhood_is_s_union_st": dict(
        S=[[0, 0, 1, 0],
           [0, 0, 0, 0],
           [0, 0, 0, 1],
           [1, 1, 0, 0]],
        lam=[1.625, 1.375, 1.75, 1.5],
        rounds=[[U_, U_, U_, U_],
                [F_, U_, C_, U_],
                [F_, U_, C_, C_],
                [F_, C_, C_, C_]],
        why="""S_0 = {2}, S_2 = {3}, S_3 = {0, 1}, S_1 = {}; S_0^T = {3}, S_1^T = {3},
        S_2^T = {0}, S_3^T = {2}.
        Round 1: 0 meets 2 (1.75) and loses; 1 meets 3 (1.5) and loses; 2 meets
        3 and 0 (1.5, 1.625) and wins; 3 meets 0, 1, 2 and loses to 0 and 2.
        F step: 0 depends on 2 (F); 3 depends on 0 and 1, neither new C (stays).
        Round 2: 1 meets 3 (1.5 > 1.375, loses); 3 meets undecided 1 only
        (1.375 < 1.5, wins).  F step: S_1 is empty, so 1 stays undecided.
        Round 3: 1 has no undecided neighbour left and becomes C.
        Taking the neighbourhood as S_i alone makes 1 C in round 1 (S_1 is
        empty) and then 3 F (it depends on 1): [0, 1, 1, 0]."""),
    "f_from_s_i_not_st": dict(
        S=[[0, 1, 0],
           [0, 0, 0],
           [1, 0, 0]],
        lam=[1.375, 1.75, 0.25],
        rounds=[[U_, U_, F_],
                [F_, C_, F_]],
        why="""S_0 = {1}, S_2 = {0}; S_0^T = {2}, S_1^T = {0}, S_2^T = {} (F).
        Round 1: 0 meets 1 (1.75 > 1.375) and loses; 1 meets 0 and wins.
        0 depends on the new C point 1 (1 in S_0) and becomes F.
        Making F the points that influence a new C point (S_i^T) instead
        leaves 0 undecided, and it becomes C in round 2: [1, 1, 0]."""),
    "ties_to_larger_index": dict(
        S=[[0, 1, 0],
           [1, 0, 1],
           [0, 1, 0]],
        lam=[1.5, 2.5, 1.5],
        rounds=[[U_, U_, U_],
                [F_, C_, F_]],
        why="""A symmetric path 0 - 1 - 2 with the middle point strongest: 1 is C in
        round 1 and both ends depend on it.  (Kept as a plain control.)"""),
    "equal_measures": dict(
        S=[[0, 1, 0, 0],
           [1, 0, 0, 0],
           [0, 0, 0, 1],
           [0, 0, 1, 0]],
        lam=[1.5, 1.5, 1.25, 1.25],
        rounds=[[U_, U_, U_, U_],
                [F_, C_, F_, C_]],
        why="""Two mutually strong pairs (0, 1) and (2, 3), each with equal measures.
        Ties go to the larger index: 1 and 3 become C in round 1, 0 and 2 F.
        The reversed tie-break gives [1, 0, 1, 0]."""),
}


def run_case(case, L=None):
    """The oracle's state after each round of `case` (list of lists)."""
    A, S = strength_case(case["S"])
    out = []
    for r in range(len(case["rounds"])):
        st, _ = O.pmis_rounds(A, S, np.asarray(case["lam"], np.float64), r, L=L)
        out.append(st.tolist())
    final, nr = O.pmis_rounds(A, S, np.asarray(case["lam"], np.float64), -1, L=L)
    return out, final.tolist(), nr


@pytest.mark.parametrize("name", sorted(CASES))
def test_pmis_rounds_hand_worked(name):
    case = CASES[name]
    states, final, nr = run_case(case)
    assert states == case["rounds"], case["why"]
    assert final == case["rounds"][-1]
    assert nr == len(case["rounds"]) - 1


def test_pmis_measures_come_from_counter_stream():
    """or_pmis equals the round rule fed lambda_i = |S_i^T| + u_i with u_i the
    counter-based SplitMix64 value of (level, i) (pinned by its test vector)."""
    rng = np.random.default_rng(5)
    n = 120
    d = np.zeros((n, n))
    for i in range(n):
        for j in rng.choice(n, 5, replace=False):
            if i != j:
                d[i, j] = d[j, i] = -10.0 ** rng.uniform(-2.0, 0.0)  # weights over two decades
    np.fill_diagonal(d, -d.sum(axis=1) + 0.1)
    A = pr.dense_to_csr(d)
    S = O.strength(A, 0.25)
    deg = np.bincount(A.col[S.astype(bool)], minlength=A.n)
    assert np.any(S.astype(bool) != S[_mirror(A)].astype(bool))  # asymmetric strength
    for level in (0, 3):
        lam = deg + np.array([O.pmis_random(11, level, i) for i in range(A.n)])
        st, _ = O.pmis_rounds(A, S, lam, -1)
        assert np.array_equal(st, O.pmis(A, S, 11, level))


def _mirror(A):
    """Position of (j, i) for every entry (i, j) of a structurally symmetric CSR."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    key = rows.astype(np.int64) * A.n + A.col
    mkey = A.col.astype(np.int64) * A.n + rows
    order = np.argsort(key)
    return order[np.searchsorted(key[order], mkey)]


# Misreadings planted one at a time in a copy of the oracle's source.
MUTANTS = {
    # new C points drop out of the comparison within their own round
    "asynchronous_rounds": [("return st[j] == ST_U || st[j] == ST_NEWC;", "return st[j] == ST_U;")],
    # the comparison runs over S_i only
    "s_i_only": [("q < tcnt[i + 1] && is_max; ++q) /* j in S_i^T */", "q < tcnt[i] && is_max; ++q) /* j in S_i^T */")],
    # ties broken towards the smaller index
    "reversed_tie_break": [("(lam[i] == lam[j] && i > j)", "(lam[i] == lam[j] && i < j)")],
    # F for the points that influence a new C point
    "f_from_s_i_transpose": [("for (int p = rp[i]; p < rp[i + 1]; ++p)\n        if (S[p] && st[ci[p]] == ST_NEWC) {",
                              "for (int p = tcnt[i]; p < tcnt[i + 1]; ++p)\n        if (st[tcol[p]] == ST_NEWC) {")],
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_misreading_fails_a_pin(mutant, tmp_path):
    src = open(O.SRC).read()
    for old, new in MUTANTS[mutant]:
        assert src.count(old) == 1, f"pattern for {mutant} not found once in the oracle source"
        src = src.replace(old, new)
    path = os.path.join(tmp_path, "amg_oracle_mutant.c")
    with open(path, "w") as f:
        f.write(src)
    so = os.path.join(tmp_path, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path, "-lm"])
    L = O.configure(C.CDLL(so))
    failed = [name for name, case in CASES.items() if run_case(case, L)[0] != case["rounds"]]
    assert failed, f"misreading {mutant} passes every PMIS pin"
