"""ctypes wrapper around the plain FP64 CPU oracle (``amg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference legs are the only callers.  It marshals numpy arrays
into the C functions; every step of the method is in ``amg_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OK, ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NO_CONVERGENCE, ERR_SETUP, ERR_MEM = 0, -1, -2, -3, -4, -5, -6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: no FMA contraction, single thread."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = configure(C.CDLL(build()))
    return _lib


def configure(L):
    """Declares the argument types of every oracle entry point on a loaded library."""
    if True:
        L.or_check_csr.argtypes = [C.c_int, _i32p, _i32p, _f64p]
        L.or_strength.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, _u8p]
        L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.or_splitmix64.restype = C.c_uint64
        L.or_pmis_random.argtypes = [C.c_uint64, C.c_int, C.c_int]
        L.or_pmis_random.restype = C.c_double
        L.or_pmis.argtypes = [C.c_int, _i32p, _i32p, _u8p, C.c_uint64, C.c_int, _i8p]
        L.or_pmis_rounds.argtypes = [C.c_int, _i32p, _i32p, _u8p, _f64p, C.c_int, _i8p, C.POINTER(C.c_int)]
        L.or_direct_interp.argtypes = [C.c_int, _i32p, _i32p, _f64p, _u8p, _i8p, _i32p, C.POINTER(C.c_int),
                                       _i32p, _i32p, _f64p, C.c_longlong]
        L.or_ext_interp.argtypes = [C.c_int, _i32p, _i32p, _f64p, _u8p, _i8p, _i32p, C.POINTER(C.c_int),
                                    _i32p, _i32p, _f64p, C.c_longlong]
        L.or_direct_interp_bs.argtypes = [C.c_int, _i32p, _i32p, _f64p, _u8p, _i8p, C.c_int, _i32p,
                                          C.POINTER(C.c_int), _i32p, _i32p, _f64p, C.c_longlong]
        L.or_block_strength.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, C.c_double, C.POINTER(C.c_int),
                                        _i32p, _i32p, _u8p, _u8p]
        L.or_setup_ex.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_uint64, C.c_int, C.c_int,
                                  C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.or_fsai.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
        L.or_fsai_sweep.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, C.c_double, _f64p, _f64p]
        L.or_G_nnz.argtypes = [C.c_void_p, C.c_int]
        L.or_get_G.argtypes = [C.c_void_p, C.c_int, _i32p, _i32p, _f64p]
        L.or_setup_bs.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_uint64, C.c_int, C.c_int,
                                  C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.or_galerkin.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, _i32p, _i32p, _f64p,
                                  C.POINTER(C.c_int), C.POINTER(C.POINTER(C.c_int)),
                                  C.POINTER(C.POINTER(C.c_int)), C.POINTER(C.POINTER(C.c_double))]
        L.or_free_array.argtypes = [C.c_void_p]
        L.or_cholesky.argtypes = [C.c_int, _f64p]
        L.or_cholesky_solve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
        L.or_spmv.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_jacobi_sweep.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, _f64p, _f64p]
        L.or_setup.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_uint64, C.c_int, C.c_int,
                               C.c_double, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.or_free.argtypes = [C.c_void_p]
        L.or_nlevels.argtypes = [C.c_void_p]
        L.or_level_info.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.or_get_A.argtypes = [C.c_void_p, C.c_int, _i32p, _i32p, _f64p]
        L.or_get_P.argtypes = [C.c_void_p, C.c_int, _i32p, _i32p, _f64p]
        L.or_get_cf.argtypes = [C.c_void_p, C.c_int, _i8p]
        L.or_get_S.argtypes = [C.c_void_p, C.c_int, _u8p]
        L.or_complexities.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_vcycle.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_pcg.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int, C.c_int, C.c_int,
                             C.POINTER(C.c_int), _f64p, C.c_void_p]
    return L


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def check_csr(A) -> int:
    return lib().or_check_csr(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val))


def strength(A, theta: float) -> np.ndarray:
    S = np.zeros(A.nnz, dtype=np.uint8)
    lib().or_strength(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), theta, S)
    return S


def splitmix64(seed: int, c: int) -> int:
    return int(lib().or_splitmix64(seed, c))


def pmis_random(seed: int, level: int, i: int) -> float:
    return float(lib().or_pmis_random(seed, level, i))


def pmis(A, S: np.ndarray, seed: int, level: int = 0) -> np.ndarray:
    cf = np.zeros(A.n, dtype=np.int8)
    st = lib().or_pmis(A.n, _i32(A.rowptr), _i32(A.col), np.ascontiguousarray(S, np.uint8), seed, level, cf)
    if st:
        raise RuntimeError(f"or_pmis failed: {st}")
    return cf


def pmis_rounds(A, S: np.ndarray, lam, max_rounds: int = -1, L=None):
    """PMIS with given measures: (state after max_rounds rounds, rounds run).

    state[i] = 1 C, 0 F, -1 still undecided; max_rounds < 0 runs to the end.
    L: a loaded oracle library (default: this one)."""
    L = L or lib()
    st = np.zeros(A.n, dtype=np.int8)
    r = C.c_int(0)
    ret = L.or_pmis_rounds(A.n, _i32(A.rowptr), _i32(A.col), np.ascontiguousarray(S, np.uint8), _f64(lam),
                           max_rounds, st, C.byref(r))
    if ret:
        raise RuntimeError(f"or_pmis_rounds failed: {ret}")
    return st, r.value


def block_strength(A, bs: int, theta: float):
    """Nodal block strength: returns (node rowptr, node col, node strength, unknown-wise strength)."""
    nn = C.c_int(0)
    Nrp = np.zeros(A.n // bs + 1, np.int32)
    Nci = np.zeros(max(A.nnz, 1), np.int32)
    SN = np.zeros(max(A.nnz, 1), np.uint8)
    S = np.zeros(max(A.nnz, 1), np.uint8)
    st = lib().or_block_strength(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), bs, theta, C.byref(nn), Nrp, Nci,
                                 SN, S)
    if st:
        raise RuntimeError(f"or_block_strength failed: {st}")
    e = int(Nrp[-1])
    return Nrp, Nci[:e].copy(), SN[:e].copy(), S[: A.nnz].copy()


def direct_interp(A, S: np.ndarray, cf: np.ndarray, bs: int = 1):
    """Returns (P_rowptr, P_col, P_val, nc); bs > 1 interpolates unknown-wise."""
    cap = A.nnz + A.n
    rp = np.zeros(A.n + 1, np.int32)
    ci = np.zeros(cap, np.int32)
    v = np.zeros(cap, np.float64)
    cidx = np.zeros(A.n, np.int32)
    nc = C.c_int(0)
    st = lib().or_direct_interp_bs(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), np.ascontiguousarray(S, np.uint8),
                                   np.ascontiguousarray(cf, np.int8), bs, cidx, C.byref(nc), rp, ci, v, cap)
    if st:
        raise RuntimeError(f"or_direct_interp failed: {st}")
    nnz = int(rp[-1])
    return rp, ci[:nnz].copy(), v[:nnz].copy(), nc.value


def ext_interp(A, S: np.ndarray, cf: np.ndarray):
    """Extended+i interpolation: (P_rowptr, P_col, P_val, nc)."""
    lens = np.diff(A.rowptr)
    cap = A.n + int(lens[A.col].sum())
    rp = np.zeros(A.n + 1, np.int32)
    ci = np.zeros(max(cap, 1), np.int32)
    v = np.zeros(max(cap, 1), np.float64)
    cidx = np.zeros(A.n, np.int32)
    nc = C.c_int(0)
    st = lib().or_ext_interp(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), np.ascontiguousarray(S, np.uint8),
                             np.ascontiguousarray(cf, np.int8), cidx, C.byref(nc), rp, ci, v, cap)
    if st:
        raise RuntimeError(f"or_ext_interp failed: {st}")
    nnz = int(rp[-1])
    return rp, ci[:nnz].copy(), v[:nnz].copy(), nc.value


def galerkin(A, P_rowptr, P_col, P_val, nc: int):
    """A_c = P^T A P as (rowptr, col, val)."""
    nnz = C.c_int(0)
    rp = C.POINTER(C.c_int)()
    ci = C.POINTER(C.c_int)()
    v = C.POINTER(C.c_double)()
    st = lib().or_galerkin(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), nc, _i32(P_rowptr), _i32(P_col),
                           _f64(P_val), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(v))
    if st:
        raise RuntimeError(f"or_galerkin failed: {st}")
    out = (np.ctypeslib.as_array(rp, (nc + 1,)).copy(), np.ctypeslib.as_array(ci, (max(nnz.value, 1),))[:nnz.value].copy(),
           np.ctypeslib.as_array(v, (max(nnz.value, 1),))[:nnz.value].copy())
    for p in (rp, ci, v):
        lib().or_free_array(C.cast(p, C.c_void_p))
    return out


def fsai(A):
    """Static FSAI factor G (lower triangle of A's pattern) as (rowptr, col, val)."""
    rp = np.zeros(A.n + 1, np.int32)
    ci = np.zeros(max(A.nnz, 1), np.int32)
    v = np.zeros(max(A.nnz, 1))
    st = lib().or_fsai(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), rp, ci, v)
    if st:
        raise RuntimeError(f"or_fsai failed: {st}")
    nnz = int(rp[-1])
    return rp, ci[:nnz].copy(), v[:nnz].copy()


def fsai_sweep(A, G, omega: float, y: np.ndarray, s: np.ndarray) -> np.ndarray:
    s = _f64(s).copy()
    lib().or_fsai_sweep(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), _i32(G[0]), _i32(G[1]), _f64(G[2]), omega,
                        _f64(y), s)
    return s


def cholesky(M: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(M, dtype=np.float64).copy()
    st = lib().or_cholesky(L.shape[0], L)
    if st:
        raise RuntimeError(f"or_cholesky failed: {st}")
    return L


def cholesky_solve(L: np.ndarray, y: np.ndarray) -> np.ndarray:
    z = np.zeros(L.shape[0])
    lib().or_cholesky_solve(L.shape[0], _f64(L), _f64(y), z)
    return z


def spmv(A, x: np.ndarray) -> np.ndarray:
    y = np.zeros(A.n)
    lib().or_spmv(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), _f64(x), y)
    return y


def jacobi_sweep(A, omega: float, y: np.ndarray, s: np.ndarray) -> np.ndarray:
    s = _f64(s).copy()
    lib().or_jacobi_sweep(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), omega, _f64(y), s)
    return s


@dataclass
class Level:
    n: int
    A: tuple
    P: tuple | None
    cf: np.ndarray | None
    S: np.ndarray | None


class Hierarchy:
    """Oracle AMG hierarchy (Algorithm 1) with V-cycle and PCG (Algorithm 2, Sec. 4)."""

    SMOOTHERS = {"jacobi": 0, "fsai": 1}
    INTERPS = {"direct": 0, "ext": 1}

    def __init__(self, A, theta=0.25, seed=0, max_coarse=64, max_levels=25, omega=2.0 / 3.0, nu1=1, nu2=1,
                 block_size=1, smoother="jacobi", interp="direct"):
        self._keep = (_i32(A.rowptr), _i32(A.col), _f64(A.val))
        h = C.c_void_p()
        st = lib().or_setup_ex(A.n, *self._keep, theta, seed, max_coarse, max_levels, omega, nu1, nu2, block_size,
                               self.SMOOTHERS[smoother], self.INTERPS[interp], C.byref(h))
        if st:
            raise RuntimeError(f"or_setup failed: {st}")
        self.h = h
        self.n = A.n

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    @property
    def nlevels(self) -> int:
        return lib().or_nlevels(self.h)

    def level_sizes(self, k: int):
        n, na, npn = C.c_int(), C.c_int(), C.c_int()
        lib().or_level_info(self.h, k, C.byref(n), C.byref(na), C.byref(npn))
        return n.value, na.value, npn.value

    def A(self, k: int):
        n, na, _ = self.level_sizes(k)
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(max(na, 1), np.int32), np.zeros(max(na, 1))
        lib().or_get_A(self.h, k, rp, ci, v)
        return rp, ci[:na], v[:na]

    def P(self, k: int):
        n, _, npn = self.level_sizes(k)
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(max(npn, 1), np.int32), np.zeros(max(npn, 1))
        lib().or_get_P(self.h, k, rp, ci, v)
        return rp, ci[:npn], v[:npn]

    def G(self, k: int):
        """FSAI factor of level k as (rowptr, col, val) (smoother "fsai", k < nlevels - 1)."""
        n, _, _ = self.level_sizes(k)
        ng = lib().or_G_nnz(self.h, k)
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(max(ng, 1), np.int32), np.zeros(max(ng, 1))
        lib().or_get_G(self.h, k, rp, ci, v)
        return rp, ci[:ng], v[:ng]

    def cf(self, k: int) -> np.ndarray:
        n, _, _ = self.level_sizes(k)
        cf = np.zeros(n, np.int8)
        lib().or_get_cf(self.h, k, cf)
        return cf

    def S(self, k: int) -> np.ndarray:
        _, na, _ = self.level_sizes(k)
        S = np.zeros(na, np.uint8)
        lib().or_get_S(self.h, k, S)
        return S

    def complexities(self):
        a, b = C.c_double(), C.c_double()
        lib().or_complexities(self.h, C.byref(a), C.byref(b))
        return a.value, b.value

    def vcycle(self, y: np.ndarray) -> np.ndarray:
        z = np.zeros(self.n)
        lib().or_vcycle(self.h, _f64(y), z)
        return z

    def pcg(self, b, x0=None, rtol=1e-8, maxit=500, flexible=False, precond=True, keep_iterates=False):
        """Returns (status, x, iters, residual-norm history[0..iters], iterates or None)."""
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        hist = np.zeros(maxit + 1)
        it = C.c_int(0)
        xh = np.zeros((maxit, self.n)) if keep_iterates else None
        st = lib().or_pcg(self.h, _f64(b), x, rtol, maxit, int(flexible), int(precond), C.byref(it), hist,
                          xh.ctypes.data if xh is not None else None)
        k = it.value
        return st, x, k, hist[:k + 1].copy(), (xh[:k].copy() if xh is not None else None)
