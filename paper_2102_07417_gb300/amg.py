"""Python binding of libamg's C ABI (include/amg.h): argument marshalling only.

Every step of the set-up and the solve runs in libamg's CUDA kernels; this
module converts numpy arrays / torch tensors to pointers, passes the current
torch CUDA stream, and optionally routes libamg's device allocations through
PyTorch's caching allocator.  There is no CPU fallback: if libamg.so cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

AMG_OK = 0
AMG_ERR_INVALID_ARG = -1
AMG_ERR_NOT_SPD = -2
AMG_ERR_BREAKDOWN = -3
AMG_ERR_NO_CONVERGENCE = -4
AMG_ERR_SETUP = -5
AMG_ERR_OOM = -6
AMG_ERR_CUDA = -7
AMG_ERR_TIMEOUT = -8
AMG_ERR_UNSUPPORTED = -9

PREC_FP64, PREC_FP32, PREC_FP32_BF16PR = 0, 1, 2
SMOOTH_JACOBI, SMOOTH_FSAI = 0, 1
INTERP_DIRECT, INTERP_EXT = 0, 1

KERNEL_NAMES = ["spmv_dot", "pcg_update", "smooth_resid", "restrict", "prolong", "smooth_post", "coarse",
                "direction", "solve_other", "strength", "pmis", "interp", "transpose", "spgemm", "setup_other",
                "smooth_fsai", "fsai"]
SOLVE_KERNELS = KERNEL_NAMES[:9] + ["smooth_fsai"]
SETUP_KERNELS = KERNEL_NAMES[9:15] + ["fsai"]

# Names exported by the C ABI (each declared in include/amg.h).
EXPORTS = ["amg_params_default", "amg_setup", "amg_pcg_solve", "amg_pcg_solve_batch", "amg_vcycle_apply", "amg_spmv", "amg_solve",
           "amg_hierarchy_info", "amg_hierarchy_export", "amg_hierarchy_bytes", "amg_free", "amg_profile_enable",
           "amg_profile_read", "amg_profile_filter", "amg_launch_count", "amg_status_string", "amg_last_error",
           "amg_spmv_dot_noalloc", "amg_slots_create", "amg_slots_admit", "amg_slots_step", "amg_slots_poll",
           "amg_slots_query", "amg_slots_wait", "amg_slots_retire", "amg_slots_free", "amg_hierarchy_export_fsai"]


class AmgError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {code})")
        self.code = code


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("theta", C.c_double), ("seed", C.c_uint64), ("max_coarse", C.c_int32), ("max_levels", C.c_int32),
                ("omega", C.c_double), ("nu1", C.c_int32), ("nu2", C.c_int32), ("precision", C.c_int32),
                ("block_size", C.c_int32), ("smoother", C.c_int32), ("interp", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("nlevels", C.c_int32), ("final_residual", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libamg.so (building it first if asked); raises if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not os.path.exists(path):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libamg.so not found at {path}; run paper_2102_07417_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.amg_params_default.argtypes = [C.POINTER(Params)]
    L.amg_setup.argtypes = [C.POINTER(Csr), C.POINTER(Params), C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.amg_pcg_solve.argtypes = [vp, vp, vp, dbl, i32, vp, C.POINTER(i32), vp, i32]
    L.amg_pcg_solve_batch.argtypes = [vp, i32, vp, vp, dbl, i32, vp, vp, vp, vp, i32]
    L.amg_vcycle_apply.argtypes = [vp, vp, vp, vp]
    L.amg_slots_create.argtypes = [vp, i32, dbl, i32, vp, C.POINTER(vp)]
    L.amg_slots_admit.argtypes = [vp, i32, vp]
    L.amg_slots_step.argtypes = [vp]
    L.amg_slots_poll.argtypes = [vp, vp, vp]
    L.amg_slots_retire.argtypes = [vp, i32, vp]
    L.amg_slots_query.argtypes = [vp, vp, vp, C.POINTER(i64), C.POINTER(i64)]
    L.amg_slots_wait.argtypes = [vp]
    L.amg_slots_free.argtypes = [vp]
    L.amg_slots_free.restype = None
    L.amg_spmv.argtypes = [vp, i32, vp, vp, vp]
    L.amg_spmv_dot_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp]
    L.amg_solve.argtypes = [C.POINTER(Csr), vp, vp, C.POINTER(Params), dbl, i32, C.POINTER(Allocator), vp,
                            C.POINTER(Result)]
    L.amg_hierarchy_info.argtypes = [vp, C.POINTER(i32), i32, vp, vp, vp, C.POINTER(dbl), C.POINTER(dbl)]
    L.amg_hierarchy_export.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.amg_hierarchy_export_fsai.argtypes = [vp, i32, C.POINTER(i64), vp, vp, vp]
    L.amg_hierarchy_bytes.argtypes = [vp]
    L.amg_hierarchy_bytes.restype = C.c_size_t
    L.amg_free.argtypes = [vp]
    L.amg_free.restype = None
    L.amg_profile_enable.argtypes = [i32]
    L.amg_profile_read.argtypes = [i32, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]
    L.amg_profile_filter.argtypes = [i32, i32]
    L.amg_launch_count.argtypes = []
    L.amg_launch_count.restype = C.c_int64
    L.amg_status_string.argtypes = [C.c_int]
    L.amg_status_string.restype = C.c_char_p
    L.amg_last_error.argtypes = []
    L.amg_last_error.restype = C.c_char_p
    _lib = L
    return L


def check(code: int, where: str):
    if code != AMG_OK:
        L = load()
        raise AmgError(code, where, f"{L.amg_status_string(code).decode()}: {L.amg_last_error().decode()}")


def default_params(**kw) -> Params:
    """amg_params_default with keyword overrides.  With smoother=SMOOTH_FSAI and no omega given,
    omega = 1 (omega rho(G^T G A) ~ 1.37 < 2 on 3-D Poisson, the condition after Eq. smoother)."""
    p = Params()
    check(load().amg_params_default(C.byref(p)), "amg_params_default")
    if kw.get("smoother") == SMOOTH_FSAI and "omega" not in kw:
        kw["omega"] = 1.0
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class TorchAllocator:
    """Routes libamg allocations through torch's caching allocator."""

    def __init__(self):
        import torch

        self._torch = torch

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
            except Exception:  # out of memory: libamg turns NULL into AMG_ERR_OOM
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


def _ptr(t) -> int:
    return int(t.data_ptr())


class Hierarchy:
    """An AMG hierarchy resident on the GPU (Algorithm 1), with PCG / V-cycle entry points.

    ``A`` is a CSR object with numpy (host) arrays ``rowptr``, ``col``, ``val``
    and ``n``, or the same fields as CUDA torch tensors (int32 / float64).
    """

    def __init__(self, A, params: Params | None = None, stream=None, torch_allocator: bool = True, **kw):
        import torch

        L = load()
        self.params = params if params is not None else default_params(**kw)
        self._alloc = TorchAllocator() if torch_allocator else None
        on_dev = isinstance(A.rowptr, torch.Tensor) and A.rowptr.is_cuda
        if on_dev:
            rp, ci, v = A.rowptr, A.col, A.val
            ptrs = (_ptr(rp), _ptr(ci), _ptr(v))
        else:
            rp = np.ascontiguousarray(A.rowptr, np.int32)
            ci = np.ascontiguousarray(A.col, np.int32)
            v = np.ascontiguousarray(A.val, np.float64)
            ptrs = (rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        self.n = int(A.n)
        self.nnz = int(rp[-1]) if not on_dev else int(rp[-1].item())
        csr = Csr(self.n, self.nnz, *ptrs, 1 if on_dev else 0)
        self.tstream = stream
        self.stream = _stream_handle(stream)
        if hasattr(stream, "wait_stream"):  # A may come from work queued on the current stream
            stream.wait_stream(torch.cuda.current_stream())
        h = C.c_void_p()
        check(L.amg_setup(C.byref(csr), C.byref(self.params), C.byref(self._alloc.struct) if self._alloc else None,
                          self.stream, C.byref(h)), "amg_setup")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().amg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _on(self, stream) -> int:
        """Handle of the stream a call runs on (the given one, else the hierarchy's), ordered
        after the work already queued on the caller's current stream."""
        import torch

        s = stream if stream is not None else self.tstream
        if hasattr(s, "wait_stream"):
            s.wait_stream(torch.cuda.current_stream())
        return _stream_handle(s) if stream is not None else self.stream

    def _after(self, stream):
        """Order the caller's current stream after a stream-ordered call."""
        import torch

        s = stream if stream is not None else self.tstream
        if hasattr(s, "wait_stream"):
            torch.cuda.current_stream().wait_stream(s)

    # -- solve phase ---------------------------------------------------------
    def solve(self, b, x=None, rtol: float = 1e-8, maxit: int = 500, hist: bool = False, stream=None):
        """PCG to ||r|| < rtol ||b||.  b, x: CUDA float64 tensors (x holds x0; default zeros).
        Returns (x, iters, status, history or None); raises on errors other than non-convergence."""
        import torch

        if x is None:
            x = torch.zeros_like(b)
        hbuf = np.zeros(maxit + 1) if hist else None
        it = C.c_int32(0)
        st = load().amg_pcg_solve(self.h, _ptr(b), _ptr(x), rtol, maxit, self._on(stream),
                                  C.byref(it), hbuf.ctypes.data if hist else None, maxit + 1 if hist else 0)
        if st not in (AMG_OK, AMG_ERR_NO_CONVERGENCE):
            check(st, "amg_pcg_solve")
        return x, it.value, st, (hbuf[: it.value + 1].copy() if hist else None)

    def solve_batch(self, B, X=None, rtol: float = 1e-8, maxit: int = 500, hist: bool = False, stream=None):
        """PCG on the k columns of B (CUDA float64, n x k row-major) at once.
        Returns (X, iters[k], status[k], overall status, history (maxit+1, k) or None)."""
        import torch

        k = 1 if B.dim() == 1 else int(B.shape[1])
        B = B.contiguous()
        if X is None:
            X = torch.zeros_like(B)
        it = np.zeros(k, np.int32)
        stv = np.zeros(k, np.int32)
        hbuf = np.zeros((maxit + 1, k)) if hist else None
        st = load().amg_pcg_solve_batch(self.h, k, _ptr(B), _ptr(X), rtol, maxit,
                                        self._on(stream), it.ctypes.data,
                                        stv.ctypes.data, hbuf.ctypes.data if hist else None, maxit + 1 if hist else 0)
        if st not in (AMG_OK, AMG_ERR_NO_CONVERGENCE, AMG_ERR_BREAKDOWN):
            check(st, "amg_pcg_solve_batch")
        return X, it.tolist(), stv.tolist(), st, hbuf

    def slots(self, capacity: int, rtol: float = 1e-8, maxit: int = 500, stream=None) -> "Slots":
        """A continuous-batching block of ``capacity`` PCG columns on this hierarchy."""
        return Slots(self, capacity, rtol, maxit, stream)

    def vcycle(self, y, z=None, stream=None):
        import torch

        if z is None:
            z = torch.empty_like(y)
        check(load().amg_vcycle_apply(self.h, _ptr(y), _ptr(z), self._on(stream)),
              "amg_vcycle_apply")
        self._after(stream)
        return z

    def spmv(self, level: int, x, y=None, stream=None):
        import torch

        if y is None:
            y = torch.empty(self.info()["n"][level], dtype=torch.float64, device=x.device)
        check(load().amg_spmv(self.h, level, _ptr(x), _ptr(y), self._on(stream)),
              "amg_spmv")
        self._after(stream)
        return y

    # -- inspection ----------------------------------------------------------
    def info(self) -> dict:
        L = load()
        nl = C.c_int32()
        cap = 64
        n = np.zeros(cap, np.int64)
        nz = np.zeros(cap, np.int64)
        npz = np.zeros(cap, np.int64)
        cgd, cop = C.c_double(), C.c_double()
        check(L.amg_hierarchy_info(self.h, C.byref(nl), cap, n.ctypes.data, nz.ctypes.data, npz.ctypes.data,
                                   C.byref(cgd), C.byref(cop)), "amg_hierarchy_info")
        k = nl.value
        return {"nlevels": k, "n": n[:k].tolist(), "nnz": nz[:k].tolist(), "nnzP": npz[:k].tolist(),
                "cgd": cgd.value, "cop": cop.value}

    def export(self, level: int) -> dict:
        inf = self.info()
        n, nnz, nnzp = inf["n"][level], inf["nnz"][level], inf["nnzP"][level]
        cf = np.zeros(n, np.int8)
        arp, aci, av = np.zeros(n + 1, np.int32), np.zeros(max(nnz, 1), np.int32), np.zeros(max(nnz, 1))
        prp, pci, pv = np.zeros(n + 1, np.int32), np.zeros(max(nnzp, 1), np.int32), np.zeros(max(nnzp, 1))
        check(load().amg_hierarchy_export(self.h, level, cf.ctypes.data, arp.ctypes.data, aci.ctypes.data,
                                          av.ctypes.data, prp.ctypes.data, pci.ctypes.data, pv.ctypes.data),
              "amg_hierarchy_export")
        return {"cf": cf, "A": (arp, aci[:nnz], av[:nnz]), "P": (prp, pci[:nnzp], pv[:nnzp])}

    def export_fsai(self, level: int):
        """FSAI factor G of a level as (rowptr, col, val), or None (Jacobi smoother, last level)."""
        L = load()
        nnz = C.c_int64(0)
        check(L.amg_hierarchy_export_fsai(self.h, level, C.byref(nnz), None, None, None), "amg_hierarchy_export_fsai")
        if nnz.value == 0:
            return None
        n = self.info()["n"][level]
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz.value, np.int32), np.zeros(nnz.value)
        check(L.amg_hierarchy_export_fsai(self.h, level, None, rp.ctypes.data, ci.ctypes.data, v.ctypes.data),
              "amg_hierarchy_export_fsai")
        return rp, ci, v

    def nbytes(self) -> int:
        return int(load().amg_hierarchy_bytes(self.h))




SLOT_FREE, SLOT_RUNNING, SLOT_CONVERGED = 0, 1, 2


class Slots:
    """Continuous batching on one hierarchy: up to 32 requests share each SpMM and V-cycle.

    ``admit(j, b)`` starts PCG (x0 = 0) for right-hand side ``b`` in slot j,
    ``step()`` runs one iteration of every running slot, ``poll()`` returns the
    per-slot states (0 free, 1 running, 2 converged, < 0 error) and iteration
    counts, ``retire(j)`` returns slot j's solution and frees the slot.  All
    calls are ordered on the object's stream; ``poll`` synchronises it.
    """

    def __init__(self, hier: Hierarchy, capacity: int, rtol: float, maxit: int, stream=None):
        import torch

        self.hier = hier
        self.capacity = int(capacity)
        self.n = hier.n
        # a stream of its own (steps are captured into a CUDA graph and replayed on it)
        self.tstream = stream if stream is not None else torch.cuda.Stream()
        self.stream = _stream_handle(self.tstream)
        self._state = np.zeros(self.capacity, np.int32)
        self._iters = np.zeros(self.capacity, np.int32)
        h = C.c_void_p()
        check(load().amg_slots_create(hier.h, self.capacity, rtol, maxit, self.stream, C.byref(h)), "amg_slots_create")
        self.s = h
        self._torch = torch

    def admit(self, slot: int, b):
        """Start PCG for right-hand side b (CUDA float64, n) in a free slot."""
        self.tstream.wait_stream(self._torch.cuda.current_stream())
        b.record_stream(self.tstream)
        check(load().amg_slots_admit(self.s, int(slot), _ptr(b)), "amg_slots_admit")

    def step(self):
        check(load().amg_slots_step(self.s), "amg_slots_step")

    def poll(self):
        check(load().amg_slots_poll(self.s, self._state.ctypes.data, self._iters.ctypes.data), "amg_slots_poll")
        return self._state.copy(), self._iters.copy()

    def query(self):
        """(state, iters, steps finished, steps launched) from the newest finished step, without
        waiting; a slot admitted after that step reads as running."""
        d, i = C.c_int64(0), C.c_int64(0)
        check(load().amg_slots_query(self.s, self._state.ctypes.data, self._iters.ctypes.data, C.byref(d),
                                     C.byref(i)), "amg_slots_query")
        return self._state.copy(), self._iters.copy(), d.value, i.value

    def wait(self):
        """Block until the oldest step in flight has finished."""
        check(load().amg_slots_wait(self.s), "amg_slots_wait")

    def retire(self, slot: int, x=None):
        """Slot's solution (into x, or a new tensor) and the slot freed; ordered before later
        work on the caller's current stream."""
        torch = self._torch
        cur = torch.cuda.current_stream()
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self.tstream.wait_stream(cur)
        check(load().amg_slots_retire(self.s, int(slot), _ptr(x)), "amg_slots_retire")
        x.record_stream(self.tstream)
        cur.wait_stream(self.tstream)
        return x

    def close(self):
        if getattr(self, "s", None):
            load().amg_slots_free(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

def profile(on: bool):
    """Start (clearing totals) or stop process-wide per-launch CUDA-event timing."""
    check(load().amg_profile_enable(1 if on else 0), "amg_profile_enable")


def profile_filter(kernel: str | None = None, level: int = -1):
    """Record only launches of one kernel class (name from KERNEL_NAMES) on one level (-1: any); None: all."""
    k = -1 if kernel is None else KERNEL_NAMES.index(kernel)
    check(load().amg_profile_filter(k, level), "amg_profile_filter")


def profile_read(level: int = -1) -> dict:
    """Per kernel class (on one level, or all with -1): launches, summed event time (ms), algorithmic bytes."""
    out = {}
    for k, name in enumerate(KERNEL_NAMES):
        n, ms, by = C.c_int64(), C.c_double(), C.c_double()
        check(load().amg_profile_read(k, level, C.byref(n), C.byref(ms), C.byref(by)), "amg_profile_read")
        out[name] = {"launches": n.value, "ms": ms.value, "bytes": by.value}
    return out


def launch_count() -> int:
    """libamg kernel launches in this process so far."""
    return int(load().amg_launch_count())


def spmv_dot_noalloc(rowptr, col, val, p, q, pq, stream=None):
    """q = A p and pq[0] = (p, A p) in one launch that allocates no device memory
    (amg_spmv_dot_noalloc).  A is CSR as contiguous CUDA tensors rowptr (int32, n + 1), col (int32)
    and val (float64); p and q are float64 CUDA tensors of n entries and pq one of at least one,
    all owned by the caller.  Stream-ordered on `stream`; nothing is synchronised.  Calls that
    overlap on the GPU share the library's scratch and must be serialised.  Returns (q, pq)."""
    import torch

    for name, t, dt in (("rowptr", rowptr, torch.int32), ("col", col, torch.int32), ("val", val, torch.float64),
                        ("p", p, torch.float64), ("q", q, torch.float64), ("pq", pq, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"spmv_dot_noalloc: {name} must be a contiguous CUDA tensor of {dt}")
    n = rowptr.numel() - 1
    if col.numel() != val.numel() or p.numel() != n or q.numel() != n or pq.numel() < 1:
        raise ValueError(f"spmv_dot_noalloc: sizes do not match n = {n} rows "
                         f"(col {col.numel()}, val {val.numel()}, p {p.numel()}, q {q.numel()}, pq {pq.numel()})")
    if col.numel() > 2**31 - 1:
        raise ValueError(f"spmv_dot_noalloc: {col.numel()} nonzeros exceed the C ABI's int32 count")
    check(load().amg_spmv_dot_noalloc(n, col.numel(), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(p), _ptr(q),
                                      _ptr(pq), _stream_handle(stream)), "amg_spmv_dot_noalloc")
    return q, pq


def solve(A, b, x0=None, params: Params | None = None, rtol: float = 1e-8, maxit: int = 500, stream=None,
          torch_allocator: bool = True, **kw):
    """One-call set-up + solve (amg_solve).  Host (numpy) or device (torch CUDA) inputs.
    A host x0 (contiguous float64) receives the solution in place.  Returns (x, Result)."""
    import torch

    L = load()
    prm = params if params is not None else default_params(**kw)
    on_dev = isinstance(A.rowptr, torch.Tensor) and A.rowptr.is_cuda
    keep = []
    if on_dev:
        ptrs = (_ptr(A.rowptr), _ptr(A.col), _ptr(A.val))
        nnz = int(A.rowptr[-1].item())
        x = torch.zeros_like(b) if x0 is None else x0
        bp, xp = _ptr(b), _ptr(x)
    else:
        rp = np.ascontiguousarray(A.rowptr, np.int32)
        ci = np.ascontiguousarray(A.col, np.int32)
        v = np.ascontiguousarray(A.val, np.float64)
        keep += [rp, ci, v]
        ptrs = (rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        nnz = int(rp[-1])
        bb = np.ascontiguousarray(b, np.float64)
        x = np.zeros(A.n) if x0 is None else np.ascontiguousarray(x0, np.float64)
        keep.append(bb)
        bp, xp = bb.ctypes.data, x.ctypes.data
    csr = Csr(int(A.n), nnz, *ptrs, 1 if on_dev else 0)
    alloc = TorchAllocator() if torch_allocator else None
    res = Result()
    st = L.amg_solve(C.byref(csr), bp, xp, C.byref(prm), rtol, maxit, C.byref(alloc.struct) if alloc else None,
                     _stream_handle(stream), C.byref(res))
    if st not in (AMG_OK, AMG_ERR_NO_CONVERGENCE):
        check(st, "amg_solve")
    return x, res
