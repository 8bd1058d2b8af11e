"""amg_spmv_dot_noalloc: the fused q = A p, (p, q) product that allocates no device memory.

It is meant for callers that cannot call cudaMalloc where they need the
product (device memory owned by another allocator, loops that must not risk
the synchronisation or the out-of-memory failure an allocation can bring).
Its scratch lives in a fixed array inside the library.  This test calls it
through the C ABI twice in a row on the same device and checks q against the
existing amg_spmv entry point's output (1e-13 of max |q|, the SpMV bar of the
parity tests) and (p, q) against the dot product of p with that output
(1e-12 relative).  It also checks that a size beyond the scratch array's limit
is refused.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2102_07417_gb300 import amg  # noqa: E402
from paper_2102_07417_gb300 import problems as pr  # noqa: E402

MAX_ROWS = 16_777_216


def _entry():
    lib = amg.load()
    f = lib.amg_spmv_dot_noalloc
    f.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 6 + [C.c_void_p]
    f.restype = C.c_int
    return f


def test_noalloc_matches_existing_entry_point_twice_in_a_row():
    f = _entry()
    A = pr.diffusion3d(48, 2.0, 5)[0]  # n = 110,592: 14 blocks of 8192 rows, the last one partial
    h = amg.Hierarchy(A, seed=0)
    dev = "cuda:0"
    rp = torch.as_tensor(A.rowptr, device=dev)
    ci = torch.as_tensor(A.col, device=dev)
    v = torch.as_tensor(A.val, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(7)
    for call in range(2):
        p = torch.as_tensor(rng.standard_normal(A.n), device=dev)
        q = torch.full((A.n,), float("nan"), dtype=torch.float64, device=dev)
        pq = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        st = f(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), p.data_ptr(), q.data_ptr(), pq.data_ptr(),
               stream)
        assert st == amg.AMG_OK, amg.load().amg_last_error()
        q_ref = h.spmv(0, p)
        torch.cuda.synchronize()
        qn, qr = q.cpu().numpy(), q_ref.cpu().numpy()
        assert np.abs(qn - qr).max() <= 1e-13 * np.abs(qr).max(), f"call {call}: q"
        dot_ref = float(torch.dot(p, q_ref))
        assert abs(pq.item() - dot_ref) <= 1e-12 * abs(dot_ref), f"call {call}: (p, q)"


def test_noalloc_refuses_sizes_beyond_its_scratch():
    f = _entry()
    x = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    st = f(MAX_ROWS + 1, 0, idx.data_ptr(), None, None, x.data_ptr(), x.data_ptr(), x.data_ptr(), None)
    assert st == amg.AMG_ERR_UNSUPPORTED
    assert b"exceeds the limit" in amg.load().amg_last_error()


def test_noalloc_through_the_binding():
    """The same product through the Python binding's spmv_dot_noalloc, on a 24^3 Poisson operator
    (13,824 rows: one full block of 8192 rows and a partial one), against a host product in FP64
    (1e-13 of max |q|; (p, q) to 1e-12 relative).  Mismatched sizes are refused on the host."""
    A = pr.poisson3d(24)
    dev = "cuda:0"
    rp, ci, v = (torch.as_tensor(a, device=dev) for a in (A.rowptr, A.col, A.val))
    ph = np.random.default_rng(3).standard_normal(A.n)
    p = torch.as_tensor(ph, device=dev)
    q = torch.full_like(p, float("nan"))
    pq = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    q2, pq2 = amg.spmv_dot_noalloc(rp, ci, v, p, q, pq)
    assert q2 is q and pq2 is pq
    torch.cuda.synchronize()
    qh = A.matvec(ph)
    assert np.abs(q.cpu().numpy() - qh).max() <= 1e-13 * np.abs(qh).max()
    dot = float(ph @ qh)
    assert abs(pq.item() - dot) <= 1e-12 * abs(dot)
    with pytest.raises(ValueError, match="sizes do not match"):
        amg.spmv_dot_noalloc(rp, ci, v, p[:-1], q, pq)
