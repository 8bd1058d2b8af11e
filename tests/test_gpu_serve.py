"""Serving with continuous batching: each result is the same alone and in the mix.

Bar: a right-hand-side request served in the mix (admitted into slot s of a
running batch, beside other requests that come and go) equals, value for
value, the same request served alone in slot s of an otherwise empty batch of
the same capacity; it is within 1e-6 relative of a single-column
amg_pcg_solve of the same system (both stop at rtol 1e-8; the summation order
of the dot products differs).  A new-matrix request equals its own set-up and
solve run alone (set-up and solve are deterministic).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2102_07417_gb300 import amg  # noqa: E402
from paper_2102_07417_gb300 import problems as pr  # noqa: E402
from paper_2102_07417_gb300 import serve  # noqa: E402


def _small_server(**kw):
    ops = serve.resident_operators(sizes=(16, 24), sigma=1.0, seed0=40)
    return ops, serve.Server(ops, precision=amg.PREC_FP32, capacity=4, rtol=1e-8, maxit=200, keep_x=True, **kw)


def test_serve_same_alone_and_in_mix():
    ops, srv = _small_server()
    reqs = serve.make_requests(40, rate=4000.0, seed=4, frac_matrix=0.25, n_resident=2, m_range=(10, 20))
    res = srv.run(reqs)
    assert len(res) == 40 and all(r.status == amg.AMG_OK for r in res)
    assert srv.stats["max_running_slots"] > 1  # requests overlapped on the device
    for r, q in zip(res, reqs):
        if q.kind == "rhs":
            h = srv.hier[q.target]
            b = serve.rhs_for(q, h.n)
            alone = h.slots(r.capacity, rtol=1e-8, maxit=200)
            alone.admit(r.slot, b)
            while True:
                alone.step()
                state, iters = alone.poll()
                if state[r.slot] != amg.SLOT_RUNNING:
                    break
            x1 = alone.retire(r.slot)
            alone.close()
            assert state[r.slot] == amg.SLOT_CONVERGED and iters[r.slot] == r.iters
            assert torch.equal(x1, r.x), f"request {q.rid}"
            xs, its, st, _ = h.solve(b, rtol=1e-8, maxit=200)
            assert torch.linalg.norm(xs - r.x) <= 1e-6 * torch.linalg.norm(xs)
        else:
            A = pr.diffusion3d_device(q.m, 1.0, q.seed)
            h = amg.Hierarchy(A, precision=amg.PREC_FP32)
            b = serve.rhs_for(q, h.n)
            xs, its, st, _ = h.solve(b, rtol=1e-8, maxit=200)
            h.close()
            assert st == amg.AMG_OK and its == r.iters
            assert torch.equal(xs, r.x), f"request {q.rid}"
    srv.close()


def test_serve_hbm_admission():
    """With an HBM budget that holds one new operator at a time, set-ups never overlap and every
    request still completes; a request larger than the whole budget is rejected, not queued forever."""
    ops, srv = _small_server(workers=2)
    one = srv.matrix_bytes(16)
    srv.hbm_budget = int(1.5 * one)
    reqs = serve.make_requests(16, rate=4000.0, seed=5, frac_matrix=0.5, n_resident=2, m_range=(16, 16))
    reqs.append(serve.Request(len(reqs), reqs[-1].t_arrival, "matrix", 0, 40, 7))
    res = srv.run(reqs)
    assert srv.stats["max_matrix_inflight"] == 1
    assert srv.stats["rejected"] == 1 and res[-1].status == amg.AMG_ERR_OOM
    assert all(r.status == amg.AMG_OK for r in res[:-1])
    srv.close()
