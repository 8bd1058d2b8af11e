"""Continuous batching (amg_slots_*): requests join and leave a running PCG batch.

Bar: a request admitted into slot s at any step, beside any mix of other
requests, gives the same iteration count and the same x (value equality) as
column s of a one-shot amg_pcg_solve_batch of the same width.  Per column the
two run the same arithmetic in the same order (the first step of an admitted
column only forms z = M b and p = z, as the batch's initialisation does), and
no column's sums involve another column, so the match is exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2102_07417_gb300 import amg  # noqa: E402
from paper_2102_07417_gb300 import problems as pr  # noqa: E402

DEV = "cuda:0"


def _rhs(n, count, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, n) for _ in range(count)]


def _run_schedule(hg, cap, bs, arrivals, rtol, maxit=500, pipelined=False):
    """Admit bs[r] at step arrivals[r] (into the lowest free slot, queueing when full);
    retire converged slots after every step (pipelined: read the state of finished steps
    without waiting, two steps in flight).  Returns {r: (slot, iters, state, x)}."""
    sl = hg.slots(cap, rtol=rtol, maxit=maxit)
    free = list(range(cap))
    queue, running, out = [], {}, {}
    bdev = [torch.as_tensor(b, device=DEV) for b in bs]
    step = 0
    while len(out) < len(bs):
        queue += [r for r in range(len(bs)) if arrivals[r] == step]
        while queue and free:
            r = queue.pop(0)
            s = free.pop(0)
            sl.admit(s, bdev[r])
            running[s] = r
        if pipelined:
            sl.step()
            state, iters, done, issued = sl.query()
            if issued - done >= 2:
                sl.wait()
        else:
            sl.step()
            state, iters = sl.poll()
        for s in list(running):
            if state[s] != amg.SLOT_RUNNING:
                r = running.pop(s)
                out[r] = (s, int(iters[s]), int(state[s]), sl.retire(s).clone())
                free.append(s)
                free.sort()
        step += 1
        assert step < 10 * maxit
    torch.cuda.synchronize()
    sl.close()
    return out


@pytest.mark.parametrize("prec,pipelined,cap,N", [(amg.PREC_FP64, False, 4, 20), (amg.PREC_FP32, False, 4, 20),
                                                   (amg.PREC_FP32, True, 4, 20), (amg.PREC_FP32, True, 8, 34)])
def test_slots_match_batch_columns(prec, pipelined, cap, N):
    """(8 columns on 39,304 rows: the sliced-ELLPACK kernels and the double-float outer product.)"""
    A, _ = pr.diffusion3d(N, 1.0, 7)
    hg = amg.Hierarchy(A, seed=0, precision=prec)
    bs = _rhs(A.n, 9, 11)
    arrivals = [0, 0, 2, 3, 3, 3, 7, 12, 12]
    out = _run_schedule(hg, cap, bs, arrivals, 1e-8, pipelined=pipelined)
    for r, (s, it, state, x) in out.items():
        assert state == amg.SLOT_CONVERGED
        B = np.repeat(bs[r][:, None], cap, axis=1)
        X, iters, stats, st, _ = hg.solve_batch(torch.as_tensor(B, device=DEV), rtol=1e-8)
        assert iters[s] == it, f"request {r} in slot {s}"
        assert torch.equal(X[:, s].contiguous(), x), f"request {r} in slot {s}"
        res = np.linalg.norm(bs[r] - A.matvec(x.cpu().numpy()))
        assert res < 1e-7 * np.linalg.norm(bs[r])


def test_slots_zero_rhs_free_and_maxit():
    A = pr.poisson2d(48)
    hg = amg.Hierarchy(A, seed=0)
    sl = hg.slots(3, rtol=1e-12, maxit=2)
    state, iters = sl.poll()
    assert list(state) == [0, 0, 0]
    b = torch.as_tensor(_rhs(A.n, 1, 3)[0], device=DEV)
    sl.admit(0, torch.zeros(A.n, dtype=torch.float64, device=DEV))
    sl.admit(2, b)
    for _ in range(3):
        sl.step()
    state, iters = sl.poll()
    assert state[0] == amg.SLOT_CONVERGED and iters[0] == 0
    assert state[1] == 0
    assert state[2] == amg.AMG_ERR_NO_CONVERGENCE and iters[2] == 2
    assert torch.count_nonzero(sl.retire(0)) == 0
    x2 = sl.retire(2)
    assert torch.isfinite(x2).all()
    state, _ = sl.poll()
    assert list(state) == [0, 0, 0]
    sl.close()


def test_slots_bad_arguments():
    A = pr.poisson2d(32)
    hg = amg.Hierarchy(A, seed=0)
    lib = amg.load()
    import ctypes as C

    h = C.c_void_p()
    assert lib.amg_slots_create(hg.h, 0, 1e-8, 10, None, C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_slots_create(hg.h, 33, 1e-8, 10, None, C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_slots_create(hg.h, 2, 0.0, 10, None, C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    sl = hg.slots(2)
    b = torch.ones(A.n, dtype=torch.float64, device=DEV)
    assert lib.amg_slots_admit(sl.s, 2, b.data_ptr()) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_slots_admit(sl.s, -1, b.data_ptr()) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_slots_retire(sl.s, 5, None) == amg.AMG_ERR_INVALID_ARG
    sl.close()
