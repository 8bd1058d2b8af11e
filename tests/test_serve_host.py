"""Host-side logic of the serving loop: the request stream and the latency summary."""
import math

import numpy as np
import pytest

from paper_2102_07417_gb300 import problems as pr
from paper_2102_07417_gb300 import serve


def test_request_stream_shape():
    reqs = serve.make_requests(512, rate=200.0, seed=4, frac_matrix=0.3, n_resident=4, m_range=(32, 160))
    assert len(reqs) == 512 and reqs[0].t_arrival == 0.0
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    # exponential gaps with mean 1/200 s: sample mean within 4 standard errors
    assert abs(gaps.mean() - 0.005) < 4 * 0.005 / math.sqrt(len(gaps))
    mats = [r for r in reqs if r.kind == "matrix"]
    frac = len(mats) / len(reqs)
    assert abs(frac - 0.3) < 4 * math.sqrt(0.3 * 0.7 / 512)
    ms = np.array([r.m for r in mats])
    assert ms.min() >= 32 and ms.max() <= 160
    # log-uniform: log m roughly uniform, median near sqrt(32 * 160)
    assert abs(np.median(ms) - math.sqrt(32 * 160)) < 20
    assert {r.target for r in reqs if r.kind == "rhs"} == {0, 1, 2, 3}
    again = serve.make_requests(512, rate=200.0, seed=4)
    assert [(r.t_arrival, r.kind, r.m, r.seed) for r in again] == [(r.t_arrival, r.kind, r.m, r.seed) for r in reqs]


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert serve.percentile(v, 50) == 50 and serve.percentile(v, 99) == 99 and serve.percentile(v, 100) == 100
    assert serve.percentile([3.0], 99) == 3.0


def test_summary():
    R = serve.Result
    res = [R(0, "rhs", 10, 0.0, 0.0, 0.010, 5, 0), R(1, "matrix", 10, 0.005, 0.005, 0.025, 7, 0),
           R(2, "rhs", 10, 0.010, 0.010, 0.014, 5, 0), R(3, "matrix", 10, 0.02, 0.02, 0.02, 0, -3)]
    s = serve.summarize(res)
    assert s["requests"] == 4 and s["ok"] == 3
    assert s["p50_ms"] == pytest.approx(10.0) and s["p99_ms"] == pytest.approx(20.0)
    assert s["rhs"]["count"] == 2 and s["matrix"]["count"] == 1
    assert s["throughput_req_s"] == pytest.approx(3 / 0.025)


def test_device_generator_recipe_on_cpu():
    """The device diffusion generator, run on the CPU: k = 1 (sigma 0) is the 7-point Poisson
    operator exactly, and a random field gives a symmetric positive definite operator."""
    torch = pytest.importorskip("torch")
    A = pr.diffusion3d_device(5, 0.0, 1, device="cpu")
    P = pr.poisson3d(5)
    assert np.array_equal(A.rowptr.numpy(), P.rowptr) and np.array_equal(A.col.numpy(), P.col)
    assert np.array_equal(A.val.numpy(), P.val)
    B = pr.diffusion3d_device(6, 1.0, 9, device="cpu")
    D = pr.CSR(B.n, B.rowptr.numpy(), B.col.numpy(), B.val.numpy()).to_dense()
    assert np.array_equal(D, D.T) and np.linalg.eigvalsh(D).min() > 0
    assert B.val.dtype == torch.float64 and B.col.dtype == torch.int32
