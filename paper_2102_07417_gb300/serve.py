"""Serving AMG-PCG solves with continuous batching.

A request loop keeps several hierarchies resident on the GPU and serves a
stream of two kinds of request:

* ``rhs``: a new right-hand side for one of the resident operators.  It is
  admitted into a free column ("slot") of that operator's running PCG batch
  (``amg.Slots``) at the next iteration boundary, shares every SpMM and
  V-cycle with the requests already there, and leaves the batch as soon as
  its own stopping test ``||r_j|| < rtol ||b_j||`` holds.
* ``matrix``: a new operator (fresh coefficients) that needs set-up and
  solve.  These run on worker threads, each with its own CUDA stream, and are
  admitted only when the HBM they are expected to need is free.

Every resident operator has its own stream and keeps up to ``depth`` PCG
steps (replayed CUDA graphs) in flight; the loop reads each step's per-slot
state from a pinned snapshot without waiting, so the steps of different
operators overlap on the device and the host never stalls the GPU between
steps.  Latency is measured from a request's arrival time to the moment the
host sees its column converged (its solution is then final in device
memory; a converged column is frozen).
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import amg
from . import problems as pr


@dataclass
class Request:
    rid: int
    t_arrival: float  # seconds after the start of the stream
    kind: str  # "rhs" | "matrix"
    target: int  # resident operator index (rhs)
    m: int  # grid size of a new operator (matrix): n = m^3
    seed: int  # right-hand side / coefficient seed


@dataclass
class Result:
    rid: int
    kind: str
    n: int
    t_arrival: float
    t_start: float
    t_done: float
    iters: int
    status: int
    slot: int = -1
    capacity: int = 0  # width of the batch the request ran in (rhs)
    x: object = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def make_requests(count: int = 512, rate: float = 200.0, seed: int = 4, frac_matrix: float = 0.3,
                  n_resident: int = 4, m_range=(32, 160), seed_base: int = 1000) -> list[Request]:
    """Poisson arrivals at ``rate`` req/s; each request is a new matrix with probability
    ``frac_matrix`` (grid size m = round(exp(U[ln lo, ln hi]))), else a new right-hand side for a
    resident operator drawn uniformly.  ``seed`` drives the arrivals and choices; request r
    draws its coefficients / right-hand side from seed ``seed_base + r``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]  # the first request arrives at t = 0
    is_mat = rng.random(count) < frac_matrix
    target = rng.integers(0, n_resident, size=count)
    lo, hi = math.log(m_range[0]), math.log(m_range[1])
    m = np.rint(np.exp(rng.uniform(lo, hi, size=count))).astype(int)
    return [Request(i, float(t[i]), "matrix" if is_mat[i] else "rhs", int(target[i]), int(m[i]), seed_base + i)
            for i in range(count)]


def percentile(v, q: float) -> float:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sequence."""
    s = sorted(v)
    k = max(1, math.ceil(q / 100.0 * len(s)))
    return float(s[k - 1])


def summarize(results: list[Result]) -> dict:
    lat = [r.latency for r in results if r.status == amg.AMG_OK]
    out = {"requests": len(results), "ok": len(lat)}
    if lat:
        t0 = min(r.t_arrival for r in results)
        t1 = max(r.t_done for r in results)
        out.update({"p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
                    "mean_ms": 1e3 * float(np.mean(lat)), "makespan_s": t1 - t0,
                    "throughput_req_s": len(lat) / (t1 - t0) if t1 > t0 else float("nan")})
        for kind in ("rhs", "matrix"):
            lk = [r.latency for r in results if r.kind == kind and r.status == amg.AMG_OK]
            if lk:
                out[kind] = {"count": len(lk), "p50_ms": 1e3 * percentile(lk, 50), "p99_ms": 1e3 * percentile(lk, 99)}
    return out


def rhs_for(req: Request, n: int, device="cuda"):
    """The request's right-hand side, b ~ U[-1, 1] from its seed (generated on the device)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(req.seed)
    return torch.rand(n, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0


class _Group:
    """One continuous-batching block on a resident operator: its slots object, free slots and
    running requests (slot -> (request, start time))."""

    def __init__(self, op: int, sl, capacity: int):
        self.op, self.sl, self.capacity = op, sl, capacity
        self.free = list(range(capacity))
        self.running = {}


class Server:
    """Resident hierarchies + continuous batching + HBM-gated set-up of new operators.

    Each resident operator has a batch group of ``capacity`` columns and (``solo``) a one-column
    group: a step costs about a + b k for k columns, so a request that finds the operator idle
    runs alone (cheapest step), and requests that overlap share the batch group's steps."""

    def __init__(self, operators, precision: int = amg.PREC_FP32, capacity: int = 4, rtol: float = 1e-8,
                 maxit: int = 200, workers: int = 8, sigma: float = 1.0, hbm_budget: int | None = None,
                 hbm_reserve: int = 2 << 30, keep_x: bool = False, depth: int = 2, solo: bool = True):
        import torch

        self.torch = torch
        self.precision, self.capacity, self.rtol, self.maxit = precision, capacity, rtol, maxit
        self.sigma, self.keep_x = sigma, keep_x
        self.hier, self.slots, self.n = [], [], []
        # per operator: [solo group (one column), batch group (capacity columns)] or [batch group]
        self.groups = []
        for i, A in enumerate(operators):
            st = torch.cuda.Stream()
            h = amg.Hierarchy(A, stream=st, precision=precision)  # waits for A's producers
            self.hier.append(h)
            self.n.append(h.n)
            gs = []
            if solo and capacity > 1:
                gs.append(_Group(i, h.slots(1, rtol=rtol, maxit=maxit, stream=torch.cuda.Stream()), 1))
            gs.append(_Group(i, h.slots(capacity, rtol=rtol, maxit=maxit, stream=st), capacity))
            self.groups.append(gs)
            self.slots.extend(g.sl for g in gs)
        # bytes of hierarchy per unknown, from the resident operators (set-up estimate: x3 for
        # the temporaries of the Galerkin products and the solve vectors)
        self.bytes_per_row = max(h.nbytes() / h.n for h in self.hier) * 3.0
        self.workers = workers
        self.hbm_budget = hbm_budget
        self.hbm_reserve = hbm_reserve
        self.depth = depth
        self._x_scratch = [None] * len(self.hier)
        # set-up streams run at high priority: a set-up is a chain of small, latency-bound kernels
        # (and host round trips) that would otherwise queue behind the resident operators' steps
        self._streams = [torch.cuda.Stream(priority=-1) for _ in range(workers)]
        self._free_streams = collections.deque(range(workers))
        self._lock = threading.Lock()
        self.stats = {"max_running_slots": 0, "max_matrix_inflight": 0, "steps": 0, "rejected": 0}

    def close(self):
        for s in self.slots:
            s.close()
        for h in self.hier:
            h.close()

    def _scratch(self, i: int):
        """A device buffer the solution of operator i is copied to when results are not kept."""
        if self._x_scratch[i] is None:
            self._x_scratch[i] = self.torch.empty(self.n[i], dtype=self.torch.float64, device="cuda")
        return self._x_scratch[i]

    # -- new operators (worker threads) --------------------------------------
    def matrix_bytes(self, m: int) -> int:
        return int(self.bytes_per_row * m ** 3)

    def _hbm_ok(self, need: int, inflight_bytes: int) -> bool:
        if self.hbm_budget is not None:
            return inflight_bytes + need <= self.hbm_budget
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return need + inflight_bytes + self.hbm_reserve <= free + cached

    def _solve_matrix(self, req: Request, t0: float, clock):
        torch = self.torch
        with self._lock:
            si = self._free_streams.popleft()
        st = self._streams[si]
        t_start = clock() - t0
        try:
            with torch.cuda.stream(st):
                A = pr.diffusion3d_device(req.m, self.sigma, req.seed, stream=st)
                # the library's own stream-ordered allocator: no Python callback (and no GIL) per
                # allocation inside the set-up
                h = amg.Hierarchy(A, stream=st, precision=self.precision, torch_allocator=False)
                b = rhs_for(req, h.n)
                x, it, status, _ = h.solve(b, rtol=self.rtol, maxit=self.maxit, stream=st)
                st.synchronize()
                h.close()
            return Result(req.rid, "matrix", req.m ** 3, req.t_arrival, t_start, clock() - t0, it, status,
                          x=x if self.keep_x else None)
        finally:
            with self._lock:
                self._free_streams.append(si)

    # -- the loop ------------------------------------------------------------
    def run(self, requests: list[Request], clock=time.perf_counter) -> list[Result]:
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        rhs_q = [collections.deque() for _ in self.hier]
        mat_q = collections.deque()
        results: list[Result] = []
        inflight = {}  # future -> (request, bytes)
        pool = ThreadPoolExecutor(max_workers=self.workers)
        nxt = 0
        t0 = clock()
        try:
            while len(results) < len(reqs):
                now = clock() - t0
                while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
                    r = reqs[nxt]
                    nxt += 1
                    if r.kind == "rhs":
                        rhs_q[r.target].append(r)
                    else:
                        mat_q.append(r)
                # new operators: admitted by HBM, at most `workers` at a time
                inflight_bytes = sum(v[1] for v in inflight.values())
                while mat_q and len(inflight) < self.workers:
                    r = mat_q[0]
                    need = self.matrix_bytes(r.m)
                    cap = self.hbm_budget if self.hbm_budget is not None else None
                    if cap is not None and need > cap:
                        mat_q.popleft()
                        self.stats["rejected"] += 1
                        results.append(Result(r.rid, "matrix", r.m ** 3, r.t_arrival, now, clock() - t0, 0,
                                              amg.AMG_ERR_OOM))
                        continue
                    if not self._hbm_ok(need, inflight_bytes):
                        break
                    mat_q.popleft()
                    inflight[pool.submit(self._solve_matrix, r, t0, clock)] = (r, need)
                    inflight_bytes += need
                self.stats["max_matrix_inflight"] = max(self.stats["max_matrix_inflight"], len(inflight))
                for f in [f for f in inflight if f.done()]:
                    inflight.pop(f)
                    results.append(f.result())
                # right-hand sides: admitted into free slots at the iteration boundary
                for i, gs in enumerate(self.groups):
                    batch = gs[-1]
                    while rhs_q[i]:
                        g = batch
                        if len(gs) > 1 and not batch.running and gs[0].free:
                            g = gs[0]  # the operator is idle: run alone
                        if not g.free:
                            break
                        r = rhs_q[i].popleft()
                        s_ = g.free.pop(0)
                        with torch.cuda.stream(g.sl.tstream):
                            b = rhs_for(r, self.n[i])
                            g.sl.admit(s_, b)
                        g.running[s_] = (r, clock() - t0)
                active = [g for gs in self.groups for g in gs if g.running]
                self.stats["max_running_slots"] = max(self.stats["max_running_slots"],
                                                      sum(len(g.running) for g in active))
                # steps stay `depth` deep in flight on every group; results are read from the
                # snapshots of finished steps without waiting (a converged column is frozen, so
                # the steps behind it leave its solution unchanged)
                progressed = False
                blocked = []
                for g in active:
                    sl, i = g.sl, g.op
                    state, iters, done, issued = sl.query()
                    for s_ in list(g.running):
                        if state[s_] == amg.SLOT_RUNNING:
                            continue
                        r, t_start = g.running.pop(s_)
                        t_done = clock() - t0
                        with torch.cuda.stream(sl.tstream):
                            x = sl.retire(s_) if self.keep_x else sl.retire(s_, self._scratch(i))
                        st = amg.AMG_OK if state[s_] == amg.SLOT_CONVERGED else int(state[s_])
                        results.append(Result(r.rid, "rhs", self.n[i], r.t_arrival, t_start, t_done,
                                              int(iters[s_]), st, slot=s_, capacity=g.capacity,
                                              x=x if self.keep_x else None))
                        g.free.append(s_)
                        g.free.sort()
                        progressed = True
                    if g.running and issued - done < self.depth:
                        sl.step()
                        self.stats["steps"] += 1
                        progressed = True
                    elif g.running:
                        blocked.append(g)
                if not active:
                    # idle: wait for the next arrival or a finishing set-up
                    wait = 0.0005
                    if nxt < len(reqs) and not inflight and not mat_q:
                        wait = max(0.0, reqs[nxt].t_arrival - (clock() - t0))
                    time.sleep(min(wait, 0.002))
                elif not progressed and blocked:
                    blocked[0].sl.wait()
        finally:
            pool.shutdown(wait=True)
            for sl in self.slots:
                sl.tstream.synchronize()
        return sorted(results, key=lambda r: r.rid)


def resident_operators(sizes=(48, 96, 128, 160), sigma: float = 1.0, seed0: int = 40):
    """The resident operators of the serving workload (device-generated diffusion, seeds seed0 + i)."""
    return [pr.diffusion3d_device(m, sigma, seed0 + i) for i, m in enumerate(sizes)]
