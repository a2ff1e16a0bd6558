"""Continuous-batching request loop over the library's pool (lbm_pool_* C ABI).

Requests (shock tubes or periodic boxes of uneven size, gamma, tau, steps)
arrive over time.  The loop admits arrived requests into the pool while its
memory budget and slots allow (in arrival order, letting later requests that
fit pass one that does not), advances everything resident by one step bundle
per iteration (one batched launch per time step, inside one CUDA graph), and
reads back the finished instances, which frees their memory for the queue.
Latency = completion time - arrival time.

The baseline is the plain method: one FP64 instance per request, one kernel
launch per time step, requests served one after another in arrival order.

All scheduling decisions are host logic over a small backend interface, so
the same loop runs against the GPU pool or against a CPU stand-in in tests.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    shape: tuple
    bc: tuple
    gamma: float
    tau_f: float
    tau_g: float
    steps: int
    fields: tuple           # (rho, u, T) host arrays
    rho0: float = 0.0       # reference state of the deviation storage (0: the precision's default)
    T0: float = 0.0

    @property
    def cells(self):
        return int(np.prod(self.shape))


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    status: str = "pending"
    result: tuple = field(default=None, repr=False)

    @property
    def latency(self):
        return self.finished - self.arrival


class PoolBackend:
    """Backend of the loop on the GPU pool (paper_1608_06345_gb300.lbm.Pool).

    It mirrors the pool's byte accounting (an admission takes
    lbm_pool_instance_bytes, reading its result gives them back) and refuses
    a request larger than the free total without calling the library: no
    layout of the arena could hold it, so the pool would refuse it too."""

    def __init__(self, pool):
        self.pool = pool
        st = pool.stats()
        self.used, self.arena = int(st["bytes_used"]), int(st["bytes_budget"])
        self._bytes = {}

    def _need(self, req):
        b = self._bytes.get(req.rid)
        if b is None:
            b = self._bytes[req.rid] = int(self.pool.instance_bytes(req.shape))
        return b

    def submit(self, req):
        need = self._need(req)
        if self.used + need > self.arena:
            return None
        t = self.pool.submit(req.gamma, req.tau_f, req.tau_g, req.shape, req.bc, req.fields, req.steps,
                             rho0=req.rho0, T0=req.T0)
        if t is not None:
            self.used += need
        return t

    def launch_bundle(self):
        self.pool.run(1)

    def wait_bundle(self):
        self.pool.sync()

    def run_bundle(self):
        self.launch_bundle()
        self.wait_bundle()

    def done(self, ticket):
        return self.pool.poll(ticket)[0]

    def result(self, ticket, req):
        from . import lbm
        rc, fields = self.pool.result(ticket, req.cells)
        self.used -= self._need(req)
        return ("ok" if rc == lbm.LBM_OK else "nonfinite"), fields


def serve(requests, arrivals, backend, clock=time.perf_counter, keep_results=False, idle_sleep=1e-4):
    """Run the continuous-batching loop.  `arrivals[i]` is request i's arrival
    time in seconds from the start.  Returns one Record per request.

    Each iteration launches a step bundle for everything resident, admits
    arrived requests while it runs (backend.launch_bundle / wait_bundle; a
    backend with only run_bundle admits between bundles instead), waits for
    it and reads back the finished instances."""
    order = np.argsort(arrivals, kind="stable")
    pending = deque((float(arrivals[i]), requests[i]) for i in order)
    records = {r.rid: Record(r.rid, float(a)) for r, a in zip(requests, arrivals)}
    overlap = hasattr(backend, "launch_bundle") and hasattr(backend, "wait_bundle")
    # queue: refused since room last freed up; fresh: arrived, not yet tried.
    # A refused submission changes nothing and room frees only when results
    # are read, so queued requests are retried only after that.
    queue = deque()
    fresh = deque()
    freed = False
    active = {}
    t0 = clock()

    def admit():
        nonlocal queue, fresh, freed
        now = clock() - t0
        while pending and pending[0][0] <= now:
            fresh.append(pending.popleft()[1])
        # arrival order; later requests may pass one that does not fit yet
        candidates = (queue + fresh) if freed else fresh
        still = deque()
        for req in candidates:
            ticket = backend.submit(req)
            if ticket is None:
                still.append(req)
            else:
                active[ticket] = req
                records[req.rid].admitted = clock() - t0
        queue = still if freed else queue + still
        fresh = deque()
        freed = False

    while pending or queue or fresh or active:
        running = bool(active)
        if running and overlap:
            backend.launch_bundle()  # the bundle advances what was resident before this iteration's admissions
            admit()
            backend.wait_bundle()
        else:
            admit()
            if running:
                backend.run_bundle()
        if running:
            finished = [t for t in active if backend.done(t)]
            for t in finished:
                req = active.pop(t)
                status, res = backend.result(t, req)
                rec = records[req.rid]
                rec.finished = clock() - t0
                rec.status = status
                if keep_results:
                    rec.result = res
            freed = freed or bool(finished)
        elif active:
            continue  # first admissions: step them next iteration
        elif pending and not queue:
            wait = pending[0][0] - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, idle_sleep) if idle_sleep else 0)
        elif queue:
            raise RuntimeError(f"request {queue[0].rid} can never be admitted (larger than the pool budget?)")
    return [records[r.rid] for r in requests]


def serve_baseline(requests, arrivals, make_solver, clock=time.perf_counter, keep_results=False):
    """One instance per request, one launch per time step, FIFO.  make_solver(req)
    returns an object with init(rho, u, T), step(n), moments()."""
    order = np.argsort(arrivals, kind="stable")
    records = {r.rid: Record(r.rid, float(a)) for r, a in zip(requests, arrivals)}
    t0 = clock()
    for i in order:
        req = requests[i]
        wait = float(arrivals[i]) - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        rec = records[req.rid]
        rec.admitted = clock() - t0
        s = make_solver(req)
        s.init(*req.fields)
        s.step(req.steps)
        try:
            res = s.moments()
            rec.status = "ok"
        except Exception as ex:  # non-finite state
            res = None
            rec.status = "nonfinite" if "NONFINITE" in str(ex) else "error"
        rec.finished = clock() - t0
        if keep_results:
            rec.result = res
        s.close()
    return [records[r.rid] for r in requests]


def summarize(records, makespan=None):
    """Solves/s and latency percentiles over the finished, finite requests."""
    ok = [r for r in records if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) if ok else np.array([np.nan])
    if makespan is None:
        makespan = max((r.finished for r in records if np.isfinite(r.finished)), default=float("nan"))
    return {
        "solves": len(records), "ok": len(ok), "nonfinite": sum(r.status == "nonfinite" for r in records),
        "makespan_s": makespan, "solves_per_s": len(ok) / makespan if makespan and makespan > 0 else float("nan"),
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(np.mean(lat) * 1e3),
    }


def shock_tube_requests(params, ny=4):
    """Requests for lbm_inputs.serving_requests(...) parameter dicts: shock
    tubes with zero-gradient x ends, periodic y, the reference state of the
    deviation storage at the volume-averaged density and pressure."""
    import lbm_inputs as li
    out = []
    for p in params:
        nx = p["nx"]
        fields = li.sod_fields(nx, ny, left=p["left"], right=p["right"])
        rho0 = 0.5 * (p["left"][0] + p["right"][0])
        T0 = 0.5 * (p["left"][0] * p["left"][2] + p["right"][0] * p["right"][2]) / rho0
        out.append(Request(p["id"], (nx, ny), (1, 0), p["gamma"], p["tau"], p["tau"], p["steps"], fields,
                           rho0=rho0, T0=T0))
    return out
