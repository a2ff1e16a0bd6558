"""Host logic of the continuous-batching loop (paper_1608_06345_gb300/serving.py)
against a CPU stand-in of the pool: admission respects the budget, every
request completes, later requests that fit may pass one that does not,
latency accounting, and a request larger than the budget is an error."""
import numpy as np
import pytest

from paper_1608_06345_gb300 import serving


class FakePool:
    """Budget in cells; a bundle advances every resident request by
    bundle_steps; records the peak budget use."""

    def __init__(self, budget_cells, bundle_steps=50, max_instances=8):
        self.budget, self.bundle, self.max_instances = budget_cells, bundle_steps, max_instances
        self.used, self.peak, self.next = 0, 0, 1
        self.res = {}
        self.admit_order = []

    def submit(self, req):
        if self.used + req.cells > self.budget or len(self.res) >= self.max_instances:
            return None
        t = self.next
        self.next += 1
        self.used += req.cells
        self.peak = max(self.peak, self.used)
        self.res[t] = [req, 0]
        self.admit_order.append(req.rid)
        return t

    def run_bundle(self):
        for v in self.res.values():
            v[1] = min(v[0].steps, v[1] + self.bundle)

    def done(self, t):
        req, s = self.res[t]
        return s >= req.steps

    def result(self, t, req):
        del self.res[t]
        self.used -= req.cells
        return "ok", None


def make_requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(rng.integers(8, 64))
        out.append(serving.Request(i, (nx, 4), (1, 0), 1.4, 0.6, 0.6, int(rng.integers(50, 400)), (None, None, None)))
    return out


def test_all_requests_complete_within_budget():
    reqs = make_requests(40)
    arr = np.sort(np.random.default_rng(1).uniform(0, 0.01, len(reqs)))
    pool = FakePool(budget_cells=600)
    recs = serving.serve(reqs, arr, pool, idle_sleep=0)
    assert all(r.status == "ok" for r in recs)
    assert pool.peak <= 600 and pool.used == 0
    for r in recs:
        assert r.admitted >= r.arrival - 1e-9 and r.finished >= r.admitted
    s = serving.summarize(recs)
    assert s["ok"] == 40 and s["solves_per_s"] > 0 and s["p99_ms"] >= s["p50_ms"]


def test_small_request_passes_a_blocked_large_one():
    reqs = [serving.Request(0, (100, 4), (1, 0), 1.4, 0.6, 0.6, 500, (None,) * 3),
            serving.Request(1, (100, 4), (1, 0), 1.4, 0.6, 0.6, 500, (None,) * 3),
            serving.Request(2, (10, 4), (1, 0), 1.4, 0.6, 0.6, 50, (None,) * 3)]
    pool = FakePool(budget_cells=450)
    recs = serving.serve(reqs, np.zeros(3), pool, idle_sleep=0)
    assert pool.admit_order[:2] == [0, 2]  # request 2 fits beside 0; request 1 waits
    assert recs[2].finished < recs[1].finished


def test_request_larger_than_budget_is_an_error():
    reqs = [serving.Request(0, (1000, 4), (1, 0), 1.4, 0.6, 0.6, 10, (None,) * 3)]
    with pytest.raises(RuntimeError):
        serving.serve(reqs, np.zeros(1), FakePool(budget_cells=100), idle_sleep=0)


def test_shock_tube_request_recipe():
    import lbm_inputs as li
    params = li.serving_requests(n=20, seed=6)
    reqs = serving.shock_tube_requests(params)
    for p, r in zip(params, reqs):
        assert 256 <= p["nx"] <= 16384 and 1.1 <= p["gamma"] <= 1.67 and 200 <= p["steps"] <= 2000
        assert 0.52 <= p["tau"] <= 1.0
        rho, u, T = r.fields
        assert rho.size == p["nx"] * 4 and u.shape == (2, p["nx"] * 4)
        # geometric normalisation of the density and pressure ratios
        assert abs(p["left"][0] * p["right"][0] - 1.0) < 1e-12
        assert abs(p["left"][0] * p["left"][2] * p["right"][0] * p["right"][2] - 1.0) < 1e-12


class CountingPool(FakePool):
    """FakePool that fails the test if a request is refused twice with no
    result read in between (a refusal changes nothing, and room only frees
    when results are read, so such a retry is wasted work)."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.generation = 0
        self.refused_at = {}
        self.attempts = 0

    def submit(self, req):
        self.attempts += 1
        t = super().submit(req)
        if t is None:
            assert self.refused_at.get(req.rid) != self.generation, f"request {req.rid} retried with no room freed"
            self.refused_at[req.rid] = self.generation
        return t

    def result(self, t, req):
        self.generation += 1
        return super().result(t, req)


def test_refused_requests_wait_for_freed_room():
    reqs = make_requests(60, seed=4)
    pool = CountingPool(budget_cells=500, bundle_steps=25)
    recs = serving.serve(reqs, np.zeros(len(reqs)), pool, idle_sleep=0)
    assert all(r.status == "ok" for r in recs)
    assert pool.peak <= 500
    # every attempt is either an admission or a refusal in a fresh generation
    assert pool.attempts <= len(reqs) * (pool.generation + 1)


class OverlapPool(FakePool):
    """FakePool whose bundles are launched and waited for separately; a
    bundle advances only the requests resident when it was launched, as the
    GPU pool does with admissions that overlap a running bundle."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.in_flight = None
        self.launches = 0
        self.advanced = {}

    def launch_bundle(self):
        assert self.in_flight is None
        self.in_flight = list(self.res)
        self.launches += 1

    def wait_bundle(self):
        for t in self.in_flight:
            if t in self.res:
                v = self.res[t]
                if v[1] < v[0].steps:
                    self.advanced[t] = self.advanced.get(t, 0) + 1
                v[1] = min(v[0].steps, v[1] + self.bundle)
        self.in_flight = None

    def result(self, t, req):
        # a bundle launched before the admission must not have advanced it
        assert self.advanced.get(t, 0) == -(-req.steps // self.bundle), (req.rid, self.advanced.get(t))
        return super().result(t, req)

    def run_bundle(self):
        raise AssertionError("the loop should launch and wait instead")


def test_admissions_overlap_the_running_bundle():
    reqs = make_requests(50, seed=9)
    arr = np.sort(np.random.default_rng(3).uniform(0, 0.005, len(reqs)))
    pool = OverlapPool(budget_cells=700, bundle_steps=40)
    recs = serving.serve(reqs, arr, pool, idle_sleep=0)
    assert all(r.status == "ok" for r in recs)
    assert pool.peak <= 700
    assert pool.launches >= max(-(-r.steps // 40) for r in reqs)
