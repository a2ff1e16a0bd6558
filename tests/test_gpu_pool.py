"""The continuous-batching pool on the GPU: every instance's result in the
mix equals (bitwise) the same instance run alone through lbm_create, the
admission never exceeds the memory budget, LBM_EBUSY leaves the pool
unchanged, and a non-finite instance is reported without disturbing the
others."""
import numpy as np
import pytest

import lbm_inputs as li
from paper_1608_06345_gb300 import serving

pytestmark = pytest.mark.gpu


def solo_status(req, prec):
    """(status, fields) of the request run alone through lbm_create."""
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0 if len(req.shape) == 2 else 1, req.gamma, req.tau_f, req.tau_g, req.shape, bc=req.bc,
                   prec=prec, rho0=req.rho0, T0=req.T0)
    s.init(*req.fields)
    s.step(req.steps)
    D = len(req.shape)
    rho, u, T = np.zeros(req.cells), np.zeros(D * req.cells), np.zeros(req.cells)
    rc = lbm.load().lbm_moments(s.h, rho.ctypes.data, u.ctypes.data, T.ctypes.data)
    s.close()
    return ("ok" if rc == lbm.LBM_OK else "nonfinite"), (rho, u.reshape(D, -1), T)


def solo(req, prec):
    status, out = solo_status(req, prec)
    assert status == "ok"
    return out


def tube_requests(n, seed):
    params = li.serving_requests(n=n, seed=seed, nx_range=(100, 900), steps_range=(20, 130))
    return serving.shock_tube_requests(params)


@pytest.mark.parametrize("prec", [1, 0, 2])
def test_pool_results_equal_solo_results(prec):
    from paper_1608_06345_gb300 import lbm
    reqs = tube_requests(7, seed=3)
    pool = lbm.Pool(0, prec, budget_bytes=256 << 20, max_instances=16, bundle_steps=16)
    tickets = {}
    for r in reqs:
        t = pool.submit(r.gamma, r.tau_f, r.tau_g, r.shape, r.bc, r.fields, r.steps, rho0=r.rho0, T0=r.T0)
        assert t is not None
        tickets[t] = r
    while tickets:
        pool.run(1)
        pool.sync()
        for t in [t for t in tickets if pool.poll(t)[0]]:
            r = tickets.pop(t)
            rc, got = pool.result(t, r.cells)
            ref = solo(r, prec)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (r.rid, np.max(np.abs(a - b)))
    pool.close()


def test_pool_3d_instance_equals_solo():
    from paper_1608_06345_gb300 import lbm
    fields = li.random_fields(20 * 6 * 5, 3, seed=4)
    req = serving.Request(0, (20, 6, 5), (1, 0, 0), 1.3, 0.7, 0.6, 9, fields)
    other = serving.Request(1, (70, 3, 4), (0, 0, 0), 1.4, 0.6, 0.6, 30, li.random_fields(70 * 12, 3, seed=5))
    pool = lbm.Pool(1, 1, budget_bytes=64 << 20, max_instances=4, bundle_steps=4)
    ta = pool.submit(req.gamma, req.tau_f, req.tau_g, req.shape, req.bc, req.fields, req.steps)
    pool.submit(other.gamma, other.tau_f, other.tau_g, other.shape, other.bc, other.fields, other.steps)
    pool.run(3)
    pool.sync()
    assert pool.poll(ta)[0]
    rc, got = pool.result(ta, req.cells)
    for a, b in zip(got, solo(req, 1)):
        assert np.array_equal(a, b)
    pool.close()


def test_admission_respects_the_budget_and_busy_changes_nothing():
    from paper_1608_06345_gb300 import lbm
    reqs = tube_requests(12, seed=9)
    one = max(r.cells for r in reqs) * 2 * 2 * 37 * 4 + 4096
    budget = 3 * one
    pool = lbm.Pool(0, 1, budget_bytes=budget, max_instances=8, bundle_steps=32)
    admitted, busy = [], 0
    for r in reqs:
        t = pool.submit(r.gamma, r.tau_f, r.tau_g, r.shape, r.bc, r.fields, r.steps, rho0=r.rho0, T0=r.T0)
        st = pool.stats()
        assert st["bytes_used"] <= st["bytes_budget"] <= budget
        if t is None:
            busy += 1
        else:
            admitted.append((t, r))
    assert busy > 0 and len(admitted) >= 3
    before = pool.stats()
    assert pool.submit(reqs[0].gamma, 0.6, 0.6, (100000, 4), (1, 0), li.sod_fields(100000, 4), 10) is None
    assert pool.stats() == before
    # results free memory: everything queued gets in eventually
    done = 0
    while admitted:
        pool.run(1)
        pool.sync()
        for t, r in [(t, r) for t, r in admitted if pool.poll(t)[0]]:
            admitted.remove((t, r))
            rc, _ = pool.result(t, r.cells)
            assert rc == lbm.LBM_OK
            done += 1
    assert pool.stats()["bytes_used"] == 0 and pool.stats()["resident"] == 0
    pool.close()


def test_nonfinite_instance_is_reported_alone():
    from paper_1608_06345_gb300 import lbm
    good = [serving.Request(k, (nx, 4), (1, 0), 1.4, 0.7, 0.7, 40, li.sod_fields(nx, 4, left=(2.0, 0, 1.0),
                                                                                  right=(1.0, 0, 1.0)))
            for k, nx in enumerate((150, 333))]
    rho, u, T = li.uniform_fields(64 * 4, 2)
    rho[10] = np.nan
    bad = serving.Request(99, (64, 4), (0, 0), 1.4, 0.6, 0.6, 20, (rho, u, T))
    pool = lbm.Pool(0, 1, budget_bytes=64 << 20, max_instances=4, bundle_steps=256)
    tb = pool.submit(bad.gamma, 0.6, 0.6, bad.shape, bad.bc, bad.fields, bad.steps)
    tg = [(pool.submit(r.gamma, r.tau_f, r.tau_g, r.shape, r.bc, r.fields, r.steps, rho0=r.rho0, T0=r.T0), r)
          for r in good]
    pool.run(1)
    pool.sync()
    rc, _ = pool.result(tb, bad.cells)
    assert rc == lbm.LBM_ENONFINITE
    for t, r in tg:
        rc, got = pool.result(t, r.cells)
        assert rc == lbm.LBM_OK
        for a, b in zip(got, solo(r, 1)):
            assert np.array_equal(a, b)
    pool.close()


def test_serving_loop_with_poisson_arrivals():
    """End to end: Poisson arrivals through serving.serve on the GPU pool;
    every result equals the solo result."""
    from paper_1608_06345_gb300 import lbm
    reqs = tube_requests(10, seed=21)
    arr = li.poisson_arrivals(len(reqs), rate=400.0, seed=2)
    pool = lbm.Pool(0, 1, budget_bytes=32 << 20, max_instances=6, bundle_steps=32)
    recs = serving.serve(reqs, arr, serving.PoolBackend(pool), keep_results=True)
    pool.close()
    # the recipe's extreme draws (tau near 0.52, large ratios) can go
    # non-finite; each request must behave exactly as it does alone
    for rec, req in zip(recs, reqs):
        status, ref = solo_status(req, 1)
        assert rec.status == status
        if status == "ok":
            for a, b in zip(rec.result, ref):
                assert np.array_equal(a, b)
    s = serving.summarize(recs)
    assert s["ok"] >= 1 and s["ok"] + s["nonfinite"] == len(reqs) and s["p99_ms"] > 0


@pytest.mark.parametrize("prec", [1, 2])
def test_admission_during_a_running_bundle(prec):
    """Requests admitted while a bundle is on the GPU (pool.run without a
    sync, then submit) are initialised on the admission stream and join at
    the next bundle; every result still equals the instance run alone,
    bitwise, including the instances the running bundle was advancing and
    one that reuses the memory and slot of a retired instance."""
    from paper_1608_06345_gb300 import lbm
    reqs = tube_requests(6, seed=11)
    pool = lbm.Pool(0, prec, budget_bytes=256 << 20, max_instances=3, bundle_steps=8)
    tickets = {}
    waiting = list(reqs)
    for r in waiting[:2]:
        tickets[pool.submit(r.gamma, r.tau_f, r.tau_g, r.shape, r.bc, r.fields, r.steps, rho0=r.rho0, T0=r.T0)] = r
    waiting = waiting[2:]
    checked = 0
    while tickets or waiting:
        pool.run(1)  # in flight while the next admissions are made
        while waiting:
            r = waiting[0]
            t = pool.submit(r.gamma, r.tau_f, r.tau_g, r.shape, r.bc, r.fields, r.steps, rho0=r.rho0, T0=r.T0)
            if t is None:
                break
            tickets[t] = r
            waiting.pop(0)
        pool.sync()
        for t in [t for t in tickets if pool.poll(t)[0]]:
            r = tickets.pop(t)
            rc, got = pool.result(t, r.cells)
            status, ref = solo_status(r, prec)  # this stream holds a tube that diverges in the scheme itself
            assert status == ("ok" if rc == lbm.LBM_OK else "nonfinite"), r.rid
            if status == "ok":
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b), (r.rid, np.max(np.abs(a - b)))
            checked += 1
    assert checked == len(reqs)
    pool.close()
