"""Serving loop (msat_submit / msat_poll): results bit for bit equal to the
same requests run alone, admission under an HBM budget, host-side failure
handling (over-budget and malformed requests, cancellation)."""
import time

import numpy as np
import pytest

from synth import Cnf, serving_stream, uniform_ksat, zipf_weighted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_03640_gb300 as p
    from paper_2402_03640_gb300 import build
    build.build()
    p.load()
    return p


def _alone(pkg, cnf, B, steps, seed, lr, with_step=False):
    with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=seed, lr=lr) as s:
        s.step(steps, want_loss=False, want_cost=False)
        assign, best = s.best()
        bstep = s.best_step()
    return (best, assign, bstep) if with_step else (best, assign)


def _mix(seed=0, count=24):
    reqs = serving_stream(count, rate_per_s=1000.0, seed=seed, n_lo=60, n_hi=3000)
    return [(r, r.instance()) for r in reqs]


@pytest.mark.parametrize("B", [8, 1])
def test_mix_equals_alone(pkg, oracle, B):
    steps, lr = 60, 3e-2
    mix = _mix(seed=B)
    with pkg.Server(restarts=B, chunk=16, lr=lr) as srv:
        tickets = [srv.submit(cnf, steps, seed_x=r.seed) for r, cnf in mix]
        results = [srv.wait(t, 300) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(mix) and st["failed"] == 0
    assert st["peak_running"] > 1  # requests really ran together
    assert st["small_direct"] > 0  # and the small ones took the single-CTA route
    for (r, cnf), res in zip(mix, results):
        best, assign, bstep = _alone(pkg, cnf, B, steps, r.seed, lr, with_step=True)
        assert np.array_equal(res["best_costs"], best), r
        assert np.array_equal(res["assignment"], assign[res["best_restart"]])
        assert res["best_cost"] == best.min() and res["steps"] == steps
        # steps to best of the best restart, as the same request alone reports it
        assert res["best_step"] == bstep[res["best_restart"]]
    # a few against the oracle directly
    for (r, cnf), res in list(zip(mix, results))[:3]:
        ref = oracle.solve(cnf, B, r.seed, steps, mode=oracle.MODE_F32, lr=lr, want_hist=False)
        assert np.array_equal(res["best_costs"], ref["best_cost"])


def test_weighted_and_zero_step_requests(pkg):
    z = zipf_weighted(800, 3000, seed=9)
    with pkg.Server(restarts=4, chunk=7) as srv:
        t0 = srv.submit(z, 0, seed_x=5)
        t1 = srv.submit(z, 23, seed_x=5)
        r0, r1 = srv.wait(t0), srv.wait(t1)
    b0, _ = _alone(pkg, z, 4, 0, 5, 1e-4)
    b1, _ = _alone(pkg, z, 4, 23, 5, 1e-4)
    assert np.array_equal(r0["best_costs"], b0) and np.array_equal(r1["best_costs"], b1)


def test_budget_limits_concurrency(pkg):
    cnfs = [uniform_ksat(2000, 8600, 3, seed=s) for s in range(8)]
    with pkg.Server(restarts=8, hbm_budget=6 << 20, chunk=10) as srv:
        tickets = [srv.submit(c, 40, seed_x=s) for s, c in enumerate(cnfs)]
        res = [srv.wait(t, 300) for t in tickets]
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert 1 <= st["peak_running"] < len(cnfs)
    assert st["hbm_in_use"] <= 6 << 20


def test_work_cap_limits_batch(pkg):
    """batch_mlits bounds the step work of the instances stepped together:
    each request below does 2000 x 8600 x 3 x 8 = 206,400 literal evaluations
    a step, so a cap of 10^6 holds at most 4 of them; a request above the cap
    still runs once nothing else does.  Results stay those of the request
    alone."""
    cnfs = [uniform_ksat(2000, 8600, 3, seed=s) for s in range(8)]
    big = uniform_ksat(20000, 86000, 3, seed=9)  # 2,064,000 a step
    with pkg.Server(restarts=8, chunk=10, batch_mlits=1) as srv:
        tickets = [srv.submit(c, 40, seed_x=s) for s, c in enumerate(cnfs)]
        tb = srv.submit(big, 20, seed_x=3)
        res = [srv.wait(t, 300) for t in tickets]
        rb = srv.wait(tb, 300)
        st = srv.stats()
    assert all(r["status"] == 0 for r in res) and rb["status"] == 0
    assert 1 <= st["peak_running"] <= 4
    for s in (0, 7):
        best, _ = _alone(pkg, cnfs[s], 8, 40, s, 1e-4)
        assert np.array_equal(res[s]["best_costs"], best)
    best, _ = _alone(pkg, big, 8, 20, 3, 1e-4)
    assert np.array_equal(rb["best_costs"], best)
    with pkg.Server(restarts=8, chunk=10, batch_mlits=-1) as srv:  # no cap
        r = srv.wait(srv.submit(cnfs[1], 40, seed_x=1), 300)
    assert np.array_equal(r["best_costs"], res[1]["best_costs"])


def test_over_budget_and_malformed_requests(pkg):
    from paper_2402_03640_gb300 import MsatError, native
    with pkg.Server(restarts=8, hbm_budget=1 << 20) as srv:
        with pytest.raises(MsatError) as e:
            srv.submit(uniform_ksat(20000, 86000, 3, seed=1), 10)
        assert e.value.code == native.MSAT_EBUDGET
        bad = Cnf(n=3, off=np.array([0, 2], np.int64), lits=np.array([1, 4], np.int32))
        with pytest.raises(MsatError) as e:
            srv.submit(bad, 10)
        assert e.value.code == native.MSAT_EINVAL
        assert srv.stats()["submitted"] == 0


def test_cancel_queued_request(pkg):
    from paper_2402_03640_gb300 import MsatError, native
    big = uniform_ksat(4000, 17200, 3, seed=2)
    small = uniform_ksat(100, 430, 3, seed=3)
    with pkg.Server(restarts=8, max_slots=1, chunk=50) as srv:
        t_big = srv.submit(big, 3000)
        t_small = srv.submit(small, 10)
        srv.cancel(t_small)
        with pytest.raises(MsatError) as e:
            srv.cancel(t_big)
        assert e.value.code in (native.MSAT_ESTATE, native.MSAT_EINVAL)
        assert srv.wait(t_big, 300)["status"] == 0
        with pytest.raises(MsatError):
            srv.poll(t_small)
        assert srv.stats()["cancelled"] == 1
