"""The serving loop's policy on the host (qmcdu_server_* with `simulate`: no
GPU work, a cost model on a virtual clock): admission against the device-memory
budget, eviction of idle pools, continuous batching, the recompute cadence,
first-come order within a class, the plain one-walker-at-a-time configuration,
and argument checks. Runs without a GPU."""
import math

import numpy as np
import pytest

from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import QmcduError, Server, qmcdu_footprint

SIZES = (128, 256, 512)


def _server(**kw):
    classes = kw.pop("classes", [dict(N=n, slots=4) for n in SIZES])
    kw.setdefault("simulate", True)
    kw.setdefault("hbm_budget", 10**10)
    return Server(classes, **kw)


def _run(srv, reqs):
    srv.submit(reqs)
    srv.run()
    res = {r["id"]: r for r in srv.results()}
    st = srv.stats()
    return res, st


def _pool_bytes(N, slots, precision="fp32", K=32):
    return qmcdu_footprint(N, min(N, K), precision, slots) + slots * N + slots * 24


def test_every_request_runs_its_sweeps_and_recomputes():
    reqs = inputs.serving_trace(3, rate_hz=400.0, duration_s=0.2, sizes=SIZES, nsweeps=7)
    srv = _server(recompute_every=3)
    res, st = _run(srv, reqs)
    assert len(res) == len(reqs) and st["finished"] == len(reqs) and st["failed"] == 0
    for q in reqs:
        r = res[q["id"]]
        assert r["status"] == 0
        assert r["accepted"] == 7 * q["N"]                  # the cost model accepts every move
        # recomputes before sweeps 3 and 6, and the final one
        assert r["recomputes"] == len([s for s in range(1, 7) if s % 3 == 0]) + 1
        assert r["arrival_s"] <= r["admit_s"] <= r["done_s"]
    assert st["walker_sweeps"] == 7 * len(reqs)
    assert st["proposals"] == sum(7 * q["N"] for q in reqs)
    srv.close()


def test_budget_is_never_exceeded_and_idle_pools_are_evicted():
    # room for the pool of one class but not both: classes alternate, so the
    # idle pool of one class must be destroyed to admit the other
    b512, b256 = _pool_bytes(512, 2), _pool_bytes(256, 2)
    budget = b512 + b256 // 2
    classes = [dict(N=256, slots=2), dict(N=512, slots=2)]
    reqs = [dict(id=i, seed=100 + i, N=(256, 512)[(i // 6) % 2], nsweeps=2, arrival_s=0.05 * i)
            for i in range(24)]
    srv = _server(classes=classes, hbm_budget=budget)
    res, st = _run(srv, reqs)
    assert st["finished"] == len(reqs)
    assert st["peak_bytes"] <= budget
    assert st["pools_destroyed"] > 0
    srv.close()


def test_request_that_can_never_fit_fails_with_oom():
    classes = [dict(N=128, slots=2), dict(N=2048, slots=4)]
    budget = _pool_bytes(128, 2) * 3
    assert _pool_bytes(2048, 4) > budget
    reqs = [dict(id=0, seed=1, N=2048, nsweeps=1, arrival_s=0.0),
            dict(id=1, seed=2, N=128, nsweeps=2, arrival_s=0.0)]
    srv = _server(classes=classes, hbm_budget=budget)
    res, st = _run(srv, reqs)
    assert res[0]["status"] == 4 and res[1]["status"] == 0
    assert st["failed"] == 1 and st["finished"] == 1
    srv.close()


def test_walkers_join_running_pools_between_rounds():
    # arrivals every 0.5 ms while a sweep of N=512 takes several ms: later
    # walkers enter pools whose earlier walkers are mid-run
    reqs = [dict(id=i, seed=7 + i, N=512, nsweeps=6, arrival_s=0.0005 * i) for i in range(8)]
    srv = _server(classes=[dict(N=512, slots=8)])
    res, st = _run(srv, reqs)
    assert st["mixed_walker_sweeps"] > 0
    assert st["pools_created"] == 1
    by_pool = {}
    for r in res.values():
        by_pool.setdefault(r["pool"], []).append(r)
    joined = False
    for rs in by_pool.values():
        for a in rs:
            for b in rs:
                # b was admitted while a was running and ran alongside it
                if a["admit_s"] < b["admit_s"] < a["done_s"] and \
                        b["first_round"] <= a["last_round"]:
                    joined = True
    assert joined
    srv.close()


def test_first_come_first_served_within_a_class():
    reqs = [dict(id=i, seed=50 + i, N=256, nsweeps=2, arrival_s=0.001 * i) for i in range(10)]
    srv = _server(classes=[dict(N=256, slots=2)], max_walkers=2)
    res, st = _run(srv, reqs)
    order = sorted(res.values(), key=lambda r: r["admit_s"])
    assert [r["id"] for r in order] == sorted(res)            # admitted in arrival order
    assert st["max_resident"] <= 2
    srv.close()


def test_plain_one_walker_at_a_time():
    reqs = inputs.serving_trace(5, rate_hz=300.0, duration_s=0.1, sizes=SIZES, nsweeps=3)
    classes = [dict(N=n, slots=1) for n in SIZES]
    srv = _server(classes=classes, max_walkers=1, max_inflight=1, precision="fp64")
    res, st = _run(srv, reqs)
    assert st["finished"] == len(reqs)
    assert st["max_resident"] == 1 and st["max_inflight"] == 1
    assert st["mixed_walker_sweeps"] == 0
    # one request at a time, in order of arrival
    done = sorted(res.values(), key=lambda r: r["done_s"])
    for a, b in zip(done, done[1:]):
        assert a["done_s"] <= b["admit_s"]
    srv.close()


def test_batching_beats_one_walker_at_a_time_on_the_cost_model():
    reqs = inputs.serving_trace(9, rate_hz=2000.0, duration_s=0.05, sizes=SIZES, nsweeps=4)
    srv = _server()
    _, st_b = _run(srv, reqs)
    srv.close()
    srv = _server(classes=[dict(N=n, slots=1) for n in SIZES], max_walkers=1, max_inflight=1)
    _, st_p = _run(srv, reqs)
    srv.close()
    assert st_b["last_round_end_s"] < st_p["last_round_end_s"]
    assert st_b["request_s_p50"] < st_p["request_s_p50"]


def test_latency_statistics_are_ordered():
    reqs = inputs.serving_trace(11, rate_hz=500.0, duration_s=0.1, sizes=SIZES, nsweeps=5)
    srv = _server()
    _, st = _run(srv, reqs)
    assert 0 < st["sweep_ms_p50"] <= st["sweep_ms_p99"]
    assert 0 < st["request_s_p50"] <= st["request_s_p99"]
    assert 0 <= st["wait_s_p50"] <= st["wait_s_p99"]
    srv.close()


def test_run_until_stops_the_clock_and_resumes():
    reqs = [dict(id=i, seed=i, N=128, nsweeps=10, arrival_s=0.01 * i) for i in range(5)]
    srv = _server()
    srv.submit(reqs)
    srv.run(until_s=0.015)
    st = srv.stats()
    assert st["clock_s"] >= 0.015 and st["finished"] < 5
    srv.run()
    assert srv.stats()["finished"] == 5
    srv.close()


def test_argument_checks():
    with pytest.raises(QmcduError):
        Server([dict(N=128), dict(N=128)], simulate=True)           # duplicate class
    with pytest.raises(QmcduError):
        Server([dict(N=100000)], simulate=True)                     # N beyond the limit
    srv = _server()
    with pytest.raises(QmcduError):
        srv.submit([dict(id=0, seed=0, N=100, nsweeps=1, arrival_s=0.0)])   # no such class
    with pytest.raises(QmcduError):
        srv.submit([dict(id=0, seed=0, N=128, nsweeps=0, arrival_s=0.0)])
    srv.close()


def test_serving_trace_is_poisson_over_the_size_set():
    tr = inputs.serving_trace(0, rate_hz=200.0, duration_s=50.0)
    assert tr == inputs.serving_trace(0, rate_hz=200.0, duration_s=50.0)
    n = len(tr)
    assert abs(n - 10000) < 5 * math.sqrt(10000)
    gaps = np.diff([0.0] + [r["arrival_s"] for r in tr])
    assert abs(gaps.mean() - 1 / 200.0) < 5 * (1 / 200.0) / math.sqrt(n)
    counts = np.bincount([inputs.SERVING_SIZES.index(r["N"]) for r in tr], minlength=6)
    assert np.all(np.abs(counts - n / 6) < 5 * math.sqrt(n / 6))
    assert len({r["seed"] for r in tr}) == n


def test_compute_cap_bounds_the_resident_walkers():
    # walker groups of 4 CTAs (N = 512); a cap of 0.1 x 148 SMs = 14.8 CTAs
    # admits three walkers at a time, whatever the slots and the budget allow
    reqs = [dict(id=i, seed=i, N=512, nsweeps=2, arrival_s=0.0) for i in range(10)]
    srv = _server(classes=[dict(N=512, slots=8, group_ctas=4)], sm_oversubscription=0.1)
    res, st = _run(srv, reqs)
    assert st["finished"] == 10 and st["max_resident"] == 3
    srv.close()
    # without the cap all ten are admitted at once (a second pool opens)
    srv = _server(classes=[dict(N=512, slots=8, group_ctas=4)], sm_oversubscription=-1.0)
    res, st = _run(srv, reqs)
    assert st["finished"] == 10 and st["max_resident"] == 10 and st["pools_created"] == 2
    srv.close()
