"""Scheduling logic of the serving loop, on the CPU with a fake solver:
memory cap, slot limit, first-fit admission past a blocked head, errors."""

import threading
import time

import numpy as np
import pytest

from paper_1805_10121_gb300 import serve


def fake_solver(duration_of, log):
    lock = threading.Lock()

    def solve(req, slot):
        with lock:
            log.append(("start", req.rid, slot, time.perf_counter()))
        time.sleep(duration_of(req))
        with lock:
            log.append(("end", req.rid, slot, time.perf_counter()))
        return {"statuses": [0] * req.nprob, "iterations": [1] * req.nprob,
                "ritz": [np.zeros(1)] * req.nprob, "resid_max_over_norm": [0.0] * req.nprob,
                "flops": 1.0}
    return solve


def mk(rid, n, arrival, nprob=2):
    return serve.Request(rid, n, 4, 1, nprob, rid + 1, arrival)


def test_trace_is_seeded_and_shaped():
    a = serve.poisson_trace(50, 20.0, 7)
    b = serve.poisson_trace(50, 20.0, 7)
    assert a == b
    assert all(r.n in (2048, 4096, 8192, 16384) for r in a)
    assert all(5 <= r.nprob <= 10 for r in a)
    assert all(r.nev == int(np.ceil(0.04 * r.n)) for r in a)
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    assert 1.0 < arr[-1] < 6.0  # 50 arrivals at 20/s


def test_memory_cap_and_slots_respected():
    log = []
    trace = [mk(i, 100 * (1 + i % 3), 0.001 * i) for i in range(9)]
    fp = lambda r: r.n  # bytes = n
    srv = serve.Server(fake_solver(lambda r: 0.05, log), mem_cap_bytes=450, max_slots=3,
                       footprint_fn=fp)
    res = srv.run(trace)
    assert [r.rid for r in res] == list(range(9))
    assert srv.peak_mem <= 450
    assert srv.peak_concurrency <= 3
    # replay the log: running footprint never exceeds the cap
    running, peak = {}, 0
    for ev, rid, slot, _ in sorted(log, key=lambda e: e[3]):
        if ev == "start":
            running[rid] = trace[rid].n
        else:
            running.pop(rid)
        peak = max(peak, sum(running.values()))
    assert peak <= 450
    assert all(r.latency >= r.queueing >= 0 for r in res)


def test_first_fit_admits_smaller_request_past_blocked_head():
    log = []
    # request 0 (300) runs; request 1 (300) cannot fit under 500 until 0 ends;
    # request 2 (150) arrives later but fits now and must start before 1
    trace = [mk(0, 300, 0.0), mk(1, 300, 0.01), mk(2, 150, 0.02)]
    srv = serve.Server(fake_solver(lambda r: 0.2 if r.rid == 0 else 0.05, log),
                       mem_cap_bytes=500, max_slots=4, footprint_fn=lambda r: r.n)
    res = srv.run(trace)
    starts = {rid: t for ev, rid, _, t in log if ev == "start"}
    assert starts[2] < starts[1]
    assert res[1].queueing > res[2].queueing


def test_oversized_request_raises():
    srv = serve.Server(fake_solver(lambda r: 0.0, []), mem_cap_bytes=10, max_slots=1,
                       footprint_fn=lambda r: r.n)
    with pytest.raises(ValueError):
        srv.run([mk(0, 100, 0.0)])


def test_solver_error_propagates():
    def bad(req, slot):
        raise RuntimeError("boom")
    srv = serve.Server(bad, mem_cap_bytes=1e9, max_slots=2, footprint_fn=lambda r: 1)
    with pytest.raises(RuntimeError):
        srv.run([mk(0, 10, 0.0)])


def test_footprint_grows_with_n_and_split():
    a = serve.footprint_bytes(2048, 82, 17, split=False)
    b = serve.footprint_bytes(2048, 82, 17, split=True)
    c = serve.footprint_bytes(4096, 164, 33, split=True)
    assert b > a and c > 3 * b


def _start_order(policy, max_wait_s=None):
    log = []
    dur = {0: 0.25, 1: 0.02, 2: 0.02}
    srv = serve.Server(fake_solver(lambda r: dur[r.rid], log), 1e12, 1,
                       lambda r: 1, policy=policy, max_wait_s=max_wait_s)
    # request 0 holds the only slot while 1 (large) and 2 (small) queue up
    trace = [mk(0, 64, 0.0), mk(1, 4096, 0.02), mk(2, 256, 0.04)]
    srv.run(trace)
    return [rid for ev, rid, _, _ in sorted(log, key=lambda e: e[3]) if ev == "start"]


def test_sjf_admits_the_cheapest_waiting_request_first():
    assert _start_order("fifo") == [0, 1, 2]
    assert _start_order("sjf") == [0, 2, 1]
    c = [serve.work_estimate(mk(i, n, 0.0)) for i, n in enumerate((256, 4096))]
    assert c[0] < c[1]


def test_sjf_aging_lets_a_long_waiter_go_first():
    # both queued requests have waited past max_wait_s when the slot frees:
    # the older one (the large request) goes first
    assert _start_order("sjf", max_wait_s=0.05) == [0, 1, 2]


def test_unknown_policy_is_rejected():
    with pytest.raises(ValueError):
        serve.Server(lambda r, s: {}, 1e9, 1, lambda r: 1, policy="lifo")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sjf_on_random_traces(seed):
    rng = np.random.default_rng(seed)
    trace = [mk(i, int(rng.choice([64, 256, 1024, 4096])), 0.0, nprob=int(rng.integers(1, 6)))
             for i in range(12)]
    # one slot, everything waiting from the start: starts in order of cost
    log = []
    serve.Server(fake_solver(lambda r: 0.002, log), 1e12, 1, lambda r: 1,
                 policy="sjf").run(trace, realtime=False)
    starts = [rid for ev, rid, _, _ in sorted(log, key=lambda e: e[3]) if ev == "start"]
    costs = [serve.work_estimate(trace[rid]) for rid in starts]
    assert sorted(starts) == list(range(12))
    assert costs == sorted(costs)
    # three slots under a memory cap: caps hold and every request finishes
    log = []
    srv = serve.Server(fake_solver(lambda r: 0.002 * r.nprob, log), 10.0, 3,
                       lambda r: 1 + (r.n >= 1024) * 3, policy="sjf")
    res = srv.run(trace, realtime=False)
    assert [r.rid for r in res] == list(range(12))
    assert srv.peak_concurrency <= 3 and srv.peak_mem <= 10.0
