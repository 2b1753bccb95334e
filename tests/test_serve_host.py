"""Host logic of the serving loop: admission, refusal, cancellation and the
library's memory estimate (no GPU needed)."""
import collections

import numpy as np
import pytest

import oracle
from paper_2603_28674_gb300 import workloads as W
from paper_2603_28674_gb300.serve import Planner, RequestQueue, roadmap_bytes


def test_admission_keeps_per_roadmap_order_and_capacities():
    # items are (arrival index, roadmap)
    q = collections.deque([(0, 0), (1, 1), (2, 0), (3, 2), (4, 0), (5, 1)])
    pl = Planner(n_roadmaps=3, handles_per_roadmap=2, host_slots=5)
    got = pl.admit(q, lambda it: it[1])
    # roadmap 0 has two handles: request 4 waits; nothing else is blocked
    assert [i for i, _ in got] == [0, 1, 2, 3, 5]
    assert [i for i, _ in q] == [4]
    assert pl.free_handles == [0, 0, 1] and pl.free_slots == 0
    # no slot left: nothing is admitted even though roadmap 2 has a handle
    q.append((6, 2))
    assert pl.admit(q, lambda it: it[1]) == []
    pl.release(0)
    got = pl.admit(q, lambda it: it[1])
    assert [i for i, _ in got] == [4]
    assert [i for i, _ in q] == [6]


def test_blocked_request_holds_back_only_its_own_roadmap():
    q = collections.deque([(0, 0), (1, 0), (2, 1), (3, 0), (4, 1)])
    pl = Planner(n_roadmaps=2, handles_per_roadmap=1, host_slots=10)
    got = pl.admit(q, lambda it: it[1])
    assert [i for i, _ in got] == [0, 2]
    # request 3 (roadmap 0) must not overtake request 1 once a handle frees
    pl.release(0)
    got = pl.admit(q, lambda it: it[1])
    assert [i for i, _ in got] == [1]
    assert [i for i, _ in q] == [3, 4]


def test_one_at_a_time_limit():
    q = collections.deque([(i, i % 3) for i in range(6)])
    pl = Planner(n_roadmaps=3, handles_per_roadmap=64, host_slots=64)
    order = []
    while q:
        got = pl.admit(q, lambda it: it[1], limit=1)
        assert len(got) == 1
        order.append(got[0][0])
        pl.release(got[0][1])
    assert order == list(range(6))


def test_queue_and_admission_work_does_not_grow_with_the_backlog():
    # a long backlog (one request per launch falling behind) must not make
    # every loop iteration walk it: a sweep looks up each arrival's
    # cancellation time once, and admission stops once nothing more fits
    q = RequestQueue()
    for i in range(10000):
        q.arrive(i)
    calls = []

    def cancel_at(i):
        calls.append(i)
        return None

    for _ in range(50):
        q.sweep(1.0, cancel_at)
    assert len(calls) == 10000
    pl = Planner(n_roadmaps=1, handles_per_roadmap=64, host_slots=64)
    seen = []

    def roadmap_of(i):
        seen.append(i)
        return 0

    assert pl.admit(q.items, roadmap_of, limit=1) == [0]
    assert seen == [0] and q.items[0] == 1 and len(q.items) == 9999
    # without a limit the walk ends when the roadmap's 64 handles are taken
    seen.clear()
    got = pl.admit(q.items, roadmap_of)
    assert got == list(range(1, 64)) and len(seen) == 63 and q.items[0] == 64


@pytest.fixture(scope="module")
def built():
    from paper_2603_28674_gb300 import build
    build.build()


def test_memory_estimate_covers_the_records(built):
    # the library's estimate (host arithmetic) counts the configurations by
    # the sample-count rule, which the oracle pins
    from paper_2603_28674_gb300 import rgg
    sc = W.workload_7dof(n_nodes=300, n_updates=0)
    rm, robot = sc.roadmap, sc.roadmap.robot
    n_e = np.array([oracle.num_samples(rm.q_from[e], rm.q_to[e], rm.step)
                    for e in range(rm.num_edges)])
    S, N = int(n_e.sum()), rm.num_edges
    L, K = robot.num_links, robot.inner_per_link
    # link-end records (the default): 12 B per (edge, link, configuration);
    # sphere records: 16 B per inner sphere; 16 B per outer sphere in both
    for fmt, records in ((rgg.RECORDS_LINK_ENDS, 12 * L * S + 16 * L * (S - N)),
                         (rgg.RECORDS_SPHERES, 16 * (K * L * S + L * (S - N)))):
        est = rgg.estimate_bytes(L, K, sc.boxes.count, rm.q_from, rm.q_to, rm.step,
                                 record_format=fmt)
        # per edge at least the offsets, box sets, counts, label, pass bits and endpoints;
        # link-end records also hold the spatial filter's round data, 24 B per
        # round slot, 32 slots per tile of at least 31 configurations
        rounds = 24 * 32 * (L * S // 31 + 1) if fmt == rgg.RECORDS_LINK_ENDS else 0
        assert est >= records + N * (8 + 8 + 4 + 1 + 8 + 16 * L)
        assert est <= records + N * (64 + 16 * L) + rounds + (1 << 20)
    est = rgg.estimate_bytes(L, K, sc.boxes.count, rm.q_from, rm.q_to, rm.step)
    assert roadmap_bytes(L, K, sc.boxes.count, rm.q_from, rm.q_to, rm.step) == est + 64 * N
    # a margin below 1e-5 m keeps sphere records
    assert rgg.estimate_bytes(L, K, sc.boxes.count, rm.q_from, rm.q_to, rm.step, margin=0.0) == \
        rgg.estimate_bytes(L, K, sc.boxes.count, rm.q_from, rm.q_to, rm.step, margin=0.0,
                           record_format=rgg.RECORDS_SPHERES)


def test_memory_estimate_rejects_bad_arguments(built):
    from paper_2603_28674_gb300 import rgg
    q = np.zeros((2, 3))
    with pytest.raises(rgg.RGGError):
        rgg.estimate_bytes(3, 4, 16, q, q, 0.0)          # step must be positive
    with pytest.raises(rgg.RGGError):
        rgg.estimate_bytes(3, 4, 16, q, q + np.inf, 0.05)
    assert rgg.estimate_bytes(3, 4, 16, q[:0], q[:0], 0.05) > 0   # no edges: fixed tables


def test_request_queue_refuses_beyond_its_length_and_cancels_waiting_requests():
    q = RequestQueue(max_len=2)
    assert q.arrive(0) and q.arrive(1)
    assert not q.arrive(2)                   # full: refused at once
    assert q.refused == [2] and list(q.items) == [0, 1]
    cancel = {0: 5.0, 1: None, 3: 1.0}
    q.sweep(1.0, cancel.get)                 # nothing due yet among the waiting
    assert list(q.items) == [0, 1]
    assert q.arrive(3) is False              # still full
    q.sweep(5.0, cancel.get)                 # request 0 withdraws while waiting
    assert q.cancelled == [0] and list(q.items) == [1]
    assert q.arrive(3)
    q.sweep(6.0, cancel.get)                 # 3's time has passed: it leaves too
    assert q.cancelled == [0, 3] and list(q.items) == [1]
    unbounded = RequestQueue()
    assert all(unbounded.arrive(i) for i in range(1000))
