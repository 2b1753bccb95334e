"""Failure detection and recovery on the GPU, without faulting it.

Device side: the classify kernel's bounded waits are given a limit of one
nanosecond (rgg_set_wait_limit), so that a wait for a tile's records or for
the box records runs out in the first launch.  The launch then ends on its own
(its copies drained), the error is latched, later passes are skipped, and
the host reads RGG_ERR_TIMEOUT.  After that the roadmap must recover: the
next classify with the normal limit re-tests every present box, and the
labels and box sets equal those of a fresh roadmap at the same poses.

Host side: rgg_inject_alloc_failure makes the nth device allocation fail as
if the device were full; every call that hits it returns RGG_ERR_OOM and
leaves the roadmap usable and unchanged.

Guard bytes: every library buffer is followed by 64 bytes of a fixed pattern
(rgg_check_guards).  A byte of the label array's guard, which lies inside
the allocation, is changed from the host side and must be reported; every
GPU test also ends with a check that no guard changed (tests/conftest.py).
"""
import numpy as np
import pytest

import oracle
from paper_2603_28674_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PIN = 1e-4


@pytest.fixture(scope="module")
def rgg():
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg as _rgg
    return _rgg


def scene(n_nodes=600, n_boxes=24, seed=11):
    rng = np.random.default_rng(seed)
    robot = W.seven_dof_arm()
    rm = W.prm_roadmap(rng, robot, n_nodes, k=10, step=0.03)
    boxes = W.random_boxes(rng, n_boxes, extent=0.7)
    ups = W.update_stream(rng, boxes, 4, 6)
    return rm, boxes, ups


def fresh_state(rgg, rm, poses):
    """Labels and box sets of a new roadmap with every box at `poses`."""
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, len(poses)) as r:
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(len(poses)), poses)
        r.classify()
        return (r.fetch_labels(), *r.fetch_box_sets())


def test_wait_that_runs_out_is_reported_and_the_roadmap_recovers(rgg):
    import torch
    rm, boxes, ups = scene()
    poses = boxes.poses().astype(np.float32)
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, boxes.count) as r:
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(boxes.count), poses)
        r.classify()
        before = r.fetch_labels()
        r.set_wait_limit(1)                  # 1 ns: a wait that is not over at once runs out
        h = None
        timed_out = False
        for k, up in enumerate(ups):
            r.update_obstacles(up.ids, up.poses.astype(np.float32))
            poses[up.ids] = up.poses.astype(np.float32)
            if k == 1:
                h = r.update_request(up.ids[:1], up.poses[:1].astype(np.float32))
            r.classify()                     # enqueued; later passes are skipped on the device
            try:
                r.check_status()
            except rgg.RGGError as e:
                assert e.status == rgg.RGG_ERR_TIMEOUT
                timed_out = True
                break
        assert timed_out, "no bounded wait ran out at a 1 ns limit"
        torch.cuda.synchronize()             # the context is healthy
        # the failed passes changed nothing; the boxes are queued again
        np.testing.assert_array_equal(r.fetch_labels(), before)
        assert r.info()["pending_boxes"] == boxes.count
        r.check_status()                     # cleared by the first report
        if h is not None:
            with pytest.raises(rgg.RGGError) as e:
                r.fetch_request_labels(h)
            assert e.value.status == rgg.RGG_ERR_TIMEOUT
            r.release_request(h)
        assert r.info()["open_requests"] == 0
        # recovery at the normal limit: every present box re-tested
        r.set_wait_limit(4_000_000_000)
        r.classify()
        got = (r.fetch_labels(), *r.fetch_box_sets())
        r.check_status()
    want = fresh_state(rgg, rm, poses)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
    ref = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, poses.astype(np.float64))
    pinned = ref["kappa"] > PIN
    assert np.array_equal(got[0][pinned], ref["labels"][pinned])


def test_batched_launch_that_times_out_latches_every_roadmap(rgg):
    rm, boxes, ups = scene(n_nodes=300, seed=12)
    rm2, boxes2, ups2 = scene(n_nodes=350, seed=13)
    rs = []
    for m, b in ((rm, boxes), (rm2, boxes2)):
        r = rgg.Roadmap(m.robot.num_links, m.robot.inner_per_link, b.count)
        r.build_edges(m.robot, m.q_from, m.q_to, m.step)
        r.update_obstacles(np.arange(b.count), b.poses().astype(np.float32))
        rs.append(r)
    rgg.classify_many(rs)
    before = [r.fetch_labels() for r in rs]
    rs[0].set_wait_limit(1)                  # the launch takes the first roadmap's limit
    failed = [False, False]
    for k in range(3):
        for r, u in zip(rs, (ups, ups2)):
            r.update_obstacles(u[k].ids, u[k].poses.astype(np.float32))
        rgg.classify_many(rs)
        for i, r in enumerate(rs):
            try:
                r.check_status()
            except rgg.RGGError as e:
                assert e.status == rgg.RGG_ERR_TIMEOUT
                failed[i] = True
        if any(failed):
            break
    assert all(failed), "a timed-out batched launch must latch the error on every roadmap"
    for r, b in zip(rs, before):
        np.testing.assert_array_equal(r.fetch_labels(), b)
    rs[0].set_wait_limit(4_000_000_000)
    rgg.classify_many(rs)
    for r, m, b, u in zip(rs, (rm, rm2), (boxes, boxes2), (ups, ups2)):
        poses, present = r.fetch_boxes()
        want = fresh_state(rgg, m, poses)
        np.testing.assert_array_equal(r.fetch_labels(), want[0])
        r.check_status()
        r.close()


def test_allocation_failures_leave_the_roadmap_usable(rgg):
    """The nth device allocation of a create / build / update / classify /
    rebuild / request sequence fails, for every n until the sequence runs
    clean: each call that meets it returns RGG_ERR_OOM, the same call then
    succeeds, a rebuild that failed keeps the previous edges, and the labels
    are always those of a fresh roadmap."""
    rm, boxes, _ = scene(n_nodes=200, seed=14)
    rm_b = W.prm_roadmap(np.random.default_rng(15), rm.robot, 150, k=8, step=0.04)
    poses = boxes.poses().astype(np.float32)
    L, K, M = rm.robot.num_links, rm.robot.inner_per_link, boxes.count
    want_a = fresh_state(rgg, rm, poses)[0]
    want_b = fresh_state(rgg, rm_b, poses)[0]
    seen = set()
    try:
        for nth in range(1, 400):
            rgg.inject_alloc_failure(nth)
            failed = []

            def attempt(name, f, *a, retry=True):
                try:
                    return f(*a)
                except rgg.RGGError as e:
                    assert e.status == rgg.RGG_ERR_OOM, (name, e)
                    failed.append(name)
                    return f(*a) if retry else None

            r = attempt("create", rgg.Roadmap, L, K, M)
            attempt("build", r.build_edges, rm.robot, rm.q_from, rm.q_to, rm.step)
            attempt("update", r.update_obstacles, np.arange(M), poses)
            attempt("classify", r.classify)
            np.testing.assert_array_equal(r.fetch_labels(), want_a)
            n_before = len(failed)
            attempt("rebuild", r.build_edges, rm_b.robot, rm_b.q_from, rm_b.q_to, rm_b.step,
                    retry=False)
            rebuilt = len(failed) == n_before
            attempt("classify after rebuild", r.classify)
            np.testing.assert_array_equal(r.fetch_labels(), want_b if rebuilt else want_a)
            h = attempt("request", r.update_request, [0], poses[:1])
            r.classify()
            np.testing.assert_array_equal(r.fetch_request_labels(h), r.fetch_labels())
            r.release_request(h)
            r.check_status()
            rgg.inject_alloc_failure(0)
            r.close()
            seen.update(failed)
            if not failed:
                break
        else:
            pytest.fail("the sequence never ran clean")
    finally:
        rgg.inject_alloc_failure(0)
    assert {"create", "build", "rebuild", "request"} <= seen, seen


def test_guard_bytes_report_a_write_past_a_buffer(rgg):
    import torch
    rm, boxes, ups = scene(n_nodes=200)
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, boxes.count) as r:
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(boxes.count), boxes.poses().astype(np.float32))
        r.classify()
        for up in ups:
            r.update_obstacles(up.ids, up.poses.astype(np.float32))
            r.classify()
        checked, bad = rgg.check_guards()
        assert checked >= 10 and bad == 0
        # the label array (N bytes) has its guard at N rounded up to 16 B:
        # inside the allocation, so this host-side write stays in bounds
        n = r.info()["num_edges"]
        at = r.labels_device_ptr() + ((n + 15) & ~15)

        class View:
            __cuda_array_interface__ = {"shape": (1,), "typestr": "|u1", "data": (at, False),
                                        "version": 3}

        g = torch.as_tensor(View(), device="cuda")
        assert int(g.item()) == 0xA5
        g.fill_(0x5A)
        torch.cuda.synchronize()
        assert rgg.check_guards() == (checked, 1)
        g.fill_(0xA5)
        torch.cuda.synchronize()
        assert rgg.check_guards() == (checked, 0)
    # the roadmap's buffers are no longer listed once it is destroyed
    assert rgg.check_guards()[0] <= checked - 10
