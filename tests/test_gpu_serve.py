"""Request snapshots (rgg_update_request) and the serving loop on the GPU.

The same rules as the other GPU tests: a request's labels equal the labels of
the one-request-at-a-time path bit for bit (same FP32 arithmetic on the same
poses), and against the FP64 oracle they agree on every edge whose clearance
exceeds 1e-4 m, any other difference being GPU gray.
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


def check_pinned(got, want, where=""):
    pinned = want["kappa"] > PIN
    bad = np.flatnonzero(pinned & (got != want["labels"]))
    assert bad.size == 0, f"{where}: {bad.size} pinned edges differ"
    off = got != want["labels"]
    assert np.all(got[off] == oracle.GRAY), f"{where}: disagreement other than GPU gray"


def small_scene(n_nodes=400, n_boxes=12, seed=0):
    rng = np.random.default_rng(seed)
    robot = W.seven_dof_arm()
    rm = W.prm_roadmap(rng, robot, n_nodes, k=10, step=0.05)
    boxes = W.random_boxes(rng, n_boxes, extent=0.6)
    return rm, boxes, rng


def new_roadmap(rgg, rm, boxes):
    r = rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, boxes.count)
    r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
    r.update_obstacles(np.arange(boxes.count), boxes.poses().astype(np.float32))
    r.classify()
    return r


def request_stream(rng, boxes, n, lo=1, hi=8):
    """n updates of 1..8 boxes each, consecutive ones often sharing boxes."""
    state = boxes.copy()
    return [W.move_boxes(rng, state, int(rng.integers(lo, hi + 1))) for _ in range(n)]


def sequential_labels(rgg, rm, boxes, ups):
    """Reference path: update + classify + fetch, one request at a time."""
    with new_roadmap(rgg, rm, boxes) as r:
        out = []
        for up in ups:
            r.update_obstacles(up.ids, up.poses.astype(np.float32))
            r.classify()
            out.append(r.fetch_labels())
        return out


def test_requests_in_one_pass_equal_one_at_a_time(rgg):
    rm, boxes, rng = small_scene()
    ups = request_stream(rng, boxes, 6)     # 6 requests, < 32 entries: one pass
    want = sequential_labels(rgg, rm, boxes, ups)
    with new_roadmap(rgg, rm, boxes) as r:
        hs = [r.update_request(up.ids, up.poses.astype(np.float32)) for up in ups]
        assert len(set(hs)) == len(hs)
        assert r.info()["open_requests"] == len(hs)
        r.classify()
        got = [r.fetch_request_labels(h) for h in hs]
        final = r.fetch_labels()
        for h in hs:
            r.release_request(h)
        assert r.info()["open_requests"] == 0
    for i, (g, w) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(g, w, err_msg=f"request {i}")
    np.testing.assert_array_equal(final, want[-1])
    # and against the oracle, replaying the box state
    state = boxes.copy()
    for i, up in enumerate(ups):
        state.centre[up.ids] = up.poses[:, :3]
        if i in (0, 3, 5):
            ref = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, state.poses())
            check_pinned(got[i], ref, f"request {i}")


def test_requests_spanning_passes_with_repeated_boxes(rgg):
    # 40 requests moving 1-8 of 12 boxes: ~180 entries over ~6 passes, the
    # same box repeated many times within a pass
    rm, boxes, rng = small_scene(seed=1)
    ups = request_stream(rng, boxes, 40)
    want = sequential_labels(rgg, rm, boxes, ups)
    with new_roadmap(rgg, rm, boxes) as r:
        hs = [r.update_request(up.ids, up.poses.astype(np.float32)) for up in ups]
        assert r.info()["pending_boxes"] == sum(len(u.ids) for u in ups)
        r.classify()
        for i, h in enumerate(hs):
            np.testing.assert_array_equal(r.fetch_request_labels(h), want[i],
                                          err_msg=f"request {i}")
        # box sets after the ordered merges equal the sequential path's
        hit, touch = r.fetch_box_sets()
    with new_roadmap(rgg, rm, boxes) as r2:
        for up in ups:
            r2.update_obstacles(up.ids, up.poses.astype(np.float32))
            r2.classify()
        hit2, touch2 = r2.fetch_box_sets()
    np.testing.assert_array_equal(hit, hit2)
    np.testing.assert_array_equal(touch, touch2)


def test_plain_moves_between_requests(rgg):
    # plain moves before, between and after requests; a plain move of a box
    # that a request moved must not rewrite the request's staged pose
    rm, boxes, rng = small_scene(seed=2)
    ups = request_stream(rng, boxes, 5)
    extra = request_stream(np.random.default_rng(7), boxes, 3)
    plan = [("plain", extra[0]), ("req", ups[0]), ("req", ups[1]), ("plain", extra[1]),
            ("req", ups[2]), ("plain", extra[2]), ("req", ups[3]), ("req", ups[4])]
    # sequential reference: every step classified on its own
    want = []
    with new_roadmap(rgg, rm, boxes) as r:
        for kind, up in plan:
            r.update_obstacles(up.ids, up.poses.astype(np.float32))
            r.classify()
            if kind == "req":
                want.append(r.fetch_labels())
        final_want = r.fetch_labels()
    with new_roadmap(rgg, rm, boxes) as r:
        hs = []
        for kind, up in plan:
            if kind == "req":
                hs.append(r.update_request(up.ids, up.poses.astype(np.float32)))
            else:
                r.update_obstacles(up.ids, up.poses.astype(np.float32))
        r.classify()
        for h, w in zip(hs, want):
            np.testing.assert_array_equal(r.fetch_request_labels(h), w)
        np.testing.assert_array_equal(r.fetch_labels(), final_want)


def test_request_handle_states_and_capacity(rgg):
    rm, boxes, rng = small_scene(n_nodes=150, seed=3)
    up = request_stream(rng, boxes, 1)[0]
    pose = up.poses.astype(np.float32)
    with new_roadmap(rgg, rm, boxes) as r:
        h = r.update_request(up.ids, pose)
        with pytest.raises(rgg.RGGError) as e:
            r.fetch_request_labels(h)          # not classified yet
        assert e.value.status == rgg.RGG_ERR_STATE
        with pytest.raises(rgg.RGGError) as e:
            r.release_request(h)
        assert e.value.status == rgg.RGG_ERR_STATE
        hs = [h] + [r.update_request(up.ids, pose) for _ in range(rgg.MAX_REQUESTS - 1)]
        with pytest.raises(rgg.RGGError) as e:
            r.update_request(up.ids, pose)     # every handle open
        assert e.value.status == rgg.RGG_ERR_CAPACITY
        with pytest.raises(rgg.RGGError) as e:
            r.update_request([], np.zeros((0, 15), np.float32))
        assert e.value.status == rgg.RGG_ERR_INVALID
        r.classify()
        for x in hs:
            r.release_request(x)
        with pytest.raises(rgg.RGGError) as e:
            r.release_request(hs[0])           # already closed
        assert e.value.status == rgg.RGG_ERR_STATE
        # rebuilding the edges closes open handles
        h = r.update_request(up.ids, pose)
        r.classify()
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        assert r.info()["open_requests"] == 0
        with pytest.raises(rgg.RGGError) as e:
            r.fetch_request_labels(h)
        assert e.value.status == rgg.RGG_ERR_STATE
        r.check_status()


def test_pending_entries_are_bounded(rgg):
    rm, _, _ = small_scene(n_nodes=150, seed=5)
    M = 4096
    far = np.zeros((M, 15), np.float32)
    far[:, 0] = 50.0 + np.arange(M) * 0.5          # far from the arm
    far[:, 3:12] = np.eye(3, dtype=np.float32).reshape(9)
    far[:, 12:15] = 0.1
    ids = np.arange(M, dtype=np.uint32)
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, M) as r:
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        cap = r.info()["pending_capacity"]
        assert cap == M + rgg.PENDING_EXTRA
        h = r.update_request(ids, far)              # M entries, then a request boundary
        r.update_obstacles(ids, far)                # M more: the list is full
        assert r.info()["pending_boxes"] == cap
        r.update_obstacles(ids[:3], far[:3])        # same run: replaces, appends nothing
        h2 = r.update_request(ids[:1], far[:1])     # joins the run, ends it
        with pytest.raises(rgg.RGGError) as e:
            r.update_obstacles(ids[:1], far[:1])    # would append entry cap + 1
        assert e.value.status == rgg.RGG_ERR_CAPACITY
        assert r.info()["pending_boxes"] == cap
        r.classify()
        assert np.all(r.fetch_request_labels(h) == rgg.GREEN)
        assert np.all(r.fetch_request_labels(h2) == rgg.GREEN)
        assert r.info()["pending_boxes"] == 0
        r.check_status()


def test_serving_alone_equals_mix(rgg):
    """Continuous batching: every request's labels equal its labels when the
    stream is served one request per launch, and a sample agrees with the
    oracle on the state after that request."""
    import torch
    from paper_2603_28674_gb300 import serve as SV
    scenes, reqs = W.workload_serving(node_counts=(250, 400, 600), rate_hz=100_000.0,
                                      duration_s=0.0015, n_boxes=16)
    assert len(reqs) >= 100
    requests = [SV.ServeRequest(q.arrival_s, q.roadmap, q.update.ids.astype(np.uint32),
                                q.update.poses.astype(np.float32)) for q in reqs]
    res = {}
    for mode in ("batched", "one_at_a_time"):
        srv = SV.Server(device=0, host_slots=48)
        for sc in scenes:
            rm = sc.roadmap
            srv.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(sc.boxes.count),
                            sc.boxes.poses())
        res[mode] = srv.serve(requests, mode, keep_results=True)
        srv.close()
    mix, alone = res["batched"], res["one_at_a_time"]
    assert mix["mean_batch"] > 1.5, "the stream did not batch"
    assert alone["mean_batch"] == 1.0
    for i in range(len(requests)):
        np.testing.assert_array_equal(mix["results"][i], alone["results"][i],
                                      err_msg=f"request {i}")
    # oracle on a sample of requests
    states = [sc.boxes.copy() for sc in scenes]
    for i, q in enumerate(reqs):
        st = states[q.roadmap]
        st.centre[q.update.ids] = q.update.poses[:, :3]
        if i % 25 == 0:
            rm = scenes[q.roadmap].roadmap
            ref = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, st.poses())
            check_pinned(mix["results"][i], ref, f"request {i}")
    torch.cuda.synchronize()


def test_library_estimate_equals_the_built_roadmap(rgg):
    """rgg_estimate_bytes (host arithmetic) equals the device bytes the built
    roadmap reports, and the first request adds the snapshot rows."""
    for seed, nodes in ((4, 200), (5, 30)):
        rm, boxes, _ = small_scene(n_nodes=nodes, seed=seed)
        L, K = rm.robot.num_links, rm.robot.inner_per_link
        est = rgg.estimate_bytes(L, K, boxes.count, rm.q_from, rm.q_to, rm.step)
        with new_roadmap(rgg, rm, boxes) as r:
            assert r.info()["device_bytes"] == est
            h = r.update_request([0], boxes.poses()[:1].astype(np.float32))
            assert r.info()["device_bytes"] == est + rgg.MAX_REQUESTS * rm.num_edges
            r.classify()
            r.release_request(h)


def test_serving_admits_roadmaps_by_memory(rgg):
    from paper_2603_28674_gb300 import serve as SV
    rm, boxes, _ = small_scene(n_nodes=200, seed=4)
    need = SV.roadmap_bytes(rm.robot.num_links, rm.robot.inner_per_link, boxes.count,
                            rm.q_from, rm.q_to, rm.step)
    srv = SV.Server(device=0, memory_budget=int(1.5 * need))
    srv.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(boxes.count),
                    boxes.poses())
    with pytest.raises(MemoryError):
        srv.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(boxes.count),
                        boxes.poses())
    assert len(srv.roadmaps) == 1
    srv.close()


def test_serving_refuses_beyond_the_queue_and_drops_cancelled_requests(rgg):
    """Admission control on the request queue and cancellation of waiting
    requests: every request is completed, refused or cancelled exactly once,
    and the completed ones get the labels of the same stream served without
    the withdrawn requests, one request per launch."""
    from paper_2603_28674_gb300 import serve as SV
    scenes, reqs = W.workload_serving(node_counts=(300, 500), rate_hz=200_000.0,
                                      duration_s=0.0004, n_boxes=16)
    assert len(reqs) >= 40
    burst = [SV.ServeRequest(0.0, q.roadmap, q.update.ids.astype(np.uint32),
                             q.update.poses.astype(np.float32),
                             cancel_s=0.0 if i % 7 == 3 else None)
             for i, q in enumerate(reqs)]
    srv = SV.Server(device=0, max_inflight=1, host_slots=8)
    for sc in scenes:
        rm = sc.roadmap
        srv.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(sc.boxes.count),
                        sc.boxes.poses())
    out = srv.serve(burst, "batched", keep_results=True, max_queue=24)
    n = len(burst)
    assert out["completed"] + out["refused"] + out["cancelled"] == n
    assert out["refused"] == n - 24                  # a burst: all arrive at once
    assert out["cancelled"] >= 1
    done = [i for i in range(n) if out["results"][i] is not None]
    assert len(done) == out["completed"]
    # the completed requests, replayed alone in order, give the same labels
    states = [sc.boxes.copy() for sc in scenes]
    srv2 = SV.Server(device=0)
    for sc in scenes:
        rm = sc.roadmap
        srv2.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(sc.boxes.count),
                         sc.boxes.poses())
    replay = [SV.ServeRequest(0.0, burst[i].roadmap, burst[i].ids, burst[i].poses) for i in done]
    ref = srv2.serve(replay, "one_at_a_time", keep_results=True)
    for j, i in enumerate(done):
        np.testing.assert_array_equal(out["results"][i], ref["results"][j], err_msg=f"request {i}")
    srv.close()
    srv2.close()
