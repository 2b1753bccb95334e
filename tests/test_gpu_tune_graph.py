"""The library's autotuner and captured step graphs on the GPU.

Neither may change a label: after autotuning, and when a step runs as one
graph launch, labels and box sets equal those of the plain call sequence
bit for bit, and a sample agrees with the FP64 oracle under the
pinned-edge rule.
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


def f32(x):
    return np.asarray(x, dtype=np.float32)


def placed(rgg, sc):
    rm = sc.roadmap
    r = rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, sc.boxes.count)
    r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
    r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
    return r


def same_state(a, b):
    np.testing.assert_array_equal(a.fetch_labels(), b.fetch_labels())
    ha, ta = a.fetch_box_sets()
    hb, tb = b.fetch_box_sets()
    np.testing.assert_array_equal(ha, hb)
    np.testing.assert_array_equal(ta, tb)


def test_autotune_sets_a_timed_shape_and_keeps_labels(rgg):
    sc = W.workload_7dof(n_nodes=1500, n_updates=2)
    with placed(rgg, sc) as r, placed(rgg, sc) as ref:
        r.classify()
        ref.classify()
        before = r.fetch_labels()
        res = rgg.autotune([r], reps=1)
        # every compiled variant with at least one warp count was timed
        assert len({x["variant"] for x in res}) == rgg.NUM_VARIANTS
        ms = [x["classify_ms"] for x in res]
        assert ms == sorted(ms) and ms[0] > 0
        np.testing.assert_array_equal(r.fetch_labels(), before)
        assert r.info()["pending_boxes"] == 0
        # the chosen shape is in effect and classifies like the default one
        for up in sc.updates:
            for x in (r, ref):
                x.update_obstacles(up.ids, f32(up.poses))
                x.classify()
        same_state(r, ref)
        r.check_status()


def test_autotune_many_roadmaps_then_batched_classify(rgg):
    scenes = W.workload_batched(n_roadmaps=4, edge_lo=300, edge_hi=3000, n_updates=1)
    tuned = [placed(rgg, sc) for sc in scenes]
    plain = [placed(rgg, sc) for sc in scenes]
    rgg.classify_many(tuned)
    rgg.classify_many(plain)
    res = rgg.autotune(tuned, reps=1)
    assert res
    for sc, t, p in zip(scenes, tuned, plain):
        up = sc.updates[0]
        t.update_obstacles(up.ids, f32(up.poses))
        p.update_obstacles(up.ids, f32(up.poses))
    rgg.classify_many(tuned)
    rgg.classify_many(plain)
    for t, p in zip(tuned, plain):
        same_state(t, p)
    for x in tuned + plain:
        x.close()


def test_autotune_without_boxes_keeps_the_shape(rgg):
    sc = W.workload_planar(n_nodes=100, n_updates=0)
    rm = sc.roadmap
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, 4) as r:
        r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        ts = r.info()["tile_samples"]
        assert rgg.autotune([r]) == []
        assert r.info()["tile_samples"] == ts


def test_step_graph_replays_equal_call_by_call(rgg):
    import torch
    scenes = W.workload_batched(n_roadmaps=5, edge_lo=300, edge_hi=4000, n_updates=3)
    calls = [placed(rgg, sc) for sc in scenes]
    graphed = [placed(rgg, sc) for sc in scenes]
    rgg.classify_many(calls)
    rgg.classify_many(graphed)
    # one graph per update index; its poses live in device buffers that are
    # refilled before each launch
    bufs = [[torch.zeros((len(sc.updates[k].ids), 15), dtype=torch.float32, device="cuda")
             for sc in scenes] for k in range(3)]
    graphs = [rgg.StepGraph(graphed, [(sc.updates[k].ids, bufs[k][i])
                                      for i, sc in enumerate(scenes)]) for k in range(3)]
    assert graphs[0].nodes() >= 4
    stream = torch.cuda.current_stream()
    for step in range(6):
        k = step % 3
        for i, sc in enumerate(scenes):
            up = sc.updates[k]
            calls[i].update_obstacles(up.ids, f32(up.poses))
            bufs[k][i].copy_(torch.from_numpy(f32(up.poses)))
        rgg.classify_many(calls)
        graphs[k].launch(stream)
        torch.cuda.synchronize()
        for c, g in zip(calls, graphed):
            same_state(c, g)
    # oracle on one roadmap after the last step (update index 2 last)
    sc, g = scenes[1], graphed[1]
    boxes = sc.boxes.copy()
    for k in (0, 1, 2):
        boxes.centre[sc.updates[k].ids] = sc.updates[k].poses[:, :3]
    rm = sc.roadmap
    want = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
    got = g.fetch_labels()
    pinned = want["kappa"] > PIN
    assert np.all(got[pinned] == want["labels"][pinned])
    assert np.all(got[got != want["labels"]] == oracle.GRAY)
    # rules: no pending moves at launch; replaced edges invalidate the graph
    up = scenes[0].updates[0]
    graphed[0].update_obstacles(up.ids, f32(up.poses))
    with pytest.raises(rgg.RGGError) as e:
        graphs[0].launch(stream)
    assert e.value.status == rgg.RGG_ERR_STATE
    graphed[0].classify()
    graphs[0].launch(stream)
    rm0 = scenes[0].roadmap
    graphed[0].build_edges(rm0.robot, rm0.q_from, rm0.q_to, rm0.step)
    graphed[0].classify()
    with pytest.raises(rgg.RGGError) as e:
        graphs[1].launch(stream)
    assert e.value.status == rgg.RGG_ERR_STATE
    up2 = scenes[2].updates[0]
    graphed[2].update_obstacles(up2.ids, f32(up2.poses))   # a pending move
    with pytest.raises(rgg.RGGError) as e:
        rgg.StepGraph(graphed, [(sc.updates[0].ids, bufs[0][i]) for i, sc in enumerate(scenes)])
    assert e.value.status == rgg.RGG_ERR_STATE
    assert graphed[2].info()["pending_boxes"] == len(up2.ids)
    for gr in graphs:
        gr.close()
    torch.cuda.synchronize()
    for x in calls + graphed:
        x.check_status()
        x.close()
