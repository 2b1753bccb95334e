"""Non-lazy resolution of gray edges (rgg_resolve_gray) against the oracle's
dense capsule-box clearance (the exact robot geometry at (n_e - 1) F + 1
configurations).

Rules checked, edge by edge:
  * edges that are not gray keep their label;
  * a gray edge resolved RED has oracle clearance < 0 (it collides), one
    resolved GREEN has clearance > 0 (it is free) -- on every edge;
  * an edge whose oracle clearance exceeds 1e-4 m in magnitude is resolved
    (never left gray);
  * the GPU clearance over the edge's touch set equals the oracle's over the
    same boxes within 2e-5 m (edges not resolved RED).
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


def scenes():
    rng = np.random.default_rng(21)
    planar = W.workload_planar(n_nodes=300, n_updates=0)
    arm = W.dh_arm(rng, 7)
    rm7 = W.prm_roadmap(rng, arm, 150, 10, 0.05)
    boxes7 = W.random_boxes(rng, 16)
    return [("planar", planar.roadmap, planar.boxes, 4), ("7dof", rm7, boxes7, 2)]


def bits_of(row, m):
    return np.array([(row[b >> 5] >> (b & 31)) & 1 for b in range(m)], dtype=np.uint8)


@pytest.mark.parametrize("which", [0, 1])
def test_resolution_matches_dense_oracle(rgg, which):
    name, rm, boxes, factor = scenes()[which]
    robot = rm.robot
    poses = boxes.poses()
    m = boxes.count
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, m) as r:
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(m), f32(poses))
        r.classify()
        lazy = r.fetch_labels()
        _, touch = r.fetch_box_sets()
        res, clear, stats = r.resolve_gray(factor)
        np.testing.assert_array_equal(r.fetch_labels(), lazy)   # lazy state untouched
        r.check_status()
    gray = np.flatnonzero(lazy == rgg.GRAY)
    assert gray.size >= 10, f"{name}: too few gray edges for a meaningful test"
    keep = lazy != rgg.GRAY
    np.testing.assert_array_equal(res[keep], lazy[keep])
    assert np.all(np.isnan(clear[keep]))
    assert stats["gray_edges"] == gray.size
    assert stats["resolved_red"] == int((res[gray] == rgg.RED).sum())
    assert stats["resolved_green"] == int((res[gray] == rgg.GREEN).sum())
    assert stats["resolved_red"] > 0 and stats["resolved_green"] > 0
    for e in gray:
        full, _ = oracle.edge_dense_clearance(robot, rm.q_from[e], rm.q_to[e], rm.step, factor,
                                              poses)
        if res[e] == rgg.RED:
            assert full < 0.0, (name, e, full)
        elif res[e] == rgg.GREEN:
            assert full > 0.0, (name, e, full)
        if abs(full) > PIN:
            assert res[e] == (rgg.RED if full < 0 else rgg.GREEN), (name, e, full)
        if res[e] != rgg.RED:
            mine, _ = oracle.edge_dense_clearance(robot, rm.q_from[e], rm.q_to[e], rm.step,
                                                  factor, poses, present=bits_of(touch[e], m))
            assert abs(float(clear[e]) - mine) <= 2e-5, (name, e, clear[e], mine)


def test_resolution_needs_built_edges_and_no_pending(rgg):
    _, rm, boxes, _ = scenes()[0]
    robot = rm.robot
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, boxes.count) as r:
        with pytest.raises(rgg.RGGError) as e:
            r.resolve_gray(2)
        assert e.value.status == rgg.RGG_ERR_STATE
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
        with pytest.raises(rgg.RGGError) as e:
            r.resolve_gray(2)          # pending moves
        assert e.value.status == rgg.RGG_ERR_STATE
        r.classify()
        for bad in (0, 101):
            with pytest.raises(rgg.RGGError) as e:
                r.resolve_gray(bad)
            assert e.value.status == rgg.RGG_ERR_INVALID
        inner, outer, soff = r.fetch_records()
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, boxes.count) as u:
        u.upload_edges(soff, inner, outer)   # no robot kept: nothing to check against
        u.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
        u.classify()
        with pytest.raises(rgg.RGGError) as e:
            u.resolve_gray(2)
        assert e.value.status == rgg.RGG_ERR_STATE
