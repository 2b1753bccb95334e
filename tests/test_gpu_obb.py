"""The OBB / shortcut-spline geometry (the paper's own primitives, Sec. 4.2
and 4.3) on the GPU against the FP64 oracle.

Rules:
  * boxes: centre and axes within FP32 rounding of the oracle's, half-extents
    at least the oracle's and at most 3e-6 m more;
  * splines: the same kept vertices (count and position within 1e-6 m);
  * labels: identical on every edge whose oracle clearance exceeds 1e-4 m,
    any other difference being GPU gray; GPU hit set within the oracle's,
    the oracle's touch set within the GPU's;
  * the spatial filter changes no bit; incremental updates equal a
    classification from scratch; requests and the gray resolution work on
    this geometry too.
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


def scene(which):
    """Sparse scenes (one box per edge box would leave nothing green):
    a planar arm among 5 boxes, a 7-DOF arm among 8."""
    rng = np.random.default_rng(40 + which)
    if which == 0:
        rm = W.prm_roadmap(rng, W.planar_arm(), 200, 6, 0.05)
        boxes = W.random_boxes(rng, 5, planar=True, oriented=False, extent=1.0)
        return rm, boxes, W.update_stream(rng, boxes, 3, 2, planar=True)
    arm = W.dh_arm(rng, 7)
    rm = W.prm_roadmap(rng, arm, 150, 10, 0.04)
    boxes = W.random_boxes(rng, 8, half_lo=0.03, half_hi=0.1)
    return rm, boxes, W.update_stream(rng, boxes, 3, 3)


def obb_roadmap(rgg, rm, m):
    r = rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, m, geometry=rgg.GEOMETRY_OBB)
    r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
    return r


def check_labels(got, want, where):
    pinned = want["kappa"] > PIN
    bad = np.flatnonzero(pinned & (got != want["labels"]))
    assert bad.size == 0, f"{where}: {bad.size} pinned edges differ, first {bad[:5]}"
    off = got != want["labels"]
    assert np.all(got[off] == oracle.GRAY), f"{where}: disagreement other than GPU gray"
    return int(off.sum())


@pytest.mark.parametrize("which", [0, 1])
def test_boxes_and_splines_match_oracle(rgg, which):
    rm, boxes, _ = scene(which)
    robot = rm.robot
    L, K = robot.num_links, robot.inner_per_link
    with obb_roadmap(rgg, rm, boxes.count) as r:
        info = r.info()
        assert info["geometry"] == rgg.GEOMETRY_OBB and info["grid_cells"] >= 1
        obb, off, verts = r.fetch_obb_records()
    for e in range(0, rm.num_edges, max(1, rm.num_edges // 60)):
        want = oracle.edge_obbs(robot, rm.q_from[e], rm.q_to[e], rm.step)
        sp = oracle.edge_splines(robot, rm.q_from[e], rm.q_to[e], rm.step)
        for i in range(L):
            g = obb[e, i]
            c, axes, half = g[:3], g[[4, 5, 6, 8, 9, 10, 12, 13, 14]].reshape(3, 3), g[[7, 11, 15]]
            np.testing.assert_allclose(c, want[i, :3], atol=1e-6)
            np.testing.assert_allclose(axes, want[i, 3:12].reshape(3, 3).T, atol=1e-6)
            assert np.all(half >= want[i, 12:] - 1e-7) and np.all(half <= want[i, 12:] + 3e-6)
            for s in range(K):
                k = (e * L + i) * K + s
                v = verts[int(off[k]):int(off[k + 1]), :3]
                assert v.shape[0] == sp[i][s].shape[0], (e, i, s)
                np.testing.assert_allclose(v, sp[i][s], atol=1e-6)


@pytest.mark.parametrize("which", [0, 1])
def test_labels_match_oracle_and_filter_changes_nothing(rgg, which):
    rm, boxes, ups = scene(which)
    robot = rm.robot
    m = boxes.count
    state = boxes.copy()
    with obb_roadmap(rgg, rm, m) as r, obb_roadmap(rgg, rm, m) as u:
        u.set_obb_filter(False)
        for x in (r, u):
            x.update_obstacles(np.arange(m), f32(state.poses()))
            x.classify()
        for step, up in enumerate([None] + list(ups)):
            if up is not None:
                state.centre[up.ids] = up.poses[:, :3]
                for x in (r, u):
                    x.update_obstacles(up.ids, f32(up.poses))
                    x.classify()
            want = oracle.classify_obb(robot, rm.q_from, rm.q_to, rm.step, state.poses(), bits=True)
            got = r.fetch_labels()
            check_labels(got, want, f"step {step}")
            hit, touch = r.fetch_box_sets()
            w = want["hit"].shape[1]
            assert np.all((hit[:, :w] & ~want["hit"]) == 0), "GPU hit outside the oracle's"
            assert np.all((want["touch"] & ~touch[:, :w]) == 0), "oracle touch missing"
            hu, tu = u.fetch_box_sets()
            np.testing.assert_array_equal(hit, hu)
            np.testing.assert_array_equal(touch, tu)
        lab = want["labels"]
        assert (lab == oracle.RED).any() and (lab == oracle.GREEN).any() and \
            (lab == oracle.GRAY).any()
        sat_f, seg_f = r.obb_work()
        sat_u, seg_u = u.obb_work()
        assert 0 < sat_f <= sat_u
        r.check_status()


def test_incremental_requests_and_resolution(rgg):
    rm, boxes, ups = scene(1)
    robot = rm.robot
    m = boxes.count
    final = boxes.copy()
    for up in ups:
        final.centre[up.ids] = up.poses[:, :3]
    with obb_roadmap(rgg, rm, m) as r, obb_roadmap(rgg, rm, m) as fresh, \
            obb_roadmap(rgg, rm, m) as req:
        for x in (r, req):
            x.update_obstacles(np.arange(m), f32(boxes.poses()))
            x.classify()
        want_each = []
        for up in ups:
            r.update_obstacles(up.ids, f32(up.poses))
            r.classify()
            want_each.append(r.fetch_labels())
        fresh.update_obstacles(np.arange(m), f32(final.poses()))
        fresh.classify()
        np.testing.assert_array_equal(r.fetch_labels(), fresh.fetch_labels())
        np.testing.assert_array_equal(r.fetch_box_sets()[0], fresh.fetch_box_sets()[0])
        np.testing.assert_array_equal(r.fetch_box_sets()[1], fresh.fetch_box_sets()[1])
        # the same updates as requests in one classify
        hs = [req.update_request(up.ids, f32(up.poses)) for up in ups]
        req.classify()
        for h, w in zip(hs, want_each):
            np.testing.assert_array_equal(req.fetch_request_labels(h), w)
        # gray resolution on this geometry's touch sets
        lazy = r.fetch_labels()
        res, clear, stats = r.resolve_gray(2)
        assert stats["gray_edges"] == int((lazy == rgg.GRAY).sum())
        for e in np.flatnonzero(lazy == rgg.GRAY)[:30]:
            v, _ = oracle.edge_dense_clearance(robot, rm.q_from[e], rm.q_to[e], rm.step, 2,
                                               final.poses())
            if res[e] == rgg.RED:
                assert v < 0
            elif res[e] == rgg.GREEN:
                assert v > 0


def test_sphere_only_calls_are_refused(rgg, tmp_path):
    rm, boxes, _ = scene(0)
    with obb_roadmap(rgg, rm, boxes.count) as r:
        r.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
        r.classify()
        for call in (lambda: r.fetch_records(), lambda: r.save(str(tmp_path / "x.rgg")),
                     lambda: rgg.autotune([r]),
                     lambda: r.upload_edges(np.array([0, 2], np.uint64),
                                            np.zeros((4, 24), np.float32),
                                            np.zeros((4, 3), np.float32))):
            with pytest.raises(rgg.RGGError) as e:
                call()
            assert e.value.status == rgg.RGG_ERR_STATE
    with rgg.Roadmap(3, 4, 4) as s:
        with pytest.raises(rgg.RGGError) as e:
            s.set_obb_filter(False)
        assert e.value.status == rgg.RGG_ERR_STATE


def test_obb_edge_cases(rgg):
    """An empty roadmap; a single resting edge (every spline one segment);
    a box that is never placed (absent: affects nothing)."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    with rgg.Roadmap(1, 4, 3, geometry=rgg.GEOMETRY_OBB) as r:
        r.build_edges(robot, np.zeros((0, 1)), np.zeros((0, 1)), 0.05)
        r.update_obstacles([0], f32([[0.15, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.05, 0.05, 0.05]]))
        r.classify()
        assert r.fetch_labels().shape == (0,)
        r.check_status()
    boxes = np.array([[0.15, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.05, 0.05, 0.05],
                      [0.15, 0.5, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.05, 0.05, 0.05],
                      [0.15, 0.07, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.05, 0.05, 0.05]])
    with rgg.Roadmap(1, 4, 4, geometry=rgg.GEOMETRY_OBB) as r:
        r.build_edges(robot, np.zeros((1, 1)), np.zeros((1, 1)), 0.05)
        obb, off, verts = r.fetch_obb_records()
        assert np.all(np.diff(off.astype(np.int64)) == 2)      # one segment per spline
        for b, want in ((0, rgg.RED), (1, rgg.GREEN), (2, rgg.GRAY)):
            r.update_obstacles([b], f32(boxes[b:b + 1]))
            r.classify()
            got = r.fetch_labels()[0]
            ref = oracle.classify_obb(robot, [[0.0]], [[0.0]], 0.05, boxes[b:b + 1])["labels"][0]
            assert got == ref == want, (b, got, ref)
            # move it far away again before the next case
            far = boxes[b:b + 1].copy()
            far[0, :3] = [40.0 + b, 40.0, 0.0]
            r.update_obstacles([b], f32(far))
            r.classify()
            assert r.fetch_labels()[0] == rgg.GREEN
        r.check_status()
