"""The sphere geometry's spatial filter (Sec. 4.3, spatially filtered
many-to-many checking, applied to the streamed records): every round of 31
configurations of a tile has a bounding sphere of its outer spheres; before
each pass the rounds are tested against the moved boxes and the classify
kernel copies only the rounds some box may reach.

Rules checked:
  * labels and per-edge hit / touch sets are bit-identical with and without
    the filter after every update: planar and 7-DOF scenes, every launch
    shape, a batched launch mixing filtered and unfiltered roadmaps,
    uploaded records, a reloaded roadmap;
  * the filtered launches copy fewer record bytes than record_bytes per
    pass, and none for a pass whose boxes are far from every edge
    (unfiltered launches copy every record and are not counted);
  * a batched launch whose filtered roadmaps list no tile (their moved
    boxes far from every edge), in the middle, at the ends or all of them,
    leaves the same state as unfiltered launches;
  * the filtered labels agree with the FP64 oracle (pinned edges equal,
    other differences GPU gray);
  * a roadmap below 262,144 tiles stays on variant 10 on a dense scene, with
    the labels and box sets of a roadmap fixed to it (the switch to variant
    12 on dense passes of larger roadmaps is checked on the full-size
    roadmap, tests/test_gpu_fullsize.py).
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
    if which == "planar":
        sc = W.workload_planar(n_nodes=300, n_updates=4)
        return sc.roadmap, sc.boxes, sc.updates
    rng = np.random.default_rng(61)
    arm = W.dh_arm(rng, 7)
    rm = W.prm_roadmap(rng, arm, 200, 10, 0.03)
    boxes = W.random_boxes(rng, 24)
    return rm, boxes, W.update_stream(rng, boxes, 4, 4)


def built(rgg, rm, m, filtered, fmt=0):
    r = rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, m, record_format=fmt)
    r.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
    r.set_round_filter(filtered)
    return r


def same_state(a, b, where):
    np.testing.assert_array_equal(a.fetch_labels(), b.fetch_labels(), err_msg=where)
    ha, ta = a.fetch_box_sets()
    hb, tb = b.fetch_box_sets()
    np.testing.assert_array_equal(ha, hb, err_msg=where)
    np.testing.assert_array_equal(ta, tb, err_msg=where)


@pytest.mark.parametrize("which", ["planar", "7dof"])
def test_filter_changes_no_bit(rgg, which):
    rm, boxes, ups = scene(which)
    m = boxes.count
    state = boxes.copy()
    with built(rgg, rm, m, True) as f, built(rgg, rm, m, False) as u:
        assert f.info()["round_filter"] == 1 and u.info()["round_filter"] == 0
        with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, m) as d:
            assert d.info()["round_filter"] == 0          # off by default
        record_bytes = u.info()["record_bytes"]
        for x in (f, u):
            x.update_obstacles(np.arange(m), f32(state.poses()))
            x.classify()
        same_state(f, u, "initial")
        f.streamed_bytes()
        u.streamed_bytes()
        for k, up in enumerate(ups):
            for x in (f, u):
                x.update_obstacles(up.ids, f32(up.poses))
                x.classify()
            state.centre[up.ids] = up.poses[:, :3]
            same_state(f, u, f"update {k}")
            bf, bu = f.streamed_bytes(), u.streamed_bytes()
            assert bu == 0
            assert bf < record_bytes, (bf, record_bytes)
        want = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, state.poses())
        got = f.fetch_labels()
        pinned = want["kappa"] > PIN
        assert np.all(got[pinned] == want["labels"][pinned])
        assert np.all(got[got != want["labels"]] == oracle.GRAY)
        f.check_status()
        u.check_status()


@pytest.mark.parametrize("fmt", [0, 1], ids=["link_ends", "spheres"])
def test_every_launch_shape(rgg, fmt):
    """The filter runs with the two default launch shapes only (variants 5
    and 7); the round data follow the tiles when a launch shape changes them
    (3 -> 5 rebuilds both).  Every shape gives the same bits, for either
    record format."""
    rm, boxes, ups = scene("7dof")
    m = boxes.count
    with built(rgg, rm, m, False, fmt) as u:
        u.update_obstacles(np.arange(m), f32(boxes.poses()))
        u.classify()
        for up in ups:
            u.update_obstacles(up.ids, f32(up.poses))
            u.classify()
        want_l = u.fetch_labels()
        want_h, want_t = u.fetch_box_sets()
    for variant in list(range(rgg.NUM_VARIANTS)) + ["3->5"]:
        with built(rgg, rm, m, True, fmt) as f:
            if variant == "3->5":
                f.set_launch_shape(3, 16)
                assert f.info()["round_filter"] == 0
                f.set_launch_shape(5, 16)
                assert f.info()["round_filter"] == 1
            else:
                f.set_launch_shape(variant, 16)
                assert f.info()["round_filter"] == (1 if variant in (5, 7, 10, 11, 12) else 0)
            f.update_obstacles(np.arange(m), f32(boxes.poses()))
            f.classify()
            for up in ups:
                f.update_obstacles(up.ids, f32(up.poses))
                f.classify()
            np.testing.assert_array_equal(f.fetch_labels(), want_l, err_msg=f"variant {variant}")
            h, t = f.fetch_box_sets()
            np.testing.assert_array_equal(h, want_h, err_msg=f"variant {variant}")
            np.testing.assert_array_equal(t, want_t, err_msg=f"variant {variant}")
            f.check_status()


def test_batched_mix_of_filtered_and_unfiltered(rgg):
    scenes = W.workload_batched(n_roadmaps=6, edge_lo=300, edge_hi=3000, n_updates=2)
    mixed, plain = [], []
    for i, sc in enumerate(scenes):
        for lst, flt in ((mixed, i % 2 == 0), (plain, False)):
            r = built(rgg, sc.roadmap, sc.boxes.count, flt)
            r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
            lst.append(r)
    rgg.classify_many(mixed)
    for r in plain:
        r.classify()
    for k in range(2):
        for sc, a, b in zip(scenes, mixed, plain):
            up = sc.updates[k]
            a.update_obstacles(up.ids, f32(up.poses))
            b.update_obstacles(up.ids, f32(up.poses))
        rgg.classify_many(mixed)
        for b in plain:
            b.classify()
        for i, (a, b) in enumerate(zip(mixed, plain)):
            same_state(a, b, f"roadmap {i} step {k}")
    for r in mixed + plain:
        r.check_status()
        r.close()


def test_uploaded_and_reloaded_roadmaps(rgg, tmp_path):
    rm, boxes, ups = scene("7dof")
    m = boxes.count
    robot = rm.robot
    # sphere records, so that the uploaded copy makes the same decisions
    with built(rgg, rm, m, False, 1) as u:
        inner, outer, soff = u.fetch_records()
        u.update_obstacles(np.arange(m), f32(boxes.poses()))
        u.classify()
        path = str(tmp_path / "r.rgg")
        u.save(path)
        with rgg.Roadmap(robot.num_links, robot.inner_per_link, m) as up_r, \
                rgg.Roadmap(robot.num_links, robot.inner_per_link, m) as ld:
            # switched on before the records arrive: computed when they do
            up_r.set_round_filter(True)
            ld.set_round_filter(True)
            up_r.upload_edges(soff, inner, outer)
            up_r.update_obstacles(np.arange(m), f32(boxes.poses()))
            up_r.classify()
            ld.load(path)
            assert up_r.info()["round_filter"] == 1 and ld.info()["round_filter"] == 1
            for k, mv in enumerate(ups):
                for x in (u, up_r, ld):
                    x.update_obstacles(mv.ids, f32(mv.poses))
                    x.classify()
                same_state(up_r, u, f"uploaded, update {k}")
                same_state(ld, u, f"reloaded, update {k}")
            up_r.check_status()
            ld.check_status()


def test_far_boxes_copy_nothing_and_clear_their_bits(rgg):
    rm, boxes, _ = scene("planar")
    m = boxes.count
    state = boxes.copy()
    with built(rgg, rm, m, True) as f, built(rgg, rm, m, False) as u:
        for x in (f, u):
            x.update_obstacles(np.arange(m), f32(state.poses()))
            x.classify()
        f.streamed_bytes()
        _, touch0 = f.fetch_box_sets()
        # the three boxes that touch the most edges move far away
        per_box = np.array([np.count_nonzero((touch0[:, b >> 5] >> (b & 31)) & 1) for b in range(m)])
        ids = np.sort(np.argsort(-per_box, kind="stable")[:3])
        assert per_box[ids].min() > 0
        mask = np.uint32(sum(1 << int(b) for b in ids))
        far = state.poses()[ids].copy()
        far[:, :3] = [[60.0, 60.0, 0.0], [61.0, 60.0, 0.0], [62.0, 60.0, 0.0]]
        for x in (f, u):
            x.update_obstacles(ids, f32(far))
            x.classify()
        state.centre[ids] = far[:, :3]
        assert f.streamed_bytes() == 0
        same_state(f, u, "far boxes")
        _, touch1 = f.fetch_box_sets()
        assert not np.any(touch1[:, 0] & mask)
        want = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, state.poses())
        got = f.fetch_labels()
        pinned = want["kappa"] > PIN
        assert np.all(got[pinned] == want["labels"][pinned])
        # switching the filter is refused for the OBB geometry only
        with rgg.Roadmap(3, 4, 4, geometry=rgg.GEOMETRY_OBB) as o:
            with pytest.raises(rgg.RGGError) as e:
                o.set_round_filter(False)
            assert e.value.status == rgg.RGG_ERR_STATE


def test_batched_launch_with_empty_tile_lists(rgg):
    # A batched launch numbers the filtered roadmaps' listed tiles one roadmap
    # after another; roadmaps whose moved boxes reach no tile (empty lists) in
    # the middle, at both ends, and a launch where every list is empty must
    # leave the same state as unfiltered launches of each roadmap alone.
    scenes = W.workload_batched(n_roadmaps=5, edge_lo=300, edge_hi=3000, n_updates=1)
    filt, plain = [], []
    for sc in scenes:
        for lst, flt in ((filt, True), (plain, False)):
            r = built(rgg, sc.roadmap, sc.boxes.count, flt)
            r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
            lst.append(r)
    rgg.classify_many(filt)
    for r in plain:
        r.classify()

    def far_move(sc, k):
        ids = np.arange(min(2, sc.boxes.count), dtype=np.uint32)
        poses = f32(sc.boxes.poses()[ids])
        poses[:, :3] = [[80.0 + k, 80.0, 0.0], [80.0 + k, 82.0, 0.0]][:len(ids)]
        return ids, poses

    for step in range(2):
        for i, (sc, a, b) in enumerate(zip(scenes, filt, plain)):
            if step == 1 or i % 2 == 0:
                ids, poses = far_move(sc, i)
            else:
                ids, poses = sc.updates[0].ids, f32(sc.updates[0].poses)
            a.update_obstacles(ids, poses)
            b.update_obstacles(ids, poses)
        for r in filt:
            r.streamed_bytes()             # restart the copied-byte counters
        rgg.classify_many(filt)
        for b in plain:
            b.classify()
        for i, (a, b) in enumerate(zip(filt, plain)):
            same_state(a, b, f"roadmap {i} step {step}")
        if step == 1:
            # every moved box is far away: no tile listed, no record copied
            assert sum(r.streamed_bytes() for r in filt) == 0
    for r in filt + plain:
        r.check_status()
        r.close()


def test_small_roadmaps_keep_the_default_shape_on_dense_passes(rgg):
    dense = True
    rng = np.random.default_rng(67)
    rm = W.prm_roadmap(rng, W.seven_dof_arm(), 400, 10, 0.02)
    # dense: 32 large boxes about the arm, so that nearly every tile is listed;
    # sparse: small boxes spread over a large cube, so that few are
    boxes = (W.random_boxes(rng, 32, extent=0.8, half_lo=0.35, half_hi=0.5) if dense
             else W.random_boxes(rng, 32, extent=3.0, half_lo=0.02, half_hi=0.04))
    ups = W.update_stream(rng, boxes, 3, 32)
    m = boxes.count
    with rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, m) as a, \
            rgg.Roadmap(rm.robot.num_links, rm.robot.inner_per_link, m) as b:
        a.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        b.build_edges(rm.robot, rm.q_from, rm.q_to, rm.step)
        b.set_launch_shape(10, 27)
        assert a.info()["variant"] == 10 and a.info()["round_filter"] == 1
        for r in (a, b):
            r.update_obstacles(np.arange(m), f32(boxes.poses()))
            r.classify()
            r.fetch_labels()  # the pass has run: the next one reads its count
        seen = set()
        for up in ups:
            for r in (a, b):
                r.update_obstacles(up.ids, f32(up.poses))
                r.classify()
            seen.add(a.info()["last_variant"])
            assert b.info()["last_variant"] == 10
            assert np.array_equal(a.fetch_labels(), b.fetch_labels())
            ha, ta = a.fetch_box_sets()
            hb, tb = b.fetch_box_sets()
            assert np.array_equal(ha, hb) and np.array_equal(ta, tb)
        assert seen == {10}
