"""rgg_save / rgg_load on the GPU: a saved and reloaded roadmap holds the
same records, box sets, labels and boxes, and classifies later updates
exactly as the original does (and within the oracle rule)."""
import os

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


def scene():
    return W.workload_7dof(n_nodes=800, n_boxes=40, n_updates=4)


def prepared(rgg, sc, n_updates=2, fmt=0):
    rm, robot = sc.roadmap, sc.roadmap.robot
    r = rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count, record_format=fmt)
    r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
    r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
    r.classify()
    for up in sc.updates[:n_updates]:
        r.update_obstacles(up.ids, f32(up.poses))
        r.classify()
    return r


def same_roadmap(a, b):
    ia, oa, sa = a.fetch_records()
    ib, ob, sb = b.fetch_records()
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(a.fetch_labels(), b.fetch_labels())
    ha, ta = a.fetch_box_sets()
    hb, tb = b.fetch_box_sets()
    np.testing.assert_array_equal(ha, hb)
    np.testing.assert_array_equal(ta, tb)


@pytest.mark.parametrize("fmt", [0, 1], ids=["link_ends", "spheres"])
def test_save_load_round_trip_and_later_updates(rgg, tmp_path, fmt):
    """Either record format reloads bit for bit, into a roadmap created with
    either format (the file's format wins)."""
    sc = scene()
    rm, robot = sc.roadmap, sc.roadmap.robot
    path = str(tmp_path / "roadmap.rgg")
    with prepared(rgg, sc, fmt=fmt) as a, rgg.Roadmap(robot.num_links, robot.inner_per_link,
                                                      sc.boxes.count, record_format=1 - fmt) as b:
        a.save(path)
        b.load(path)
        assert b.info()["num_edges"] == a.info()["num_edges"]
        assert b.info()["record_format"] == fmt
        assert b.info()["record_bytes"] == a.info()["record_bytes"]
        assert b.info()["pending_boxes"] == 0
        same_roadmap(a, b)
        # the reloaded roadmap continues exactly like the original
        boxes = sc.boxes.copy()
        for up in sc.updates[:4]:
            boxes.centre[up.ids] = up.poses[:, :3]
        for up in sc.updates[2:4]:
            for x in (a, b):
                x.update_obstacles(up.ids, f32(up.poses))
                x.classify()
        same_roadmap(a, b)
        want = oracle.classify(robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
        got = b.fetch_labels()
        pinned = want["kappa"] > PIN
        assert np.all(got[pinned] == want["labels"][pinned])
        assert np.all(got[got != want["labels"]] == oracle.GRAY)
        # loading over existing edges replaces them
        b.load(path)
        assert b.info()["pending_boxes"] == 0


def test_load_rejects_other_shapes_and_damaged_files(rgg, tmp_path):
    sc = scene()
    robot = sc.roadmap.robot
    path = str(tmp_path / "roadmap.rgg")
    with prepared(rgg, sc) as a:
        a.save(path)
        before = a.fetch_labels()
        size = os.path.getsize(path)
        # another robot shape or box count
        for L, K, M in ((robot.num_links, robot.inner_per_link + 1, sc.boxes.count),
                        (robot.num_links, robot.inner_per_link, sc.boxes.count + 40)):
            with rgg.Roadmap(L, K, M) as c:
                with pytest.raises(rgg.RGGError) as e:
                    c.load(path)
                assert e.value.status == rgg.RGG_ERR_INVALID
        # one flipped byte inside the records, and a truncated copy
        bad = str(tmp_path / "bad.rgg")
        data = bytearray(open(path, "rb").read())
        data[size // 2] ^= 0x40
        open(bad, "wb").write(bytes(data))
        short = str(tmp_path / "short.rgg")
        open(short, "wb").write(bytes(data[: size - 100]))
        for p, status in ((bad, rgg.RGG_ERR_INVALID), (short, rgg.RGG_ERR_INVALID),
                          (str(tmp_path / "missing.rgg"), rgg.RGG_ERR_IO)):
            with pytest.raises(rgg.RGGError) as e:
                a.load(p)
            assert e.value.status == status, p
        # a failed load leaves the roadmap as it was
        np.testing.assert_array_equal(a.fetch_labels(), before)
        a.check_status()


def test_save_needs_edges_and_no_pending_moves(rgg, tmp_path):
    sc = scene()
    robot = sc.roadmap.robot
    path = str(tmp_path / "x.rgg")
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count) as e0:
        with pytest.raises(rgg.RGGError) as e:
            e0.save(path)
        assert e.value.status == rgg.RGG_ERR_STATE
    with prepared(rgg, sc, n_updates=0) as a:
        up = sc.updates[0]
        a.update_obstacles(up.ids, f32(up.poses))
        with pytest.raises(rgg.RGGError) as e:
            a.save(path)
        assert e.value.status == rgg.RGG_ERR_STATE
        a.classify()
        a.save(path)
        assert os.path.getsize(path) > a.info()["record_bytes"]
