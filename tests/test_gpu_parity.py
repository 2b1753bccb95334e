"""GPU path (through the C ABI) against the FP64 CPU oracle.

Rules, for every comparison:
  * sample counts and offsets: bit-exact;
  * sphere records: within one FP32 rounding of the oracle's FP64 spheres,
    inner radii rounded down and outer radii rounded up;
  * labels: identical on every edge whose oracle clearance kappa exceeds
    1e-4 m; any other disagreement must be GPU = GRAY (never red <-> green),
    and is counted;
  * per-box sets: GPU hit set within the oracle's hit set, the oracle's
    touch set within the GPU touch set (the margin delta only ever moves a
    decision toward gray).
"""
import numpy as np
import pytest

import oracle
from paper_2603_28674_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PIN = 1e-4
MARGIN = 2e-5


@pytest.fixture(scope="module")
def rgg():
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg as _rgg
    return _rgg


def make_roadmap(rgg, rm, n_boxes, margin=MARGIN, record_format=0):
    robot = rm.robot
    r = rgg.Roadmap(robot.num_links, robot.inner_per_link, n_boxes, margin,
                    record_format=record_format)
    r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
    return r


# built roadmaps store link ends (the default) or every inner sphere
FORMATS = pytest.mark.parametrize("fmt", [0, 1], ids=["link_ends", "spheres"])


def f32(poses):
    return np.asarray(poses, dtype=np.float32)


def check_labels(got, want, where=""):
    lab = want["labels"]
    pinned = want["kappa"] > PIN
    bad = np.flatnonzero(pinned & (got != lab))
    assert bad.size == 0, f"{where}: {bad.size} pinned edges differ, first {bad[:5]}"
    off = got != lab
    assert np.all(got[off] == oracle.GRAY), f"{where}: disagreement other than GPU gray"
    return int(off.sum())


def check_sets(hit, touch, want):
    w = want["hit"].shape[1]
    assert np.all((hit[:, :w] & ~want["hit"]) == 0), "GPU hit outside the oracle's hit set"
    assert np.all((want["touch"] & ~touch[:, :w]) == 0), "oracle touch missing from GPU"
    assert np.all((hit & ~touch) == 0), "hit without touch"


# --------------------------------------------------------------------------
# records (a0)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["planar", "7dof"])
@FORMATS
def test_records_match_oracle_spheres(rgg, which, fmt):
    """Sample counts are exact; the records stand for the oracle's spheres
    within FP32 rounding: sphere records are the FP64 spheres rounded once;
    link-end records keep each link end rounded once, so the centres read
    back (interpolated in FP64 and rounded again) carry up to two end
    roundings at |coordinate| <= 2 m besides their own."""
    if which == "planar":
        sc = W.workload_planar(n_updates=0)
    else:
        sc = W.workload_7dof(n_nodes=400, n_updates=0)
    rm = sc.roadmap
    robot = rm.robot
    L, K = robot.num_links, robot.inner_per_link
    with make_roadmap(rgg, rm, sc.boxes.count, record_format=fmt) as r:
        inner, outer, soff = r.fetch_records()
        info = r.info()
    assert info["record_format"] == fmt
    per_g = 12 if fmt == 0 else 16 * K
    assert info["record_bytes"] == per_g * L * int(soff[-1]) + 16 * L * (int(soff[-1]) - rm.num_edges)
    n_e = np.diff(soff.astype(np.int64))
    want_n = np.array([oracle.num_samples(rm.q_from[e], rm.q_to[e], rm.step)
                       for e in range(rm.num_edges)])
    np.testing.assert_array_equal(n_e, want_n)
    sel = np.random.default_rng(0).choice(rm.num_edges, size=min(150, rm.num_edges),
                                          replace=False)
    for e in sel:
        n = int(n_e[e])
        s0 = int(soff[e])
        oi, oo = oracle.edge_spheres(robot, rm.q_from[e], rm.q_to[e], rm.step)
        # GPU layout: inner (link, sample, sphere); outer (link, interval)
        gi = inner[:, K * L * s0: K * L * (s0 + n)].reshape(4, L, n, K)
        go = outer[:, L * (s0 - e): L * (s0 - e + n - 1)].reshape(4, L, n - 1)
        wi = oi.transpose(3, 1, 0, 2)            # [4, L, n, K]
        wo = oo.transpose(2, 1, 0)               # [4, L, n-1]
        tol_i = 1.2e-7 * np.abs(wi[:3]) + (1e-12 if fmt == 1 else 2.4e-7)
        tol_o = 1.2e-7 * np.abs(wo[:3]) + 1e-12
        assert np.all(np.abs(gi[:3] - wi[:3]) <= tol_i)
        assert np.all(np.abs(go[:3] - wo[:3]) <= tol_o)
        assert np.all(gi[3] <= wi[3]) and np.all(gi[3] >= wi[3] * (1 - 2.4e-7))
        assert np.all(go[3] >= wo[3] * (1 - 1e-13)) and np.all(go[3] <= wo[3] * (1 + 2.4e-7))


# --------------------------------------------------------------------------
# labels (a1..a6)
# --------------------------------------------------------------------------
def run_updates(rgg, sc, n_updates=None, check_every=True, fmt=0):
    """Place every box, classify, then apply the update stream; compare with
    the oracle from scratch after each step.  Returns the roadmap handle."""
    rm, robot = sc.roadmap, sc.roadmap.robot
    boxes = sc.boxes.copy()
    r = make_roadmap(rgg, rm, boxes.count, record_format=fmt)
    r.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
    r.classify()
    ups = sc.updates if n_updates is None else sc.updates[:n_updates]
    steps = [None] + list(ups)
    stats = []
    for i, up in enumerate(steps):
        if up is not None:
            r.update_obstacles(up.ids, f32(up.poses))
            r.classify()
            boxes.centre[up.ids] = up.poses[:, :3]
        if check_every or i == len(steps) - 1:
            got = r.fetch_labels()
            want = oracle.classify(robot, rm.q_from, rm.q_to, rm.step, boxes.poses(), bits=True)
            stats.append(check_labels(got, want, f"step {i}"))
            hit, touch = r.fetch_box_sets()
            check_sets(hit, touch, want)
    r.check_status()
    return r, boxes, stats


@FORMATS
def test_planar_update_stream(rgg, fmt):
    sc = W.workload_planar(n_updates=8)
    r, _, stats = run_updates(rgg, sc, fmt=fmt)
    info = r.info()
    assert info["num_tiles"] > 4
    r.close()
    assert max(stats) <= 0.01 * sc.roadmap.num_edges


@FORMATS
def test_7dof_update_stream_two_passes(rgg, fmt):
    """64 boxes: the first classification runs two 32-box passes and uses
    the second mask word."""
    sc = W.workload_7dof(n_nodes=1200, n_updates=4)
    r, _, stats = run_updates(rgg, sc, fmt=fmt)
    assert r.info()["mask_words"] == 2
    r.close()


def test_incremental_equals_from_scratch(rgg):
    """After an update stream, the incremental state equals a fresh roadmap
    that classifies every box at its final pose in one go (bit-exact)."""
    sc = W.workload_7dof(n_nodes=600, n_boxes=40, n_updates=6)
    r, boxes, _ = run_updates(rgg, sc, check_every=False)
    with make_roadmap(rgg, sc.roadmap, boxes.count) as fresh:
        fresh.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
        fresh.classify()
        np.testing.assert_array_equal(r.fetch_labels(), fresh.fetch_labels())
        h1, t1 = r.fetch_box_sets()
        h2, t2 = fresh.fetch_box_sets()
        np.testing.assert_array_equal(h1, h2)
        np.testing.assert_array_equal(t1, t2)
    r.close()


@FORMATS
def test_long_edges_span_tiles(rgg, fmt):
    """Edges with ~1500 configurations per link run across several streaming
    tiles (halo intervals, link-end halos reaching one link's run back, and
    cross-tile merges)."""
    rng = np.random.default_rng(3)
    robot = W.planar_arm()
    qa = rng.uniform(-np.pi, np.pi, (60, 3))
    qb = qa + rng.uniform(-3.0, 3.0, (60, 3))
    rm = W.Roadmap(robot, qa, qb, 0.002)
    boxes = W.random_boxes(rng, 12, planar=True, oriented=False, half_hi=0.08)
    with make_roadmap(rgg, rm, boxes.count, record_format=fmt) as r:
        info = r.info()
        assert info["num_samples"] / rm.num_edges > info["tile_samples"]
        r.update_obstacles(np.arange(boxes.count), f32(boxes.poses()))
        r.classify()
        got = r.fetch_labels()
        hit, touch = r.fetch_box_sets()
    want = oracle.classify(robot, qa, qb, rm.step, boxes.poses(), bits=True)
    check_labels(got, want, "long edges")
    check_sets(hit, touch, want)
    assert len(set(got.tolist())) >= 2


def test_edge_cases(rgg):
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    box = np.array([[0.2, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.05, 0.05, 0.05]], np.float32)
    # empty roadmap
    with rgg.Roadmap(1, 4, 8) as r:
        r.build_edges(robot, np.zeros((0, 1)), np.zeros((0, 1)), 0.05)
        r.update_obstacles([3], box)
        r.classify()
        assert r.fetch_labels().shape == (0,)
    # classify before edges
    with rgg.Roadmap(1, 4, 8) as r:
        with pytest.raises(rgg.RGGError):
            r.classify()
    # zero-motion edges (two identical configurations), box never placed,
    # ids above 32, nothing pending
    with rgg.Roadmap(1, 4, 70) as r:
        r.build_edges(robot, np.zeros((3, 1)), np.zeros((3, 1)), 0.05)
        assert r.info()["num_samples"] == 6
        r.classify()  # nothing pending: no launch
        assert np.all(r.fetch_labels() == rgg.GREEN)
        r.update_obstacles([65], box)
        r.classify()
        assert np.all(r.fetch_labels() == rgg.RED)
        hit, touch = r.fetch_box_sets()
        assert np.all(hit[:, 2] == 1 << 1) and np.all(hit[:, :2] == 0)
        far = box.copy()
        far[0, 1] = 5.0
        r.update_obstacles([65], far)
        r.classify()
        assert np.all(r.fetch_labels() == rgg.GREEN)
        hit, touch = r.fetch_box_sets()
        assert not hit.any() and not touch.any()
    # bad input is rejected and changes nothing
    with rgg.Roadmap(1, 4, 8) as r:
        r.build_edges(robot, np.zeros((2, 1)), np.ones((2, 1)), 0.05)
        with pytest.raises(rgg.RGGError):
            r.update_obstacles([8], box)                      # id out of range
        skew = box.copy()
        skew[0, 3] = 2.0                                      # not a rotation
        with pytest.raises(rgg.RGGError):
            r.update_obstacles([0], skew)
        with pytest.raises(rgg.RGGError):
            r.update_obstacles([1, 1], np.repeat(box, 2, 0))  # repeated id
        assert r.info()["pending_boxes"] == 0
        with pytest.raises(rgg.RGGError):
            r.upload_edges(np.array([0, 1], np.uint64), np.zeros((4, 4), np.float32),
                           np.zeros((4, 0), np.float32))      # an edge with one sample
        with pytest.raises(rgg.RGGError):
            r.fetch_labels(1, 5)


def test_many_boxes_in_one_update(rgg):
    """70 boxes moved at once: three passes of up to 32 boxes."""
    sc = W.workload_7dof(n_nodes=300, n_boxes=70, n_updates=0)
    rm = sc.roadmap
    with make_roadmap(rgg, rm, 70) as r:
        r.update_obstacles(np.arange(70), f32(sc.boxes.poses()))
        assert r.info()["pending_boxes"] == 70
        r.classify()
        got = r.fetch_labels()
        hit, touch = r.fetch_box_sets()
    want = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, sc.boxes.poses(), bits=True)
    check_labels(got, want, "70 boxes")
    check_sets(hit, touch, want)


def test_upload_of_fetched_records_and_device_poses(rgg):
    """Sphere records uploaded by the caller (host and device) classify the
    same as the sphere records built in place; device-side poses equal host
    poses."""
    import torch
    sc = W.workload_planar(n_nodes=200, n_updates=1)
    rm, robot = sc.roadmap, sc.roadmap.robot
    poses = f32(sc.boxes.poses())
    ids = np.arange(sc.boxes.count)
    with make_roadmap(rgg, rm, sc.boxes.count, record_format=1) as a:
        inner, outer, soff = a.fetch_records()
        a.update_obstacles(ids, poses)
        a.classify()
        want = a.fetch_labels()
        with rgg.Roadmap(3, 4, sc.boxes.count) as b:
            b.upload_edges(soff, inner, outer)
            b.update_obstacles(ids, torch.from_numpy(poses).cuda())
            b.classify()
            np.testing.assert_array_equal(b.fetch_labels(), want)
        with rgg.Roadmap(3, 4, sc.boxes.count) as c:
            c.update_obstacles(ids, poses)          # placed before the edges exist
            c.upload_edges(soff, torch.from_numpy(inner).cuda(), torch.from_numpy(outer).cuda())
            assert c.info()["pending_boxes"] == sc.boxes.count
            c.classify()
            out = torch.empty(rm.num_edges, dtype=torch.uint8, device="cuda")
            c.fetch_labels(out=out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_batched_equals_alone(rgg):
    """classify_many over roadmaps with different robots, sizes and update
    sizes gives exactly the labels and sets of classifying each alone."""
    scenes = W.workload_batched(n_roadmaps=6, edge_lo=200, edge_hi=3000, n_updates=2)
    alone, together = [], []
    for sc in scenes:
        for group in (alone, together):
            r = make_roadmap(rgg, sc.roadmap, sc.boxes.count)
            r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
            group.append(r)
    for r in alone:
        r.classify()
    rgg.classify_many(together)
    for step in range(2):
        for sc, a, t in zip(scenes, alone, together):
            up = sc.updates[step]
            a.update_obstacles(up.ids, f32(up.poses))
            t.update_obstacles(up.ids, f32(up.poses))
            a.classify()
        rgg.classify_many(together)
    for sc, a, t in zip(scenes, alone, together):
        np.testing.assert_array_equal(a.fetch_labels(), t.fetch_labels())
        ha, ta = a.fetch_box_sets()
        ht, tt = t.fetch_box_sets()
        np.testing.assert_array_equal(ha, ht)
        np.testing.assert_array_equal(ta, tt)
    # and against the oracle on one of them
    sc, t = scenes[0], together[0]
    boxes = sc.boxes.copy()
    for up in sc.updates[:2]:
        boxes.centre[up.ids] = up.poses[:, :3]
    rm = sc.roadmap
    want = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
    check_labels(t.fetch_labels(), want, "batched")
    for r in alone + together:
        r.close()


def test_batched_launch_of_both_record_formats(rgg):
    """One launch runs every roadmap at the first roadmap's shape: a sphere-
    record roadmap first (69 KB stages) also runs link-end tiles, with the
    labels of classifying each alone; link-end first (27 KB stages) cannot
    hold sphere tiles and is refused before anything runs."""
    sc = W.workload_7dof(n_nodes=300, n_boxes=20, n_updates=1)
    rm = sc.roadmap
    rs = [make_roadmap(rgg, rm, 20, record_format=f) for f in (1, 0)]
    alone = [make_roadmap(rgg, rm, 20, record_format=f) for f in (1, 0)]
    for r in rs + alone:
        r.update_obstacles(np.arange(20), f32(sc.boxes.poses()))
    with pytest.raises(rgg.RGGError) as e:
        rgg.classify_many(rs[::-1])
    assert e.value.status == rgg.RGG_ERR_INVALID
    assert all(r.info()["pending_boxes"] == 20 for r in rs)
    rgg.classify_many(rs)
    for r in alone:
        r.classify()
    for a, b in zip(rs, alone):
        np.testing.assert_array_equal(a.fetch_labels(), b.fetch_labels())
        ha, ta = a.fetch_box_sets()
        hb, tb = b.fetch_box_sets()
        np.testing.assert_array_equal(ha, hb)
        np.testing.assert_array_equal(ta, tb)
    for r in rs + alone:
        r.check_status()
        r.close()


def test_kernel_timing_counts_launches(rgg):
    sc = W.workload_planar(n_nodes=100, n_updates=1)
    with make_roadmap(rgg, sc.roadmap, sc.boxes.count) as r:
        r.set_kernel_timing(True)
        r.update_obstacles(np.arange(16), f32(sc.boxes.poses()))
        r.classify()
        ms, mm, n = r.kernel_time()
        assert n == 1 and ms > 0 and mm > 0


def test_interpolated_and_per_sphere_inner_tests(rgg):
    """Records built in place take the interpolated inner test; the same
    records uploaded from device memory are not inspected and take the
    per-sphere test.  Both meet the oracle rule, and they differ only on
    unpinned edges."""
    import torch
    sc = W.workload_7dof(n_nodes=600, n_updates=3)
    rm, robot = sc.roadmap, sc.roadmap.robot
    boxes = sc.boxes.copy()
    ids = np.arange(boxes.count)
    with make_roadmap(rgg, rm, boxes.count) as a:
        inner, outer, soff = a.fetch_records()
        with rgg.Roadmap(robot.num_links, robot.inner_per_link, boxes.count) as b:
            b.upload_edges(soff, torch.from_numpy(inner).cuda(), torch.from_numpy(outer).cuda())
            for x in (a, b):
                x.update_obstacles(ids, f32(boxes.poses()))
                x.classify()
            for up in sc.updates:
                boxes.centre[up.ids] = up.poses[:, :3]
                for x in (a, b):
                    x.update_obstacles(up.ids, f32(up.poses))
                    x.classify()
                want = oracle.classify(robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
                la, lb = a.fetch_labels(), b.fetch_labels()
                check_labels(la, want, "interpolated")
                check_labels(lb, want, "per-sphere")
                assert np.all(want["kappa"][la != lb] <= PIN)


def test_irregular_uploads_take_the_exact_sphere_test(rgg):
    """Host-uploaded records whose inner spheres are not equally spaced with
    one radius are classified sphere by sphere: a third of the samples get a
    second sphere of radius 0.1 m next to the link's midpoint (still inside
    the interval's outer spheres), and the labels follow the oracle on those
    exact sphere sets."""
    sc = W.workload_planar(n_nodes=200, n_updates=0)
    rm, robot = sc.roadmap, sc.roadmap.robot
    L, K = robot.num_links, robot.inner_per_link
    n_boxes = 4
    poses = sc.boxes.poses()[:n_boxes]
    with make_roadmap(rgg, rm, n_boxes) as a:
        inner, outer, soff = a.fetch_records()
    soff = soff.astype(np.int64)
    n_edges = len(soff) - 1
    in_off = K * L * soff
    out_off = L * (soff - np.arange(n_edges + 1))
    original = oracle.classify_spheres(in_off, inner.T, out_off, outer.T, poses)
    rng = np.random.default_rng(3)
    bent = inner.copy()
    n_samp = bent.shape[1] // K
    s0 = rng.choice(n_samp, size=n_samp // 3, replace=False) * K
    mid = (bent[:3, s0] + bent[:3, s0 + K - 1]) / 2
    bent[:3, s0 + 1] = mid + np.array([[0.03], [0.03], [0.0]], dtype=np.float32)
    bent[3, s0 + 1] = 0.1
    want = oracle.classify_spheres(in_off, bent.T, out_off, outer.T, poses)
    changed = (want["labels"] != original["labels"]) & (want["kappa"] > PIN)
    assert changed.sum() >= 10, "the perturbation must matter for the test to mean anything"
    with rgg.Roadmap(L, K, n_boxes) as b:
        b.upload_edges(soff.astype(np.uint64), bent, outer)
        b.update_obstacles(np.arange(n_boxes), f32(poses))
        b.classify()
        got = b.fetch_labels()
    check_labels(got, want, "irregular upload")


def test_fetch_boxes_returns_the_table(rgg):
    sc = W.workload_planar(n_nodes=60, n_updates=2)
    with make_roadmap(rgg, sc.roadmap, sc.boxes.count) as r:
        poses, present = r.fetch_boxes()
        assert not present.any()
        r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
        up = sc.updates[0]
        r.update_obstacles(up.ids, f32(up.poses))    # pending: the table has the new pose
        poses, present = r.fetch_boxes()
        want = f32(sc.boxes.poses())
        want[up.ids] = f32(up.poses)
        assert present.all()
        np.testing.assert_array_equal(poses, want)


def test_work_counting_changes_no_bit(rgg):
    """The counting instance makes the same decisions and counts what it
    executed: rounds, outer tests after the cull, inner pairs."""
    sc = W.workload_7dof(n_nodes=400, n_updates=2)
    rm = sc.roadmap
    a = make_roadmap(rgg, rm, sc.boxes.count)
    b = make_roadmap(rgg, rm, sc.boxes.count)
    b.set_work_counting(True)
    for r in (a, b):
        r.update_obstacles(np.arange(sc.boxes.count), f32(sc.boxes.poses()))
        r.classify()
    for up in sc.updates:
        for r in (a, b):
            r.update_obstacles(up.ids, f32(up.poses))
            r.classify()
    np.testing.assert_array_equal(a.fetch_labels(), b.fetch_labels())
    ha, ta = a.fetch_box_sets()
    hb, tb = b.fetch_box_sets()
    np.testing.assert_array_equal(ha, hb)
    np.testing.assert_array_equal(ta, tb)
    c = b.work_counts()
    info = b.info()
    assert 0 < c["rounds"] <= 4 * info["num_tiles"] * 32
    assert 0 < c["outer_tests"]
    assert c["outer_tests"] < 4 * info["num_outer"] * 32    # the cull leaves a fraction
    assert 0 < c["inner_pairs"]
    assert b.work_counts() == {"rounds": 0, "outer_tests": 0, "inner_pairs": 0}
    assert a.work_counts()["rounds"] == 0                  # not counting
    for r in (a, b):
        r.check_status()
        r.close()
