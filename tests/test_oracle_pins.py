"""Pins of the FP64 oracle to facts outside itself.

Each test ties one oracle function to the paper's definitions or to
independent mathematics: closed forms, hand-derived cases, a different
formulation of the same quantity (constrained minimisation, product of
exponentials), invariants the definitions imply, and a brute-force check
against the exact robot geometry.  No test compares the oracle with itself
or with the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation

from paper_2603_28674_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_scenes.json")


def box_pose(centre, rot, half):
    return np.concatenate([np.asarray(centre, float), np.asarray(rot, float).reshape(9),
                           np.asarray(half, float)])


# --------------------------------------------------------------------------
# point-box distance
# --------------------------------------------------------------------------
def test_box_distance_closed_form_regions(oracle):
    """Arvo's distance: zero inside, the axis gap in a face region, the 2-D
    norm in an edge region, the 3-D norm in a corner region."""
    box = box_pose([0, 0, 0], np.eye(3), [1, 2, 3])
    assert oracle.box_distance(box, [0.5, -1.0, 2.0]) == 0.0
    assert oracle.box_distance(box, [1.0, 2.0, 3.0]) == 0.0          # corner contact
    assert oracle.box_distance(box, [2.0, 0.0, 0.0]) == pytest.approx(1.0, abs=1e-15)
    assert oracle.box_distance(box, [0.0, -2.5, 0.0]) == pytest.approx(0.5, abs=1e-15)
    assert oracle.box_distance(box, [2.0, 3.0, 0.0]) == pytest.approx(math.sqrt(2), abs=1e-15)
    assert oracle.box_distance(box, [-2.0, -3.0, -4.0]) == pytest.approx(math.sqrt(3), abs=1e-15)
    # translated box
    box2 = box_pose([10, -5, 1], np.eye(3), [1, 1, 1])
    assert oracle.box_distance(box2, [13.0, -5.0, 1.0]) == pytest.approx(2.0, abs=1e-14)


def test_box_distance_matches_constrained_minimisation(oracle):
    """d(x, box) = min over points y of the box of |x - y|, with the box
    parametrised in world coordinates as centre + R u, |u_k| <= h_k.  This is
    a different formulation (no change to the box frame), solved by bounded
    L-BFGS; a transposed rotation or a wrong clamp fails it."""
    rng = np.random.default_rng(7)
    rots = Rotation.random(30, random_state=11).as_matrix()
    for i in range(30):
        c = rng.uniform(-1, 1, 3)
        h = rng.uniform(0.05, 0.4, 3)
        x = c + rng.uniform(-1.2, 1.2, 3)
        r = rots[i]
        f = lambda u: float(np.sum((x - (c + r @ u)) ** 2))
        g = lambda u: -2.0 * r.T @ (x - (c + r @ u))
        best = min((minimize(f, u0, jac=g, method="L-BFGS-B",
                             bounds=list(zip(-h, h)), tol=1e-14)
                    for u0 in (np.zeros(3), h * 0.5, -h * 0.5)), key=lambda s: s.fun)
        want = math.sqrt(max(best.fun, 0.0))
        assert oracle.box_distance(box_pose(c, r, h), x) == pytest.approx(want, abs=2e-7)


def test_box_distance_rigid_motion_invariance(oracle):
    """Moving box and point by the same rigid motion keeps the distance."""
    rng = np.random.default_rng(3)
    for i in range(50):
        c = rng.uniform(-1, 1, 3)
        r = Rotation.random(random_state=100 + i).as_matrix()
        h = rng.uniform(0.05, 0.3, 3)
        x = rng.uniform(-1.5, 1.5, 3)
        q = Rotation.random(random_state=200 + i).as_matrix()
        t = rng.uniform(-2, 2, 3)
        d0 = oracle.box_distance(box_pose(c, r, h), x)
        d1 = oracle.box_distance(box_pose(q @ c + t, q @ r, h), q @ x + t)
        assert d1 == pytest.approx(d0, abs=1e-12)


# --------------------------------------------------------------------------
# forward kinematics
# --------------------------------------------------------------------------
def test_fk_planar_closed_form(oracle):
    """Planar revolute arm: o_i = sum_m l_m (cos phi_m, sin phi_m, 0) with
    phi_m the sum of the first m joint angles."""
    robot = W.planar_arm(3, 0.3)
    rng = np.random.default_rng(1)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, 3)
        o = oracle.forward_kinematics(robot, q)
        phi = np.cumsum(q)
        want = np.zeros((4, 3))
        want[1:, 0] = np.cumsum(0.3 * np.cos(phi))
        want[1:, 1] = np.cumsum(0.3 * np.sin(phi))
        np.testing.assert_allclose(o, want, atol=1e-14)


def _poe_origins(robot, q):
    """Frame origins by the product of exponentials: build the zero
    configuration from each joint's fixed part Tz(d) Tx(a) Rx(alpha), then
    rotate by q_j about joint j's home axis (z of frame j-1 through o_{j-1}),
    innermost joint last.  Uses scipy rotations, not DH matrices at q."""
    L = robot.num_links
    home_rot = [np.eye(3)]
    home_o = [np.zeros(3)]
    for i in range(L):
        r = home_rot[-1]
        o = home_o[-1] + r @ np.array([robot.a[i], 0.0, robot.d[i]])
        home_o.append(o)
        home_rot.append(r @ Rotation.from_rotvec([robot.alpha[i], 0, 0]).as_matrix())
    out = []
    for i in range(L + 1):
        p = home_o[i].copy()
        for j in reversed(range(min(i, L))):
            axis = home_rot[j][:, 2]
            piv = home_o[j]
            p = Rotation.from_rotvec(axis * q[j]).as_matrix() @ (p - piv) + piv
        out.append(p)
    return np.array(out)


@pytest.mark.parametrize("with_offsets", [False, True])
def test_fk_matches_product_of_exponentials(oracle, with_offsets):
    """The DH chain agrees with an independent product-of-exponentials
    construction on seeded 7-DOF arms (with and without link offsets d)."""
    rng = np.random.default_rng(5)
    robot = W.dh_arm(rng, 7)
    if with_offsets:
        robot = W.Robot(a=robot.a, alpha=robot.alpha, d=rng.uniform(-0.2, 0.2, 7),
                        radius=robot.radius, inner_per_link=5)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, 7)
        np.testing.assert_allclose(oracle.forward_kinematics(robot, q), _poe_origins(robot, q),
                                   atol=1e-12)


def test_fk_preserves_link_lengths(oracle):
    rng = np.random.default_rng(9)
    robot = W.dh_arm(rng, 7)
    for _ in range(20):
        o = oracle.forward_kinematics(robot, rng.uniform(-4, 4, 7))
        np.testing.assert_allclose(np.linalg.norm(np.diff(o, axis=0), axis=1),
                                   np.hypot(robot.a, robot.d), atol=1e-13)


# --------------------------------------------------------------------------
# discretisation and spheres
# --------------------------------------------------------------------------
def test_num_samples_cases(oracle):
    """n = max(2, ceil(|dq|_inf / step) + 1), both endpoints included
    (values chosen exactly representable)."""
    assert oracle.num_samples([0.0, 0.0], [0.0, 0.0], 0.125) == 2
    assert oracle.num_samples([0.0], [0.0625], 0.125) == 2
    assert oracle.num_samples([0.0], [0.125], 0.125) == 2
    assert oracle.num_samples([0.0], [0.25], 0.125) == 3
    assert oracle.num_samples([0.0], [0.3125], 0.125) == 4
    assert oracle.num_samples([1.0, 0.0, 2.0], [0.9375, -0.5, 2.25], 0.125) == 5
    assert oracle.num_samples([0.0], [1.0], 0.0) == -1


def test_inner_sphere_placement(oracle):
    """K spheres of radius R on the link axis at fractions (j + 1/2)/K
    (Sec. 4.2); a one-link arm along +x, l = 0.3, K = 4."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    inner, outer = oracle.edge_spheres(robot, [0.0], [0.0], 0.05)
    assert inner.shape == (2, 1, 4, 4) and outer.shape == (1, 1, 4)
    np.testing.assert_allclose(inner[0, 0, :, 0], [0.0375, 0.1125, 0.1875, 0.2625], atol=1e-15)
    np.testing.assert_allclose(inner[:, 0, :, 1:3], 0.0, atol=1e-15)
    np.testing.assert_allclose(inner[:, 0, :, 3], 0.03, atol=0)
    # static edge: outer sphere = the capsule's bounding sphere
    np.testing.assert_allclose(outer[0, 0], [0.15, 0.0, 0.0, 0.18], atol=1e-15)


def test_outer_sphere_hand_values(oracle):
    """Planar 3-link arm, l = 0.3, R = 0.03.  Only joint 1 moves, by 0.05 per
    interval: the radius of link i grows by 1/2 * 0.05 * (l_1 + ... + l_i).
    Only joint 3 moves: links 1 and 2 keep the static radius 0.18.  The centre
    is the link midpoint at the interval's middle configuration."""
    robot = W.planar_arm(3, 0.3, 0.03, 4)
    inner, outer = oracle.edge_spheres(robot, [0.0, 0.0, 0.0], [0.1, 0.0, 0.0], 0.05)
    assert inner.shape[0] == 3
    np.testing.assert_allclose(outer[0, :, 3], [0.18 + 0.025 * 0.3, 0.18 + 0.025 * 0.6,
                                                0.18 + 0.025 * 0.9], atol=1e-15)
    th = 0.025  # middle of the first interval
    mids = np.array([0.15, 0.45, 0.75]) * np.array([[math.cos(th)], [math.sin(th)]])
    np.testing.assert_allclose(outer[0, :, 0], mids[0], atol=1e-14)
    np.testing.assert_allclose(outer[0, :, 1], mids[1], atol=1e-14)
    inner, outer = oracle.edge_spheres(robot, [0.0, 0.0, 0.0], [0.0, 0.0, -0.1], 0.05)
    np.testing.assert_allclose(outer[1, :, 3], [0.18, 0.18, 0.18 + 0.025 * 0.3], atol=1e-15)


def test_outer_sphere_contains_swept_capsule(oracle):
    """Outer sphere of (interval, link) contains the link's capsule at every
    configuration of the interval (Sec. 3.2's outer approximation), checked
    with the product-of-exponentials kinematics on a dense grid; and it
    contains the inner spheres of both end samples."""
    rng = np.random.default_rng(21)
    robot = W.dh_arm(rng, 7)
    for _ in range(4):
        qa = rng.uniform(-math.pi, math.pi, 7)
        qb = qa + rng.uniform(-0.3, 0.3, 7)
        inner, outer = oracle.edge_spheres(robot, qa, qb, 0.05)
        n = inner.shape[0]
        for k in range(n - 1):
            for t in np.linspace(0.0, 1.0, 9):
                q = qa + ((k + t) / (n - 1)) * (qb - qa)
                o = _poe_origins(robot, q)
                for i in range(7):
                    pts = o[i] + np.linspace(0, 1, 11)[:, None] * (o[i + 1] - o[i])
                    far = np.linalg.norm(pts - outer[k, i, :3], axis=1).max() + robot.radius[i]
                    assert far <= outer[k, i, 3] + 1e-12
            for i in range(7):
                for s in (inner[k, i], inner[k + 1, i]):
                    gap = np.linalg.norm(s[:, :3] - outer[k, i, :3], axis=1) + s[:, 3]
                    assert np.all(gap <= outer[k, i, 3] + 1e-12)


# --------------------------------------------------------------------------
# labels on hand-derived cases
# --------------------------------------------------------------------------
def test_golden_tiny_scenes(oracle):
    g = json.load(open(GOLDEN))
    rb = g["robot"]
    robot = W.Robot(a=np.array(rb["a"]), alpha=np.array(rb["alpha"]), d=np.array(rb["d"]),
                    radius=np.array(rb["radius"]), inner_per_link=rb["inner_per_link"])
    for case in g["cases"]:
        out = oracle.classify(robot, [case["qa"]], [case["qb"]], g["step"], [case["box"]])
        assert out["labels"][0] == case["label"], case["name"]
        assert out["kappa"][0] == pytest.approx(case["kappa"], abs=1e-12), case["name"]
        for k in ("h_in", "h_out"):
            if k in case:
                assert out[k][0] == pytest.approx(case[k], abs=1e-12), case["name"]
        if "n_samples" in case:
            assert oracle.num_samples(case["qa"], case["qb"], g["step"]) == case["n_samples"]


def test_absent_boxes_and_empty_scene(oracle):
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    box = box_pose([0.2, 0, 0], np.eye(3), [0.05] * 3)
    out = oracle.classify(robot, [[0.0]], [[0.0]], 0.05, [box], present=[0])
    assert out["labels"][0] == oracle.GREEN
    assert math.isinf(out["kappa"][0])
    out = oracle.classify(robot, np.zeros((0, 1)), np.zeros((0, 1)), 0.05, [box])
    assert out["labels"].shape == (0,)


def test_last_sample_is_checked(oracle):
    """A box reached only at the final configuration of the edge must not
    leave it green: q from 1.0 to 0.0 rad ends with the arm along +x."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    box = box_pose([0.2, 0, 0], np.eye(3), [0.01] * 3)
    out = oracle.classify(robot, [[1.0]], [[0.0]], 0.05, [box])
    assert out["labels"][0] == oracle.RED
    out = oracle.classify(robot, [[0.0]], [[1.0]], 0.05, [box])
    assert out["labels"][0] == oracle.RED


# --------------------------------------------------------------------------
# invariants on seeded scenes
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_7dof():
    sc = W.workload_7dof(n_nodes=300, n_boxes=40, n_updates=0)
    return sc.roadmap, sc.boxes


def test_inner_inside_outer_implies_order(oracle, small_7dof):
    """inner subset of outer => h_out >= h_in per edge and hit bits subset of
    touch bits; the label agrees with the clearances."""
    rm, boxes = small_7dof
    out = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses(), bits=True)
    assert np.all(out["h_out"] >= out["h_in"] - 1e-12)
    assert np.all((out["hit"] & ~out["touch"]) == 0)
    lab = out["labels"]
    np.testing.assert_array_equal(lab == oracle.RED, out["h_in"] >= 0)
    np.testing.assert_array_equal(lab == oracle.GREEN, out["h_out"] < 0)
    assert set(np.unique(lab)) <= {0, 1, 2}
    assert (lab == oracle.GREEN).any() and (lab == oracle.RED).any() and \
        (lab == oracle.GRAY).any()


def test_per_box_decomposition(oracle, small_7dof):
    """Bits of the full box set are the per-box bits side by side (40 boxes
    span two 32-bit words), and labels follow from the union."""
    rm, boxes = small_7dof
    sel = slice(0, 60)
    full = oracle.classify(rm.robot, rm.q_from[sel], rm.q_to[sel], rm.step, boxes.poses(),
                           bits=True)
    for b in range(boxes.count):
        one = oracle.classify(rm.robot, rm.q_from[sel], rm.q_to[sel], rm.step,
                              boxes.poses([b]), bits=True)
        np.testing.assert_array_equal((full["hit"][:, b // 32] >> (b % 32)) & 1, one["hit"][:, 0])
        np.testing.assert_array_equal((full["touch"][:, b // 32] >> (b % 32)) & 1,
                                      one["touch"][:, 0])


def test_permutation_and_direction_invariance(oracle, small_7dof):
    rm, boxes = small_7dof
    base = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
    perm = np.random.default_rng(4).permutation(boxes.count)
    shuf = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses()[perm])
    np.testing.assert_array_equal(base["labels"], shuf["labels"])
    rev = oracle.classify(rm.robot, rm.q_to, rm.q_from, rm.step, boxes.poses())
    pinned = base["kappa"] > 1e-9
    np.testing.assert_array_equal(base["labels"][pinned], rev["labels"][pinned])


def test_growing_boxes_never_moves_toward_green(oracle, small_7dof):
    rm, boxes = small_7dof
    base = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
    big = boxes.copy()
    big.half *= 1.15
    grown = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, big.poses())
    assert np.all(grown["labels"] >= base["labels"])   # GREEN < GRAY < RED
    assert np.any(grown["labels"] > base["labels"])


# --------------------------------------------------------------------------
# brute force against the exact robot geometry
# --------------------------------------------------------------------------
def test_segment_box_distance_vs_dense_sampling(oracle):
    rng = np.random.default_rng(12)
    for i in range(10):
        box = box_pose(rng.uniform(-0.5, 0.5, 3), Rotation.random(random_state=i).as_matrix(),
                       rng.uniform(0.05, 0.3, 3))
        p0, p1 = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
        ts = np.linspace(0, 1, 100_001)
        dense = min(oracle.box_distance(box, p0 + t * (p1 - p0)) for t in ts[::100])
        fine = np.linspace(0, 1, 100_001)
        # refine around the coarse minimum with every sample of the dense grid
        lo = max(0, int(np.argmin([oracle.box_distance(box, p0 + t * (p1 - p0))
                                   for t in ts[::100]])) * 100 - 200)
        dense = min(dense, min(oracle.box_distance(box, p0 + t * (p1 - p0))
                               for t in fine[lo:lo + 400]))
        got = oracle.segment_box_distance(p0, p1, box)
        assert got <= dense + 1e-12
        assert got >= dense - 1e-4   # grid spacing 1e-5 * segment length


@pytest.mark.parametrize("which", ["planar", "7dof"])
def test_red_collides_and_green_is_free(oracle, which):
    """RED edges collide at some original sample and GREEN edges are free on
    a 10x finer resampling, by exact capsule-box distances (segment-box
    minimisation) that do not use the sphere approximations."""
    rng = np.random.default_rng(31)
    # a few small boxes away from the arm's base, so that all three labels occur
    if which == "planar":
        rm = W.prm_roadmap(rng, W.planar_arm(), 120, 6, 0.05)
        poses = np.array([box_pose([0.6, 0.3, 0.0], np.eye(3), [0.06, 0.05, 0.05]),
                          box_pose([-0.45, -0.55, 0.0], np.eye(3), [0.04, 0.07, 0.05])])
    else:
        rm = W.prm_roadmap(rng, W.dh_arm(rng, 7), 120, 10, 0.02)
        rot = Rotation.random(2, random_state=5).as_matrix()
        poses = np.array([box_pose([0.9, 0.4, 0.3], rot[0], [0.08, 0.05, 0.1]),
                          box_pose([-0.3, -0.8, 0.7], rot[1], [0.06, 0.09, 0.05])])
    out = oracle.classify(rm.robot, rm.q_from, rm.q_to, rm.step, poses)
    lab = out["labels"]
    red = np.flatnonzero(lab == oracle.RED)[:40]
    green = np.flatnonzero(lab == oracle.GREEN)[:40]
    assert red.size and green.size
    for e in red:
        v, _ = oracle.edge_dense_clearance(rm.robot, rm.q_from[e], rm.q_to[e], rm.step, 1, poses)
        assert v <= 1e-12
    for e in green:
        v, _ = oracle.edge_dense_clearance(rm.robot, rm.q_from[e], rm.q_to[e], rm.step, 10, poses)
        assert v > 0.0


# --------------------------------------------------------------------------
# labels from caller-supplied sphere sets
# --------------------------------------------------------------------------
def test_classify_spheres_hand_cases(oracle):
    """Hand-derived labels and clearances for single spheres against the box
    of half-extent 0.1 at the origin (a second, far box is absent)."""
    box = box_pose([0, 0, 0], np.eye(3), [0.1] * 3)
    far = box_pose([0.3, 0, 0], np.eye(3), [0.05] * 3)   # would hit edge 1: absent
    inner = [[0.15, 0, 0, 0.06],      # e0: d = 0.05 <= 0.06: hit by 0.01
             [0.3, 0, 0, 0.05],       # e1: d = 0.2: miss by 0.15
             [1, 1, 1, 0.1],          # e2: d = 0.9 sqrt(3)
             [0.2, 0, 0, 0.1]]        # e3: d = 0.1 = r: contact counts
    outer = [[0.15, 0, 0, 0.2],       # e0
             [0.25, 0, 0, 0.2],       # e1: d = 0.15 <= 0.2: touch by 0.05
             [1, 1, 1, 0.2],          # e2: miss
             [0.2, 0, 0, 0.15]]       # e3
    in_off = [0, 1, 2, 3, 4, 4]       # e4 has no spheres at all
    out_off = [0, 1, 2, 3, 4, 4]
    out = oracle.classify_spheres(in_off, inner, out_off, outer, [box, far], present=[1, 0],
                                  bits=True)
    R, G, Y = oracle.RED, oracle.GREEN, oracle.GRAY
    assert list(out["labels"]) == [R, Y, G, R, G]
    d2 = 0.9 * math.sqrt(3)
    np.testing.assert_allclose(out["kappa"][:4], [0.01, 0.05, min(d2 - 0.1, d2 - 0.2), 0.0],
                               atol=1e-12)
    assert math.isinf(out["kappa"][4])
    assert list(out["hit"][:, 0]) == [1, 0, 0, 1, 0]
    assert list(out["touch"][:, 0]) == [1, 1, 0, 1, 0]
    # with the far box present, edge 1's inner sphere (d = 0.05 to it) is a hit
    out = oracle.classify_spheres(in_off, inner, out_off, outer, [box, far], bits=True)
    assert out["labels"][1] == R and out["hit"][1, 0] == 2


def test_classify_spheres_agrees_with_robot_classify(oracle, small_7dof):
    """The robot's own spheres fed as explicit sets give the robot
    classification's labels and clearances."""
    rm, boxes = small_7dof
    ins, outs, io, oo = [], [], [0], [0]
    for e in range(40):
        si, so = oracle.edge_spheres(rm.robot, rm.q_from[e], rm.q_to[e], rm.step)
        ins.append(si.reshape(-1, 4))
        outs.append(so.reshape(-1, 4))
        io.append(io[-1] + ins[-1].shape[0])
        oo.append(oo[-1] + outs[-1].shape[0])
    got = oracle.classify_spheres(io, np.concatenate(ins), oo, np.concatenate(outs),
                                  boxes.poses())
    want = oracle.classify(rm.robot, rm.q_from[:40], rm.q_to[:40], rm.step, boxes.poses())
    np.testing.assert_array_equal(got["labels"], want["labels"])
    np.testing.assert_allclose(got["kappa"], want["kappa"], rtol=0, atol=1e-12)


def test_dense_clearance_hand_cases(oracle):
    """Closed-form clearances of a 1-link planar arm (length 0.3, R 0.03):
    a resting arm 0.15 m from a box face; an arm sweeping 0 -> pi/2 through a
    box centred on the 45 degree ray (the resampled configuration t = 0.5 is
    exactly q = pi/4); and the same box moved out of reach along that ray."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    box = box_pose([0.5, 0.0, 0.0], np.eye(3), [0.05] * 3)
    v, t = oracle.edge_dense_clearance(robot, [0.0], [0.0], 0.05, 3, [box])
    assert v == pytest.approx(0.15 - 0.03, abs=1e-9)
    c45 = math.cos(math.pi / 4)
    inside = box_pose([0.2 * c45, 0.2 * c45, 0.0], np.eye(3), [0.02] * 3)
    v, t = oracle.edge_dense_clearance(robot, [0.0], [math.pi / 2], 0.05, 2, [inside])
    # the axis meets the box over a range of angles around pi/4
    assert v == pytest.approx(-0.03, abs=1e-9) and 0.3 < t <= 0.5
    beyond = box_pose([0.5 * c45, 0.5 * c45, 0.0], np.eye(3), [0.02] * 3)
    v, t = oracle.edge_dense_clearance(robot, [0.0], [math.pi / 2], 0.05, 2, [beyond])
    # the nearest box corner lies on the ray at 0.5 - 0.02 sqrt(2)
    assert v == pytest.approx(0.5 - 0.02 * math.sqrt(2) - 0.3 - 0.03, abs=1e-9)
    assert t == pytest.approx(0.5)


# --------------------------------------------------------------------------
# the paper's primitives: OBBs, separating axes, shortcut splines
# --------------------------------------------------------------------------
def test_obb_separation_hand_values(oracle):
    I = np.eye(3)
    a = box_pose([0, 0, 0], I, [0.5] * 3)
    assert oracle.obb_separation(a, box_pose([2, 0, 0], I, [0.5] * 3)) == pytest.approx(1.0)
    assert oracle.obb_separation(a, box_pose([0.5, 0, 0], I, [0.5] * 3)) == pytest.approx(-0.5)
    rz = Rotation.from_euler("z", 45, degrees=True).as_matrix()
    # the rotated box reaches 0.5 sqrt(2) along x
    assert oracle.obb_separation(a, box_pose([2, 0, 0], rz, [0.5] * 3)) == \
        pytest.approx(2 - 0.5 - 0.5 * math.sqrt(2))


def test_obb_separation_sign_matches_lp_feasibility(oracle):
    """Boxes meet exactly when a point satisfies both boxes' slab
    constraints (a linear feasibility problem); SAT must agree."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(8)
    agree = 0
    for i in range(300):
        A = box_pose(rng.uniform(-0.3, 0.3, 3), Rotation.random(random_state=2 * i).as_matrix(),
                     rng.uniform(0.05, 0.4, 3))
        B = box_pose(rng.uniform(-0.3, 0.3, 3) + rng.uniform(-1, 1, 3) * 0.6,
                     Rotation.random(random_state=2 * i + 1).as_matrix(), rng.uniform(0.05, 0.4, 3))
        rows, rhs = [], []
        for box in (A, B):
            c, R, h = box[:3], box[3:12].reshape(3, 3), box[12:]
            for k in range(3):
                u = R[:, k]
                rows += [u, -u]
                rhs += [h[k] + u @ c, h[k] - u @ c]
        lp = linprog(np.zeros(3), A_ub=np.array(rows), b_ub=np.array(rhs), bounds=[(None, None)] * 3,
                     method="highs")
        sep = oracle.obb_separation(A, B)
        if abs(sep) < 1e-9:
            continue
        assert (sep <= 0) == (lp.status == 0), (i, sep, lp.status)
        agree += 1
    assert agree > 250


def test_edge_obbs_hold_the_swept_capsules(oracle):
    """Points of every link capsule at a 10x finer resampling (axis points
    pushed out by the radius in random directions) lie inside the body's
    box; a resting planar link gets the hand-derived box."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    ob = oracle.edge_obbs(robot, [0.0], [0.0], 0.05)[0]
    np.testing.assert_allclose(ob[:3], [0.15, 0, 0], atol=1e-12)
    np.testing.assert_allclose(np.abs(ob[3:12].reshape(3, 3)), np.eye(3), atol=1e-12)
    np.testing.assert_allclose(ob[12:], [0.18, 0.03, 0.03], atol=1e-12)
    rng = np.random.default_rng(4)
    rm = W.prm_roadmap(rng, W.dh_arm(rng, 7), 60, 6, 0.05)
    rob = rm.robot
    for e in range(0, rm.num_edges, 7):
        obbs = oracle.edge_obbs(rob, rm.q_from[e], rm.q_to[e], rm.step)
        n = oracle.num_samples(rm.q_from[e], rm.q_to[e], rm.step)
        for t in np.linspace(0, 1, 10 * (n - 1) + 1):
            q = rm.q_from[e] + t * (rm.q_to[e] - rm.q_from[e])
            J = oracle.forward_kinematics(rob, q)
            for i in range(rob.num_links):
                c, R, h = obbs[i, :3], obbs[i, 3:12].reshape(3, 3), obbs[i, 12:]
                for f in (0.0, 0.5, 1.0):
                    p = J[i] + f * (J[i + 1] - J[i])
                    d = rng.normal(size=3)
                    p = p + rob.radius[i] * d / np.linalg.norm(d)
                    assert np.all(np.abs(R.T @ (p - c)) <= h + 1e-9), (e, t, i)


def _obb_parts(ob):
    return ob[:3], ob[3:12].reshape(3, 3), ob[12:]


def test_edge_obbs_moving_planar_links_hand_derived(oracle):
    """Moving edges whose boxes follow by hand (Sec. 4.2's per-body box; the
    axes come from the motion, the growth is the outer spheres' motion bound).

    Planar links of length 0.3 m and radius 0.03 m; a joint sweeps 0 -> 0.5
    rad in 4 steps of 0.125 rad (5 configurations, the middle one at 0.25).
    A link that rotates rigidly about a fixed point has its axis u1 along the
    bisector (cos .25, sin .25, 0); its midpoint moves along a chord, which is
    normal to the bisector, so u2 = (-sin .25, cos .25, 0) and u3 = +z.  A
    link point at distance s from the pivot projects to s cos(q - .25) on u1
    and s sin(q - .25) on u2.  Each half-extent grows by R plus half of
    sum_{j<=i} |dq_j| rho_{j,i} with rho_{j,i} = sum_{m=j..i} l_m."""
    c, s = math.cos(0.25), math.sin(0.25)
    u1, u2, u3 = np.array([c, s, 0.0]), np.array([-s, c, 0.0]), np.array([0.0, 0.0, 1.0])
    rot = np.stack([u1, u2, u3], axis=1)
    dq = 0.5 / 4

    # one link about the origin: spans [0, 0.3] on u1, +-0.3 sin .25 on u2
    ob = oracle.edge_obbs(W.planar_arm(1, 0.3, 0.03, 4), [0.0], [0.5], 0.125)
    ctr, R, h = _obb_parts(ob[0])
    grow = 0.03 + 0.5 * 0.3 * dq
    np.testing.assert_allclose(R, rot, atol=1e-12)
    np.testing.assert_allclose(ctr, 0.15 * u1, atol=1e-12)
    np.testing.assert_allclose(h, [0.15 + grow, 0.3 * s + grow, grow], atol=1e-12)

    # two links, joint 0 turning: link 1 (from 0.3 to 0.6 m along the arm)
    # turns rigidly about the origin; rho_{0,1} = l_0 + l_1
    ob = oracle.edge_obbs(W.planar_arm(2, 0.3, 0.03, 4), [0.0, 0.0], [0.5, 0.0], 0.125)
    ctr, R, h = _obb_parts(ob[1])
    lo1 = 0.3 * c - 0.3          # the near end at the first / last configuration
    grow = 0.03 + 0.5 * (0.3 + 0.3) * dq
    np.testing.assert_allclose(R, rot, atol=1e-12)
    np.testing.assert_allclose(ctr, 0.3 * u1 + 0.5 * (lo1 + 0.3) * u1, atol=1e-12)
    np.testing.assert_allclose(h, [0.5 * (0.3 - lo1) + grow, 0.6 * s + grow, grow], atol=1e-12)

    # two links, joint 1 turning: link 0 rests (no displacement: u2 is the
    # world axis least aligned with u1 = x, i.e. y), link 1 turns about
    # (0.3, 0, 0); rho_{1,1} = l_1 and joint 0 contributes nothing
    ob = oracle.edge_obbs(W.planar_arm(2, 0.3, 0.03, 4), [0.0, 0.0], [0.0, 0.5], 0.125)
    ctr, R, h = _obb_parts(ob[0])
    np.testing.assert_allclose(R, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(ctr, [0.15, 0, 0], atol=1e-12)
    np.testing.assert_allclose(h, [0.18, 0.03, 0.03], atol=1e-12)
    ctr, R, h = _obb_parts(ob[1])
    grow = 0.03 + 0.5 * 0.3 * dq
    np.testing.assert_allclose(R, rot, atol=1e-12)
    np.testing.assert_allclose(ctr, [0.3, 0, 0] + 0.15 * u1, atol=1e-12)
    np.testing.assert_allclose(h, [0.15 + grow, 0.3 * s + grow, grow], atol=1e-12)


def test_edge_splines_follow_the_shortcut_rule(oracle):
    """Kept vertices are original centres, first and last included; every
    dropped centre lies closer than R to its covering segment; and no kept
    segment could be stretched to the next centre (greedy)."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    sp = oracle.edge_splines(robot, [0.0], [0.0], 0.05)
    assert all(v.shape == (2, 3) for v in sp[0])      # a resting link: one segment
    rng = np.random.default_rng(6)
    rm = W.prm_roadmap(rng, W.dh_arm(rng, 7), 40, 6, 0.02)
    rob = rm.robot
    L, K = rob.num_links, rob.inner_per_link
    for e in range(0, rm.num_edges, 5):
        n = oracle.num_samples(rm.q_from[e], rm.q_to[e], rm.step)
        J = np.array([oracle.forward_kinematics(rob, rm.q_from[e] + c / (n - 1) *
                                                (rm.q_to[e] - rm.q_from[e])) for c in range(n)])
        sp = oracle.edge_splines(rob, rm.q_from[e], rm.q_to[e], rm.step)
        for i in range(L):
            R = rob.radius[i]
            for s in range(K):
                f = (s + 0.5) / K
                V = J[:, i] + f * (J[:, i + 1] - J[:, i])
                kept = [int(np.argmin(np.linalg.norm(V - v, axis=1))) for v in sp[i][s]]
                np.testing.assert_allclose(sp[i][s], V[kept], atol=1e-12)
                assert kept[0] == 0 and kept[-1] == n - 1
                for j, p in zip(kept[:-1], kept[1:]):
                    for m in range(j + 1, p):
                        assert oracle.segment_point_distance(V[j], V[p], V[m]) < R
                    if p < n - 1:
                        assert max(oracle.segment_point_distance(V[j], V[p + 1], V[m])
                                   for m in range(j + 1, p + 1)) >= R


def test_classify_obb_hand_scenes(oracle):
    """A resting planar link along +x (length 0.3, R 0.03, spheres at 0.0375,
    0.1125, 0.1875, 0.2625): its box is [0, 0.3] x [-0.03, 0.03] grown to
    half-extents (0.18, 0.03, 0.03) about (0.15, 0, 0)."""
    robot = W.planar_arm(1, 0.3, 0.03, 4)
    I = np.eye(3)
    cases = [  # (box centre, half, label, kappa)
        ([0.15, 0.0, 0.0], 0.05, oracle.RED, 0.05 - 0.0375),
        ([0.15, 0.5, 0.0], 0.05, oracle.GREEN, 0.5 - 0.03 - 0.05),
        ([0.15, 0.07, 0.0], 0.05, oracle.GRAY, 0.01),
    ]
    for c, h, lab, kap in cases:
        out = oracle.classify_obb(robot, [[0.0]], [[0.0]], 0.05, [box_pose(c, I, [h] * 3)])
        assert out["labels"][0] == lab, c
        assert out["kappa"][0] == pytest.approx(kap, abs=1e-12), c


def test_classify_obb_green_edges_are_free(oracle):
    """Green by the boxes means no box meets the swept capsules: a 10x finer
    exact capsule-box check finds every green edge free."""
    rng = np.random.default_rng(9)
    rm = W.prm_roadmap(rng, W.dh_arm(rng, 7), 100, 8, 0.05)
    boxes = W.random_boxes(rng, 6, extent=1.0)
    out = oracle.classify_obb(rm.robot, rm.q_from, rm.q_to, rm.step, boxes.poses())
    green = np.flatnonzero(out["labels"] == oracle.GREEN)
    assert green.size >= 10 and (out["labels"] != oracle.GREEN).any()
    for e in green[:25]:
        v, _ = oracle.edge_dense_clearance(rm.robot, rm.q_from[e], rm.q_to[e], rm.step, 10,
                                           boxes.poses())
        assert v > 0.0
