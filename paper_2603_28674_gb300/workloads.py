"""Seeded synthetic workloads for the Red-Green-Gray edge-classification pass.

This module only draws inputs: robot models (Denavit-Hartenberg parameters,
link radii), roadmap edges (pairs of joint-space endpoints), obstacle boxes
(centre, rotation, half-extents) and the streams of obstacle moves.  None of
the classification arithmetic lives here: sample counts, kinematics, sphere
placement, box tests and labels are computed independently by the CUDA
library and by the CPU oracle, which both read these inputs.

The paper's environments, planner roadmaps and robot models are not
available, so every workload is a stand-in drawn with a fixed seed.  The
paper's own experiments translate obstacles between updates (Sec. 5) and
build the roadmap as a PRM without obstacles; the recipes below follow that.

Workloads (sizes as in the project's five configurations):
  1  planar 3-link arm, 500-node k=6 PRM, 0.05 rad step, 16 AABBs, 2 moved
  2  7-DOF DH arm, 10k-node k=10 PRM, 0.02 rad step, 64 OBBs, 8 moved
  3  same arm, ~500k-edge PRM, ~80 samples/edge, 256 OBBs, 32 moved (and a
     mixed-label variant: the same roadmap among 256 small boxes in a 4 m cube)
  4  128 roadmaps (3/6/7-DOF), log-uniform edge and sample counts, own boxes
  5  8 resident roadmaps (4x ~50k, 4x ~200k edges) and a Poisson stream of
     obstacle-move requests
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Every workload draws from numpy's PCG64 with seed 1000 + workload index;
# independent sub-streams come from SeedSequence.spawn.
BASE_SEED = 1000


# --------------------------------------------------------------------------
# data containers
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Robot:
    """A serial arm in standard DH form; link i is the segment between frame
    origins i and i+1, a capsule of radius ``radius[i]`` carrying
    ``inner_per_link`` inscribed spheres."""
    a: np.ndarray
    alpha: np.ndarray
    d: np.ndarray
    radius: np.ndarray
    inner_per_link: int

    @property
    def num_links(self) -> int:
        return int(self.a.shape[0])


@dataclasses.dataclass
class Roadmap:
    """Roadmap edges as joint-space segments; ``step`` is the resolution eps."""
    robot: Robot
    q_from: np.ndarray  # [N, L] float64
    q_to: np.ndarray    # [N, L] float64
    step: float

    @property
    def num_edges(self) -> int:
        return int(self.q_from.shape[0])


@dataclasses.dataclass
class BoxSet:
    """Oriented boxes: centre [M,3], rotation [M,3,3] (columns are the box
    axes in world coordinates), half-extents [M,3]."""
    centre: np.ndarray
    rot: np.ndarray
    half: np.ndarray

    @property
    def count(self) -> int:
        return int(self.centre.shape[0])

    def poses(self, ids: Optional[np.ndarray] = None) -> np.ndarray:
        """Pose records [m, 15] float64: centre(3), R(9 row-major), half(3)."""
        sel = slice(None) if ids is None else np.asarray(ids, dtype=np.int64)
        c, r, h = self.centre[sel], self.rot[sel], self.half[sel]
        return np.concatenate([c, r.reshape(-1, 9), h], axis=1).astype(np.float64)

    def copy(self) -> "BoxSet":
        return BoxSet(self.centre.copy(), self.rot.copy(), self.half.copy())


@dataclasses.dataclass
class Update:
    """One obstacle update: the boxes ``ids`` take the absolute ``poses``."""
    ids: np.ndarray    # [m] uint32
    poses: np.ndarray  # [m, 15] float64


@dataclasses.dataclass
class Scene:
    name: str
    roadmap: Roadmap
    boxes: BoxSet            # initial poses (all boxes placed before updates)
    updates: List[Update]    # applied in order after the initial placement


@dataclasses.dataclass
class Request:
    """A serving request: at ``arrival_s`` move boxes of roadmap ``roadmap``."""
    arrival_s: float
    roadmap: int
    update: Update


# --------------------------------------------------------------------------
# robots
# --------------------------------------------------------------------------
def planar_arm(num_links: int = 3, length: float = 0.3, radius: float = 0.03,
               inner_per_link: int = 4) -> Robot:
    """Planar revolute arm in the z=0 plane (all twists zero)."""
    z = np.zeros(num_links)
    return Robot(a=np.full(num_links, length), alpha=z.copy(), d=z.copy(),
                 radius=np.full(num_links, radius), inner_per_link=inner_per_link)


def dh_arm(rng: np.random.Generator, dof: int, inner_per_link: int = 5) -> Robot:
    """Seeded DH arm: a_i ~ U[0.1, 0.4] m, twists alternating +pi/2, -pi/2,
    d_i = 0, capsule radius R_i ~ U[0.03, 0.06] m per link."""
    a = rng.uniform(0.1, 0.4, size=dof)
    alpha = np.array([math.pi / 2 if i % 2 == 0 else -math.pi / 2 for i in range(dof)])
    radius = rng.uniform(0.03, 0.06, size=dof)
    return Robot(a=a, alpha=alpha, d=np.zeros(dof), radius=radius,
                 inner_per_link=inner_per_link)


# --------------------------------------------------------------------------
# roadmaps
# --------------------------------------------------------------------------
def prm_knn_edges(rng: np.random.Generator, n_nodes: int, dof: int, k: int):
    """PRM without obstacles: nodes uniform in [-pi, pi]^dof, undirected union
    of each node's k nearest neighbours (Euclidean, no angle wrap-around).
    Returns (nodes [n, dof], pairs [N, 2] with pairs[:,0] < pairs[:,1])."""
    from scipy.spatial import cKDTree

    nodes = rng.uniform(-math.pi, math.pi, size=(n_nodes, dof))
    tree = cKDTree(nodes)
    _, nbr = tree.query(nodes, k=k + 1)
    src = np.repeat(np.arange(n_nodes), k)
    dst = nbr[:, 1:].reshape(-1)
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    keep = lo != hi
    pairs = np.unique(np.stack([lo[keep], hi[keep]], axis=1), axis=0)
    # random edge order, so that neighbouring edges are not spatially sorted
    pairs = pairs[rng.permutation(pairs.shape[0])]
    return nodes, pairs


def prm_roadmap(rng: np.random.Generator, robot: Robot, n_nodes: int, k: int,
                step: float) -> Roadmap:
    nodes, pairs = prm_knn_edges(rng, n_nodes, robot.num_links, k)
    return Roadmap(robot=robot, q_from=np.ascontiguousarray(nodes[pairs[:, 0]]),
                   q_to=np.ascontiguousarray(nodes[pairs[:, 1]]), step=float(step))


def segment_roadmap(rng: np.random.Generator, robot: Robot, n_edges: int, step: float,
                    len_lo: float, len_hi: float) -> Roadmap:
    """Edges drawn as independent joint-space segments: start uniform in
    [-pi, pi]^dof, random direction, max-norm length log-uniform in
    [len_lo, len_hi] * step (so the number of configurations per edge is
    spread log-uniformly)."""
    dof = robot.num_links
    qa = rng.uniform(-math.pi, math.pi, size=(n_edges, dof))
    u = rng.uniform(-1.0, 1.0, size=(n_edges, dof))
    u /= np.max(np.abs(u), axis=1, keepdims=True)
    length = step * np.exp(rng.uniform(math.log(len_lo), math.log(len_hi), size=n_edges))
    qb = qa + u * length[:, None]
    return Roadmap(robot=robot, q_from=qa, q_to=qb, step=float(step))


# --------------------------------------------------------------------------
# boxes and their motion
# --------------------------------------------------------------------------
def random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """Uniformly random rotations from normalised Gaussian quaternions."""
    q = rng.normal(size=(m, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.empty((m, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def random_boxes(rng: np.random.Generator, m: int, planar: bool = False,
                 oriented: bool = True, extent: float = 1.0,
                 half_lo: float = 0.05, half_hi: float = 0.2) -> BoxSet:
    """Centres uniform in [-extent, extent]^3 (z = 0 when planar),
    half-extents U[half_lo, half_hi]^3, uniformly random rotations when
    ``oriented`` (identity otherwise)."""
    c = rng.uniform(-extent, extent, size=(m, 3))
    if planar:
        c[:, 2] = 0.0
    h = rng.uniform(half_lo, half_hi, size=(m, 3))
    r = random_rotations(rng, m) if oriented else np.tile(np.eye(3), (m, 1, 1))
    return BoxSet(centre=c, rot=r, half=h)


def move_boxes(rng: np.random.Generator, boxes: BoxSet, n_moved: int,
               planar: bool = False, max_shift: float = 0.3) -> Update:
    """Pick ``n_moved`` boxes uniformly without replacement and translate each
    by U[-max_shift, max_shift] per axis (in the plane when ``planar``),
    keeping its orientation.  ``boxes`` is advanced to the new poses; the
    returned update carries the absolute poses."""
    ids = np.sort(rng.choice(boxes.count, size=n_moved, replace=False)).astype(np.uint32)
    shift = rng.uniform(-max_shift, max_shift, size=(n_moved, 3))
    if planar:
        shift[:, 2] = 0.0
    boxes.centre[ids] += shift
    return Update(ids=ids, poses=boxes.poses(ids))


def update_stream(rng: np.random.Generator, boxes: BoxSet, n_updates: int, n_moved: int,
                  planar: bool = False) -> List[Update]:
    state = boxes.copy()
    return [move_boxes(rng, state, n_moved, planar) for _ in range(n_updates)]


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
# Calibrated stand-ins for the large single roadmap: a k=10 PRM over this many
# nodes has ~500k edges, and this step gives ~80 configurations per edge.
LARGE_NODES = 82_000
LARGE_STEP = 0.0118


def _streams(index: int, n: int):
    ss = np.random.SeedSequence(BASE_SEED + index)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


def seven_dof_arm() -> Robot:
    """The 7-DOF arm shared by workloads 2, 3 and 5."""
    (r_robot,) = _streams(2, 1)
    return dh_arm(r_robot, 7)


def workload_planar(n_nodes: int = 500, n_updates: int = 8, index: int = 1) -> Scene:
    r_nodes, r_boxes, r_upd = _streams(index, 3)
    robot = planar_arm()
    roadmap = prm_roadmap(r_nodes, robot, n_nodes, k=6, step=0.05)
    boxes = random_boxes(r_boxes, 16, planar=True, oriented=False)
    ups = update_stream(r_upd, boxes, n_updates, 2, planar=True)
    return Scene("planar3_500n", roadmap, boxes, ups)


def workload_7dof(n_nodes: int = 10_000, n_boxes: int = 64, n_moved: int = 8,
                  step: float = 0.02, n_updates: int = 8, index: int = 2,
                  name: Optional[str] = None) -> Scene:
    _, r_nodes, r_boxes, r_upd = _streams(index, 4)
    robot = seven_dof_arm()
    roadmap = prm_roadmap(r_nodes, robot, n_nodes, k=10, step=step)
    boxes = random_boxes(r_boxes, n_boxes)
    ups = update_stream(r_upd, boxes, n_updates, n_moved)
    return Scene(name or f"dh7_{n_nodes}n", roadmap, boxes, ups)


def workload_large(n_nodes: int = LARGE_NODES, n_updates: int = 8) -> Scene:
    return workload_7dof(n_nodes=n_nodes, n_boxes=256, n_moved=32, step=LARGE_STEP,
                         n_updates=n_updates, index=3, name=f"dh7_large_{n_nodes}n")


def large_mixed_boxes(n_updates: int = 8):
    """Boxes and updates of the mixed-label variant of the large roadmap:
    the same 256 boxes and 32 moves per update as workload 3, but small
    (half-extents U[0.02, 0.06] m) and spread over a 4 m cube, so that green,
    gray and red edges all occur (the surveyed scene leaves every edge red).
    Returns (boxes, updates); the roadmap is workload 3's."""
    rb, ru = [np.random.Generator(np.random.PCG64(s)) for s in
              np.random.SeedSequence([BASE_SEED + 3, 1]).spawn(2)]
    boxes = random_boxes(rb, 256, extent=2.0, half_lo=0.02, half_hi=0.06)
    return boxes, update_stream(ru, boxes, n_updates, 32)


def workload_large_mixed(n_nodes: int = LARGE_NODES, n_updates: int = 8) -> Scene:
    """Workload 3's roadmap (same seed and edges) among large_mixed_boxes."""
    sc = workload_large(n_nodes=n_nodes, n_updates=0)
    boxes, ups = large_mixed_boxes(n_updates)
    return Scene(f"dh7_large_mixed_{n_nodes}n", sc.roadmap, boxes, ups)


def workload_batched(n_roadmaps: int = 128, edge_lo: int = 1_000, edge_hi: int = 100_000,
                     step: float = 0.02, n_updates: int = 4) -> List[Scene]:
    """Independent roadmaps: DOF from {3, 6, 7}, edge counts log-uniform in
    [edge_lo, edge_hi], max-norm edge lengths log-uniform in [9, 399] steps
    (10-400 configurations), 32-256 boxes each, 1-16 moved per update."""
    (r_top,) = _streams(4, 1)
    scenes = []
    for i in range(n_roadmaps):
        rr, re, rb, ru = [np.random.Generator(np.random.PCG64(s)) for s in
                          np.random.SeedSequence([BASE_SEED + 4, i]).spawn(4)]
        dof = int(r_top.choice([3, 6, 7]))
        n_edges = int(round(math.exp(r_top.uniform(math.log(edge_lo), math.log(edge_hi)))))
        n_boxes = int(r_top.integers(32, 257))
        n_moved = int(r_top.integers(1, 17))
        robot = dh_arm(rr, dof)
        roadmap = segment_roadmap(re, robot, n_edges, step, 9.0, 399.0)
        boxes = random_boxes(rb, n_boxes)
        ups = update_stream(ru, boxes, n_updates, n_moved)
        scenes.append(Scene(f"batch{i}_dof{dof}_{n_edges}e", roadmap, boxes, ups))
    return scenes


def workload_serving(node_counts=(8_000, 8_000, 8_000, 8_000, 32_500, 32_500, 32_500, 32_500),
                     rate_hz: float = 2000.0, duration_s: float = 10.0,
                     n_boxes: int = 64):
    """Resident roadmaps (7-DOF, k=10 PRMs; the default node counts give
    ~50k and ~200k edges) with their own 64 OBBs, plus a Poisson stream of
    requests, each moving 1-8 boxes of a uniformly chosen roadmap.
    Returns (scenes without updates, requests in arrival order)."""
    r_req, r_sel = _streams(5, 2)
    robot = seven_dof_arm()
    scenes = []
    for i, n in enumerate(node_counts):
        rn, rb = [np.random.Generator(np.random.PCG64(s)) for s in
                  np.random.SeedSequence([BASE_SEED + 5, i]).spawn(2)]
        roadmap = prm_roadmap(rn, robot, n, k=10, step=0.02)
        scenes.append(Scene(f"serve{i}_{roadmap.num_edges}e", roadmap,
                            random_boxes(rb, n_boxes), []))
    states = [s.boxes.copy() for s in scenes]
    t, reqs = 0.0, []
    while True:
        t += r_req.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        rm = int(r_sel.integers(0, len(scenes)))
        up = move_boxes(r_sel, states[rm], int(r_sel.integers(1, 9)))
        reqs.append(Request(arrival_s=t, roadmap=rm, update=up))
    return scenes, reqs


def workload(index: int, **kw):
    """Workload by its index 1..5 (see the module docstring)."""
    return {1: workload_planar, 2: workload_7dof, 3: workload_large,
            4: workload_batched, 5: workload_serving}[index](**kw)
