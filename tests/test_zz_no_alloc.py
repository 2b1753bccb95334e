"""rgg_classify_noalloc, the entry point for callers that may not allocate
device memory, against the regular classify path and the FP64 oracle.

The caller (this test) owns every device buffer: it copies a roadmap's
records and offsets into its own tensors, keeps the per-edge box sets,
counts and labels, and calls the no-alloc pass several times in a row --
first placing every box, 32 per call, then with one update's moved boxes.  With the records
flagged as built by rgg_build_edges (regular_records), the pass makes the
same decisions as rgg_classify, so after each call its labels and box sets
must equal rgg_classify's exactly; they must also meet the rule every GPU
test applies against the oracle (equal labels on edges whose clearance
exceeds 1e-4 m, any other difference GPU gray).  Without the flag the pass
tests sphere by sphere and must still meet the oracle rule.  A wait limit of
1 ns makes the pass give up: it must report that through its status word and
leave the caller's state as it was.  This file is collected last so that a
failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_2603_28674_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PIN = 1e-4


def _padded_planes(torch, planes):
    n = planes.shape[1]
    stride = ((n + 4 + 3) // 4) * 4
    out = torch.zeros((4, stride), dtype=torch.float32, device="cuda")
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    return out


def _scene(which):
    if which == "planar":
        return W.workload_planar(n_updates=2)
    return W.workload_7dof(n_nodes=500, n_updates=2)


class _Caller:
    """Device buffers a caller without an allocator of its own would hold."""

    def __init__(self, torch, r, rm):
        inner, outer, soff = r.fetch_records()
        self.wm = r.info()["mask_words"]
        n = rm.num_edges
        self.num_samples = int(soff[-1])
        self.soff = torch.from_numpy(soff.astype(np.int64)).cuda()
        self.inner = _padded_planes(torch, inner)
        self.outer = _padded_planes(torch, outer)
        self.hit = torch.zeros((n, self.wm), dtype=torch.int32, device="cuda")
        self.touch = torch.zeros_like(self.hit)
        self.counts = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.labels = torch.zeros(n, dtype=torch.uint8, device="cuda")
        self.status = torch.full((1,), -7, dtype=torch.int32, device="cuda")

    def call(self, rgg, robot, ids, poses, regular, wait_limit_ns=0):
        rgg.classify_noalloc(num_links=robot.num_links, inner_per_link=robot.inner_per_link,
                             sample_off=self.soff, num_samples=self.num_samples,
                             inner=self.inner, outer=self.outer, box_ids=ids, box_poses=poses,
                             mask_words=self.wm, hit=self.hit, touch=self.touch,
                             counts=self.counts, labels=self.labels,
                             regular_records=regular, status=self.status,
                             wait_limit_ns=wait_limit_ns)

    def state(self):
        return (self.labels.cpu().numpy(), self.hit.cpu().numpy().view(np.uint32),
                self.touch.cpu().numpy().view(np.uint32), self.counts.cpu().numpy())


def _check_oracle(labels, hit, touch, want, where):
    pinned = want["kappa"] > PIN
    bad = np.flatnonzero(pinned & (labels != want["labels"]))
    assert bad.size == 0, f"{where}: {bad.size} pinned edges differ from the oracle"
    off = labels != want["labels"]
    assert np.all(labels[off] == oracle.GRAY), f"{where}: disagreement other than GPU gray"
    w = want["hit"].shape[1]
    assert np.all((hit[:, :w] & ~want["hit"]) == 0), f"{where}: hit outside the oracle's"
    assert np.all((want["touch"] & ~touch[:, :w]) == 0), f"{where}: oracle touch missing"


@pytest.mark.parametrize("which", ["planar", "7dof"])
def test_noalloc_two_calls_match_classify_and_the_oracle(which):
    torch = pytest.importorskip("torch")
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg

    sc = _scene(which)
    rm, robot = sc.roadmap, sc.roadmap.robot
    n_boxes = sc.boxes.count
    boxes = sc.boxes.copy()
    up = sc.updates[0]
    # a call tests at most 32 boxes: the initial placement takes one call per
    # 32 ids, as rgg_classify takes one pass per 32 pending boxes
    steps = [(np.arange(a, min(a + 32, n_boxes), dtype=np.uint32),
              boxes.poses()[a:a + 32].astype(np.float32)) for a in range(0, n_boxes, 32)]
    steps.append((up.ids, up.poses.astype(np.float32)))

    # sphere records: the layout the allocation-free pass reads
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, n_boxes,
                     record_format=rgg.RECORDS_SPHERES) as r:
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        regular = _Caller(torch, r, rm)
        exact = _Caller(torch, r, rm)
        want = []
        for ids, poses in steps:
            r.update_obstacles(ids, poses)
            r.classify()
            want.append((r.fetch_labels(), *r.fetch_box_sets()))

    for k, ((ids, poses), (w_lab, w_hit, w_touch)) in enumerate(zip(steps, want)):
        regular.call(rgg, robot, ids, poses, True)
        exact.call(rgg, robot, ids, poses, False)
        torch.cuda.synchronize()
        if k == len(steps) - 1:
            boxes.centre[up.ids] = up.poses[:, :3]
        placed = np.zeros(n_boxes, dtype=bool)
        placed[:min(n_boxes, 32 * (k + 1))] = True
        ref = oracle.classify(robot, rm.q_from, rm.q_to, rm.step, boxes.poses(), bits=True,
                              present=placed)
        lab, hit, touch, _ = regular.state()
        assert int(regular.status.item()) == 0
        np.testing.assert_array_equal(lab, w_lab)
        np.testing.assert_array_equal(hit, w_hit)
        np.testing.assert_array_equal(touch, w_touch)
        _check_oracle(lab, hit, touch, ref, f"{which} call {k}, regular")
        lab, hit, touch, _ = exact.state()
        assert int(exact.status.item()) == 0
        _check_oracle(lab, hit, touch, ref, f"{which} call {k}, sphere by sphere")


def test_noalloc_wait_that_runs_out_leaves_the_callers_state():
    torch = pytest.importorskip("torch")
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg

    sc = _scene("7dof")
    rm, robot = sc.roadmap, sc.roadmap.robot
    ids = np.arange(sc.boxes.count, dtype=np.uint32)
    poses = sc.boxes.poses().astype(np.float32)
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count,
                     record_format=rgg.RECORDS_SPHERES) as r:
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        c = _Caller(torch, r, rm)
        r.update_obstacles(ids, poses)
        r.classify()
        want = r.fetch_labels()
    for a in range(0, len(ids), 32):                     # normal calls place every box
        c.call(rgg, robot, ids[a:a + 32], poses[a:a + 32], True)
    torch.cuda.synchronize()
    first = c.state()
    np.testing.assert_array_equal(first[0], want)
    up = sc.updates[0]
    gave_up = False
    for _ in range(4):
        before = c.state()
        c.call(rgg, robot, up.ids, up.poses.astype(np.float32), True, wait_limit_ns=1)
        torch.cuda.synchronize()
        if int(c.status.item()) != 0:
            gave_up = True
            for a, b in zip(c.state(), before):      # nothing of the pass was merged
                np.testing.assert_array_equal(a, b)
            break
    assert gave_up, "no bounded wait ran out at a 1 ns limit"
    c.call(rgg, robot, up.ids, up.poses.astype(np.float32), True)   # the retry works
    torch.cuda.synchronize()
    assert int(c.status.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pytest.importorskip("torch")
    from paper_2603_28674_gb300 import rgg
    import torch
    n = rgg.NOALLOC_MAX_EDGES + 1
    labels = torch.empty(n, dtype=torch.uint8, device="cuda")
    planes = torch.empty((4, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(rgg.RGGError) as err:
        rgg.classify_noalloc(num_links=3, inner_per_link=4, sample_off=labels, num_samples=2 * n,
                             inner=planes, outer=planes, box_ids=[0],
                             box_poses=np.eye(1, 15, dtype=np.float32), mask_words=1, hit=labels,
                             touch=labels, counts=labels, labels=labels)
    assert err.value.status == rgg.RGG_ERR_CAPACITY
