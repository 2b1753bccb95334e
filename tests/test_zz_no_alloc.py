"""rgg_classify_noalloc, the entry point for callers that may not allocate
device memory, against the regular classify path.

The caller (this test) owns every device buffer: it copies a roadmap's
records and offsets into its own tensors, keeps the per-edge box sets,
counts and labels, and calls the no-alloc pass twice in a row -- first with
every box placed, then with one update's moved boxes.  After each call the
labels and box sets must equal those of rgg_classify on the same roadmap,
exactly (same arithmetic; the tolerance of the other GPU tests is equality
of labels).  This file is collected last so that a failure here leaves every
other test already run.
"""
import numpy as np
import pytest

from paper_2603_28674_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _padded_planes(torch, planes):
    n = planes.shape[1]
    stride = ((n + 4 + 3) // 4) * 4
    out = torch.zeros((4, stride), dtype=torch.float32, device="cuda")
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    return out


def test_noalloc_two_calls_match_classify():
    torch = pytest.importorskip("torch")
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg

    sc = W.workload_planar(n_updates=2)
    rm, robot = sc.roadmap, sc.roadmap.robot
    n_boxes = sc.boxes.count
    all_ids = np.arange(n_boxes, dtype=np.uint32)
    all_poses = sc.boxes.poses().astype(np.float32)
    up = sc.updates[0]
    up_poses = up.poses.astype(np.float32)

    with rgg.Roadmap(robot.num_links, robot.inner_per_link, n_boxes) as r:
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        inner, outer, soff = r.fetch_records()
        r.update_obstacles(all_ids, all_poses)
        r.classify()
        want = [(r.fetch_labels(), *r.fetch_box_sets())]
        r.update_obstacles(up.ids, up_poses)
        r.classify()
        want.append((r.fetch_labels(), *r.fetch_box_sets()))
        wm = r.info()["mask_words"]

    n = rm.num_edges
    d_soff = torch.from_numpy(soff.astype(np.int64)).cuda()
    d_inner = _padded_planes(torch, inner)
    d_outer = _padded_planes(torch, outer)
    hit = torch.zeros((n, wm), dtype=torch.int32, device="cuda")
    touch = torch.zeros_like(hit)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    labels = torch.zeros(n, dtype=torch.uint8, device="cuda")
    for (ids, poses), (w_lab, w_hit, w_touch) in zip(((all_ids, all_poses), (up.ids, up_poses)),
                                                     want):
        rgg.classify_noalloc(num_links=robot.num_links, inner_per_link=robot.inner_per_link,
                             sample_off=d_soff, num_samples=int(soff[-1]), inner=d_inner,
                             outer=d_outer, box_ids=ids, box_poses=poses, mask_words=wm,
                             hit=hit, touch=touch, counts=counts, labels=labels)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(labels.cpu().numpy(), w_lab)
        np.testing.assert_array_equal(hit.cpu().numpy().view(np.uint32), w_hit)
        np.testing.assert_array_equal(touch.cpu().numpy().view(np.uint32), w_touch)


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
