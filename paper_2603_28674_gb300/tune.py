"""Sweep the classify kernel's launch shapes on a seeded workload.

For every compiled pipeline variant (ring depth x tile size) and a range of
consumer-warp counts, time classification passes (one update + classify per
step, device-resident poses) with CUDA events and report the classify
kernel's time and its record bandwidth.  Labels are checked to be the same
for every shape.

    python -m paper_2603_28674_gb300.tune --workload large [--steps 20]

Prints one line per shape and the fastest one; `--set-default` is not
offered: the library's default is compiled in (see rgg_set_launch_shape).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def sweep(workload: str = "7dof", steps: int = 20, warps=(16, 20, 24, 27), variants=None,
          log=print):
    import torch

    from . import build, rgg
    from . import workloads as W

    build.build()
    sc = {"large": W.workload_large, "7dof": W.workload_7dof,
          "planar": W.workload_planar}[workload](n_updates=32)
    rm, robot = sc.roadmap, sc.roadmap.robot
    r = rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count)
    r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
    r.update_obstacles(np.arange(sc.boxes.count), sc.boxes.poses().astype(np.float32))
    r.classify()
    dev = [torch.from_numpy(u.poses.astype(np.float32)).cuda() for u in sc.updates]
    ids = [u.ids for u in sc.updates]
    rb = r.info()["record_bytes"]
    results, ref = [], None
    for v in (variants if variants is not None else range(rgg.NUM_VARIANTS)):
        for cw in warps:
            try:
                r.set_launch_shape(v, cw)
            except rgg.RGGError:
                continue
            # every shape replays the same updates from the same state
            for i in range(3):
                r.update_obstacles(ids[i], dev[i])
                r.classify()
            torch.cuda.synchronize()
            r.set_kernel_timing(True)
            r.kernel_time()
            for i in range(steps):
                k = 3 + i % 29
                r.update_obstacles(ids[k], dev[k])
                r.classify()
            ms, mm, n = r.kernel_time()
            r.set_kernel_timing(False)
            # return to the state after update 2 so the next shape starts alike
            for k in list(range(3, 32)) + [0, 1, 2]:
                r.update_obstacles(ids[k], dev[k])
            r.classify()
            lab = r.fetch_labels()
            if ref is None:
                ref = lab
            same = bool(np.array_equal(lab, ref))
            row = {"variant": v, "consumer_warps": cw, "classify_ms": ms / n,
                   "record_gbs": rb / (ms / n / 1e3) / 1e9, "tile_samples": r.info()["tile_samples"],
                   "labels_match": same}
            results.append(row)
            log(json.dumps(row))
    r.check_status()
    r.close()
    best = min(results, key=lambda x: x["classify_ms"])
    log(json.dumps({"best": best, "workload": workload, "record_bytes": rb}))
    if not all(x["labels_match"] for x in results):
        raise RuntimeError("labels differ between launch shapes")
    return results


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="7dof", choices=["large", "7dof", "planar"])
    ap.add_argument("--steps", type=int, default=20)
    a = ap.parse_args()
    sweep(a.workload, a.steps)


if __name__ == "__main__":
    main()
