"""Run the library's autotuner (rgg_autotune) on a seeded workload and print
the timed launch shapes.

For every compiled pipeline variant (ring depth x tile size) and consumer-warp
count, the autotuner times the classify launch on the roadmap's own records
and boxes with CUDA events and keeps the fastest shape; labels are not
changed.

    python -m paper_2603_28674_gb300.tune --workload large [--reps 3]
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def run(workload: str = "7dof", reps: int = 3, log=print):
    from . import build, rgg
    from . import workloads as W

    build.build()
    sc = {"large": W.workload_large, "large_mixed": W.workload_large_mixed,
          "7dof": W.workload_7dof, "planar": W.workload_planar}[workload](n_updates=0)
    rm, robot = sc.roadmap, sc.roadmap.robot
    with rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count) as r:
        r.build_edges(robot, rm.q_from, rm.q_to, rm.step)
        r.update_obstacles(np.arange(sc.boxes.count), sc.boxes.poses().astype(np.float32))
        r.classify()
        rb = r.info()["record_bytes"]
        res = rgg.autotune([r], reps=reps)
        for row in res:
            row["record_gbs"] = rb / (row["classify_ms"] / 1e3) / 1e9
            log(json.dumps(row))
        log(json.dumps({"best": res[0] if res else None, "workload": workload,
                        "record_bytes": rb, "tile_samples": r.info()["tile_samples"]}))
        r.check_status()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="7dof", choices=["large", "large_mixed", "7dof", "planar"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    run(a.workload, a.reps)


if __name__ == "__main__":
    main()
