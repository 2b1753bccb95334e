"""Benchmark of the RGG edge-classification pass on GB300.

One step = one obstacle update (the update's moved boxes written into the
device box table) followed by one classification of every roadmap edge
against the moved boxes, merged into the per-edge box sets and labels.

Default workload: the large single roadmap (7-DOF DH arm, ~500k edges,
~80 configurations per edge, ~27 GB of FP32 sphere records resident in HBM,
256 oriented boxes, 32 moved per update).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|7dof|planar]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the same metric

Prints one JSON line (rank 0).  For N > 1 (launched by torch.distributed.run)
every rank runs an independent replica on its own GPU: the edges are not
sharded and no collective touches the data path (barrier and max-over-ranks
timing only).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import re
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2603_28674_gb300 import workloads as W  # noqa: E402

METRIC = "RGG edges classified/s"
UNIT = "edges/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "classify_kernel_traffic.txt")
KERNEL_HEADERS = [os.path.join(ROOT, "paper_2603_28674_gb300", "csrc", f)
                  for f in ("rgg_device.cuh", "rgg_kernels.h")]
KERNEL_FILE = os.path.join(ROOT, "paper_2603_28674_gb300", "csrc", "rgg_kernels.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "7dof", "planar", "batched", "serve"])
    ap.add_argument("--roadmaps", type=int, default=128, help="batched workload: roadmaps")
    ap.add_argument("--geometry", default="spheres", choices=["spheres", "obb"],
                    help="obb: time the paper's OBB / spline geometry beside the sphere one "
                         "on the same roadmap and updates")
    ap.add_argument("--persist", action="store_true",
                    help="also time rgg_save / rgg_load of the roadmap through a temporary file")
    ap.add_argument("--resolve", type=int, default=0, metavar="F",
                    help="also time the non-lazy resolution of the gray edges at F-times "
                         "finer resampling (0: off)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="serving: seconds of Poisson arrivals at 2000 requests/s")
    ap.add_argument("--serve-stress-rate", type=float, default=16000.0,
                    help="serving: a second, shorter stream at this rate (requests/s), above "
                         "what one request per launch sustains; 0: off")
    ap.add_argument("--serve-stress-seconds", type=float, default=2.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the mixed-label scene and the batched and "
                         "serving measurements that follow the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def make_scene(name: str, n_updates: int):
    if name == "large":
        return W.workload_large(n_updates=n_updates)
    if name == "7dof":
        return W.workload_7dof(n_updates=n_updates)
    if name == "batched":
        # the oracle's sample: the largest roadmap of the batch, its own updates
        scenes = W.workload_batched(n_updates=max(1, min(n_updates, 8)))
        return max(scenes, key=lambda x: x.roadmap.num_edges)
    if name == "serve":
        # the oracle's sample: a ~200k-edge resident roadmap and the updates
        # the request stream sends it
        scenes, reqs = W.workload_serving(duration_s=2.0)
        k = len(scenes) - 1
        ups = [q.update for q in reqs if q.roadmap == k][:max(1, n_updates)]
        sc = scenes[k]
        return W.Scene(sc.name, sc.roadmap, sc.boxes, ups)
    return W.workload_planar(n_updates=n_updates)


def workload_config(name: str, sc, world: int = 1) -> dict:
    """The workload's description, the same for the GPU arm and the oracle's
    reference arm (only what the inputs fix, nothing measured)."""
    rm = sc.roadmap
    moved = len(sc.updates[0].ids) if sc.updates else 0
    cfg = {
        "workload": {"large": "large single roadmap", "7dof": "7-DOF 10k-node roadmap",
                     "planar": "planar 3-link 500-node roadmap",
                     "batched": "largest roadmap of the 128-roadmap batch",
                     "serve": "one ~200k-edge roadmap of the serving set"}[name],
        "robot": f"{rm.robot.num_links}-link DH arm, {rm.robot.inner_per_link} inner spheres/link",
        "edges": rm.num_edges,
        "step_rad": rm.step,
        "boxes": sc.boxes.count,
        "moved_per_update": moved,
        "record_dtype": "fp32",
        "l2": "records > L2 (129 MB); no flush needed",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }
    return cfg


def _code_only(src: bytes) -> bytes:
    """C++ source without // comments and with runs of blank space
    collapsed: edits to comments do not change what is compiled."""
    out = re.sub(rb"//[^\n]*", b"", src)
    return re.sub(rb"\s+", b" ", out).strip()


def kernel_sha() -> str:
    """Hash of the code classify_kernel is compiled from: the two kernel
    headers and the classify section of rgg_kernels.cu (from its a2..a5
    banner to the a6 banner) without the spatial filter's own kernels inside
    it, comments left out, so that edits to the other kernels or to comments
    do not invalidate the traffic profile."""
    h = hashlib.sha256()
    for p in KERNEL_HEADERS:
        h.update(_code_only(open(p, "rb").read()))
    t = open(KERNEL_FILE, "rb").read()
    a = t.index(b"// a2..a5: persistent streaming classification")
    sec = t[a:t.index(b"// a6: merge", a)]
    f0 = sec.index(b"// Spatial filter (Sec. 4.3)")
    f1 = sec.index(b"// Bound of the final wait for the CTA's own bulk copies", f0)
    h.update(_code_only(sec[:f0]))
    h.update(_code_only(sec[f1:]))
    return h.hexdigest()[:16]


def profiled_counters(workload: str) -> dict:
    """ncu counters of one classify launch from the committed summary
    (bytes_per_launch, and when recorded inst_per_launch and issue_active),
    or an empty dict when it is missing, for another workload, or the kernel
    changed since."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return {}
    kv = {}
    for line in open(PROFILE_TRAFFIC):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sha") != kernel_sha() or kv.get("workload") != workload:
        return {}
    out = {}
    for k in ("bytes_per_launch", "inst_per_launch", "issue_active"):
        try:
            out[k] = float(kv[k])
        except (KeyError, ValueError):
            pass
    return out


def profiled_traffic(workload: str):
    """DRAM bytes per classify launch from the committed ncu summary (None
    when it does not apply)."""
    return profiled_counters(workload).get("bytes_per_launch")


def issue_roofline(counters: dict, k_ms: float, sm_mhz, num_sms: int):
    """The classify kernel against the schedulers' issue rate: ncu's warp
    instructions per launch over the live launch time, against one warp
    instruction per cycle on each of an SM's 4 schedulers at the sampled SM
    clock.  None without counters or a clock sample."""
    inst = counters.get("inst_per_launch")
    if not inst or not sm_mhz or k_ms <= 0:
        return None
    peak = num_sms * 4 * sm_mhz * 1e6
    achieved = inst / (k_ms / 1000.0)
    return {"warp_instructions_per_launch": inst, "achieved_warp_inst_per_s": achieved,
            "peak_warp_inst_per_s": peak, "frac": achieved / peak,
            "issue_active_ncu": counters.get("issue_active"),
            "note": "instructions from the committed ncu summary (classify kernel only); time "
                    "is the live classify interval, which includes the round filter"}


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
         "clocks.mem,temperature.gpu")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.skip = 0     # rows written before the timed region started
        self.path = os.path.join("/tmp", f"rgg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return self
        # start timing only once the sampler is writing (at most 3 s), so a
        # short timed region still gets its samples
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        self.skip = 1 if os.path.getsize(self.path) > 0 else 0
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, mem, power = [], [], set(), [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [[x.strip() for x in line.split(",")] for line in open(self.path)]
        rows = [f for f in rows if len(f) >= 9]
        if len(rows) > self.skip:
            rows = rows[self.skip:]
        for f in rows:
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
                if len(f) > 9:
                    mem.append(float(f[9]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
               "reasons": sorted(reasons), "samples": len(sm),
               "power_w_median": float(np.median(power)) if power else None}
        if mem:
            out["mem_mhz"] = float(np.median(mem))
        return out


ROUND_SLOT_BYTES = 16 + 4 + 4 + 4   # per (tile, round) slot: sphere, candidates written + read, range
TILE_LIST_BYTES = 4 + 4 + 16        # per tile: its list entry written and read, its sphere read


def algorithmic_bytes(info: dict, record_bytes_per_launch=None) -> int:
    """Bytes one classify launch must move: the records it copies
    (unfiltered: every record once, 12 B per link end or 16 B per inner
    sphere, 16 B per outer sphere; with the spatial filter: the rounds some
    moved box may reach, as counted on the device), each edge's pass result (hit and touch words, 8 B) and,
    with the filter, its per-round data (bounding sphere read, candidate
    mask written and read, record range read), its tile spheres and its tile
    list.  Tile
    descriptors, edge tables and the moved boxes' records are overhead and
    not counted."""
    if record_bytes_per_launch is None or not info.get("round_filter"):
        return info["record_bytes"] + 8 * info["num_edges"]
    return (int(record_bytes_per_launch) + 8 * info["num_edges"]
            + (ROUND_SLOT_BYTES * 32 + TILE_LIST_BYTES) * info["num_tiles"])


# --------------------------------------------------------------------------
# CPU oracle timing
# --------------------------------------------------------------------------
def oracle_rate(sc, seconds: float, seed: int = 0):
    """Edges/s of the FP64 oracle classifying a random sample of the
    workload's edges against the boxes moved in one update, on all host
    cores: a short calibration run, then runs sized to fill `seconds`."""
    import oracle
    rm = sc.roadmap
    up = sc.updates[0]
    rng = np.random.default_rng(seed)
    total_e, total_t, n = 0, 0.0, 256
    for _ in range(3):
        idx = rng.choice(rm.num_edges, size=min(n, rm.num_edges), replace=False)
        t0 = time.perf_counter()
        oracle.classify(rm.robot, rm.q_from[idx], rm.q_to[idx], rm.step, up.poses)
        dt = time.perf_counter() - t0
        total_e += idx.size
        total_t += dt
        left = seconds - total_t
        if left <= 0.1 * seconds or idx.size == rm.num_edges:
            break
        n = int(min(rm.num_edges, max(64, idx.size * left / max(dt, 1e-4))))
    return total_e / total_t, total_e, total_t, oracle.max_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sc = make_scene(args.workload, n_updates=max(1, args.warmup + args.steps))
    import oracle
    rm = sc.roadmap
    rng = np.random.default_rng(1)
    # size each step so that the whole run takes about two and a half minutes
    rate, _, _, _ = oracle_rate(sc, 3.0)
    budget = 150.0 / max(1, args.steps + args.warmup)
    per_step = int(max(16, min(rm.num_edges, rate * budget)))
    times = []
    for i in range(args.warmup + args.steps):
        up = sc.updates[i % len(sc.updates)]
        idx = rng.choice(rm.num_edges, size=per_step, replace=False)
        t0 = time.perf_counter()
        oracle.classify(rm.robot, rm.q_from[idx], rm.q_to[idx], rm.step, up.poses)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(sum(times))
    value = per_step * args.steps / t
    sample = (f"{per_step} random edges per step, each classified from its endpoints against "
              f"the {len(sc.updates[0].ids)} boxes one update moves (FP64, OpenMP over edges)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, sc, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# replicas (N > 1): barrier + max-over-ranks timing, no data-path collective
# --------------------------------------------------------------------------
def max_over_ranks(dist, x: float, device=None) -> float:
    """The largest x over all ranks (x itself without a process group).  NCCL
    reduces a CUDA tensor on `device`; other backends a CPU tensor."""
    if dist is None:
        return float(x)
    import torch
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, units_per_rank: float, slowest_s: float) -> float:
    """Whole-job rate of `world` replicas that each processed units_per_rank
    units, timed by the slowest rank (weak scaling)."""
    return world * units_per_rank / slowest_s


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gpu(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg

    n_ups = 64
    sc = make_scene(args.workload, n_updates=n_ups)
    rm, robot = sc.roadmap, sc.roadmap.robot
    moved = len(sc.updates[0].ids)
    stream = torch.cuda.current_stream()
    r = rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count, device=local)
    r.build_edges(robot, rm.q_from, rm.q_to, rm.step, stream)
    r.update_obstacles(np.arange(sc.boxes.count), sc.boxes.poses().astype(np.float32), stream)
    r.classify(stream)
    info = r.info()

    # device-resident update inputs for the device-timed loop
    dev_poses = [torch.from_numpy(u.poses.astype(np.float32)).to(f"cuda:{local}")
                 for u in sc.updates]
    ids = [u.ids for u in sc.updates]
    # pinned host buffers for the end-to-end loop
    host_poses = [torch.from_numpy(u.poses.astype(np.float32)).pin_memory().numpy()
                  for u in sc.updates]
    labels_host = torch.empty(info["num_edges"], dtype=torch.uint8).pin_memory().numpy()

    def device_step(i):
        k = i % n_ups
        r.update_obstacles(ids[k], dev_poses[k], stream)
        r.classify(stream)

    for i in range(args.warmup):
        device_step(i)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM, records 27 GB >> L2
    r.set_kernel_timing(True)
    r.kernel_time()
    r.streamed_bytes()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for i in range(args.steps):
            device_step(args.warmup + i)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    k_ms, m_ms, k_launches = r.kernel_time()
    r.set_kernel_timing(False)
    streamed = r.streamed_bytes()
    ms = max_over_ranks(dist, ms, f"cuda:{local}")
    clk = clocks.summary()
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- end to end through the C ABI with host buffers
    for i in range(min(args.warmup, 3)):
        k = i % n_ups
        r.update_obstacles(ids[k], host_poses[k], stream)
        r.classify(stream)
        r.fetch_labels(out=labels_host, stream=stream)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        k = (args.warmup + i) % n_ups
        r.update_obstacles(ids[k], host_poses[k], stream)
        r.classify(stream)
        r.fetch_labels(out=labels_host, stream=stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s, f"cuda:{local}")
    # ---- the same steps with the spatial filter in its other state (after
    # the end-to-end loop): the headline runs the library's default (the
    # filter on for link-end records), this one streams every record, or the
    # other way round
    filtered = None
    default_on = bool(info["round_filter"])
    r.set_round_filter(not default_on)
    if bool(r.info()["round_filter"]) != default_on:
        n_cmp = min(args.steps, 100)
        for i in range(3):
            device_step(2 * args.steps + args.warmup + i)
        torch.cuda.synchronize()
        r.set_kernel_timing(True)
        r.kernel_time()
        r.streamed_bytes()
        for i in range(n_cmp):
            device_step(2 * args.steps + args.warmup + 3 + i)
        torch.cuda.synchronize()
        kf_ms, _, kf_n = r.kernel_time()
        r.set_kernel_timing(False)
        sf = r.streamed_bytes()
        filtered = {"kernel_ms": kf_ms / max(1, kf_n),
                    "record_bytes_per_launch": sf / max(1, kf_n), "launches": kf_n,
                    "info": r.info()}
    r.set_round_filter(default_on)

    # ---- the work the kernel executed, from its counting instance, over a
    # few more of the same steps (the headline instance counts nothing)
    r.set_work_counting(True)
    r.work_counts()
    n_cnt = 3
    for i in range(n_cnt):
        device_step(2 * args.steps + args.warmup + i)
    executed = r.work_counts()
    r.set_work_counting(False)

    r.check_status(stream)
    resolve = measure_resolve(r, sc, args.resolve, stream, rank == 0 and world == 1) \
        if args.resolve else None
    persist = measure_persist(r, robot, sc.boxes.count, stream) if args.persist else None

    n_edges = info["num_edges"]
    value = replica_throughput(world, n_edges * args.steps, ms / 1000.0)
    e2e_value = replica_throughput(world, n_edges * args.steps, e2e_s)
    peak, peak_kind = hbm_peak()
    k_avg_ms = k_ms / max(1, k_launches)
    rec_per_launch = streamed / max(1, k_launches)
    b_alg = algorithmic_bytes(info, rec_per_launch)
    achieved = b_alg / (k_avg_ms / 1000.0) / 1e9
    counters = profiled_counters(args.workload)
    traffic = counters.get("bytes_per_launch")
    filt = None
    if filtered is not None:
        on = bool(filtered["info"]["round_filter"])
        rb = filtered["record_bytes_per_launch"] if on else info["record_bytes"]
        b_f = algorithmic_bytes(filtered["info"], filtered["record_bytes_per_launch"])
        filt = {"round_filter": on, "kernel_ms": filtered["kernel_ms"],
                "record_bytes_per_launch": rb,
                "records_copied_frac": rb / info["record_bytes"],
                "bytes_per_launch": b_f,
                "frac": b_f / (filtered["kernel_ms"] / 1000.0) / 1e9 / peak,
                "edges_per_s": n_edges / (filtered["kernel_ms"] / 1000.0),
                "headline_speedup": filtered["kernel_ms"] / k_avg_ms,
                "note": "the same steps with the spatial filter (rgg_set_round_filter) in the "
                        "state the headline does not use; with the filter the kernel interval "
                        "holds the round-filter kernel and the bytes are those copied"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rate, n_s, t_s, cores = oracle_rate(sc, args.cpu_seconds)
        # the same oracle on one thread, on a shorter sample
        oracle.set_threads(1)
        try:
            rate1, n_1, t_1, _ = oracle_rate(sc, max(1.0, args.cpu_seconds / 3), seed=1)
        finally:
            oracle.set_threads(cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"{n_s} random edges classified from their endpoints against the "
                          f"{moved} boxes one update moves (FP64, OpenMP over edges), "
                          f"{t_s:.1f} s"),
               "single_thread_value": rate1,
               "single_thread_sample": f"{n_1} random edges, {t_1:.1f} s, one thread"}

    cfg = workload_config(args.workload, sc, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "sizes": {"samples": info["num_samples"], "record_gb": info["record_bytes"] / 1e9,
                  "tile_samples": info["tile_samples"], "grid_ctas": info["grid_ctas"]},
        # every (sphere, moved box) pair the definition asks about; the kernel
        # culls most of them per warp before an exact test
        "sphere_box_tests_per_s": {
            "logical": world * (info["num_inner"] + info["num_outer"]) * moved
            * args.steps / (ms / 1000.0),
            "note": "(inner + outer spheres) x moved boxes per update, per second; the "
                    "kernel culls most of them per warp, see executed_per_launch"},
        "executed_per_launch": {
            "rounds": executed["rounds"] / n_cnt,
            "outer_sphere_box_tests": executed["outer_tests"] / n_cnt,
            "inner_pairs": executed["inner_pairs"] / n_cnt,
            "inner_sphere_box_tests_max": executed["inner_pairs"] * info["inner_per_link"] / n_cnt,
            "logical_sphere_box_tests": (info["num_inner"] + info["num_outer"]) * moved,
            "note": "from the classify kernel's counting instance over %d further steps; an "
                    "inner pair is one (configuration, box) pair, up to K sphere tests" % n_cnt},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     # ncu-measured DRAM bytes per launch over the live launch time
                     "traffic_frac": (traffic / (k_avg_ms / 1000.0) / 1e9 / peak
                                      if traffic else None),
                     "peak_source": f"{peak_kind} HBM copy bandwidth",
                     "kernel": "classify_kernel", "bytes_per_launch": b_alg,
                     "kernel_ms": k_avg_ms,
                     "merge_kernel_ms": m_ms / max(1, k_launches),
                     # the bound the dense scene actually meets: instruction issue
                     "issue": issue_roofline(counters, k_avg_ms, clk.get("sm_mhz"),
                                             num_sms)},
        "round_filter_used": bool(info["round_filter"]),
        "other_filter_state": filt,
        # label mix after the end-to-end steps (the paper's roadmaps: 0.3-10% gray)
        "labels": {"green": float(np.mean(labels_host == 0)), "gray": float(np.mean(labels_host == 1)),
                   "red": float(np.mean(labels_host == 2))},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": moved * (4 + 60),
                "d2h_bytes_per_step": n_edges + 4},
        # per step: box update, box prep, (round filter,) classify, merge
        "gpu_launches": (5 if info["round_filter"] else 4) * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if resolve is not None:
        line["resolve"] = resolve
    if persist is not None:
        line["persist"] = persist
    extras = (args.workload == "large" and world == 1 and not args.no_extras)
    if extras:
        line["mixed_scene"] = measure_mixed(r, args, stream, peak)
    r.close()
    del dev_poses
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if extras:
        # the latency half of the metric: the batched form (workload 4) and
        # the served form (workload 5) against one launch per update
        with ClockSampler(local) as clk_b:
            line["batched"] = measure_batched(args, args.steps, max(3, args.warmup),
                                              args.roadmaps)
        line["batched"]["clocks"] = clk_b.summary()
        with ClockSampler(local) as clk_s:
            line["serving"] = measure_serving(args, args.serve_seconds)
        line["serving"]["clocks"] = clk_s.summary()
        if args.serve_stress_rate > 0:
            with ClockSampler(local) as clk_t:
                line["serving_stress"] = measure_serving(args, args.serve_stress_seconds,
                                                         args.serve_stress_rate)
            line["serving_stress"]["clocks"] = clk_t.summary()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_mixed(r, args, stream, peak: float) -> dict:
    """The same roadmap among the mixed-label boxes (256 small boxes spread
    over a 4 m cube, 32 moved per update): every box is placed at its new
    pose, then K updates are timed like the headline, with the library's
    default configuration and again with the spatial filter in its other
    state.  The labels must be the same both ways."""
    import torch
    boxes, ups = W.large_mixed_boxes(n_updates=max(8, args.warmup + args.steps))
    dev = [torch.from_numpy(u.poses.astype(np.float32)).to(stream.device) for u in ups]
    r.update_obstacles(np.arange(boxes.count), boxes.poses().astype(np.float32), stream)
    r.classify(stream)

    def step(i):
        r.update_obstacles(ups[i % len(ups)].ids, dev[i % len(ups)], stream)
        r.classify(stream)

    def timed(n_warm):
        # the updates of the timed steps (absolute poses: the final state,
        # and the labels, are the same whichever run came first)
        for i in range(n_warm):
            step(args.warmup + i)
        torch.cuda.synchronize()
        r.set_kernel_timing(True)
        r.kernel_time()
        r.streamed_bytes()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
        k_ms, m_ms, n = r.kernel_time()
        r.set_kernel_timing(False)
        info = r.info()
        rec = r.streamed_bytes() / max(1, n) if info["round_filter"] else info["record_bytes"]
        lab = r.fetch_labels(stream=stream)
        k_avg = k_ms / max(1, n)
        b_alg = algorithmic_bytes(info, rec)
        mix = np.bincount(lab, minlength=3) / max(1, lab.size)
        return {"round_filter": bool(info["round_filter"]), "ms_per_step": e0.elapsed_time(e1) / args.steps,
                "edges_per_s": info["num_edges"] * args.steps / (e0.elapsed_time(e1) / 1e3),
                "kernel_ms": k_avg, "merge_kernel_ms": m_ms / max(1, n),
                "record_bytes_per_launch": rec, "records_copied_frac": rec / info["record_bytes"],
                "bytes_per_launch": b_alg, "achieved_gbs": b_alg / (k_avg / 1e3) / 1e9,
                "frac": b_alg / (k_avg / 1e3) / 1e9 / peak,
                "labels": {"green": float(mix[0]), "gray": float(mix[1]), "red": float(mix[2])}}, lab

    out, lab = timed(args.warmup)
    out.update({"boxes": "256, half-extents U[0.02, 0.06] m, centres in a 4 m cube",
                "moved_per_update": 32, "steps": args.steps})
    default_on = out["round_filter"]
    r.set_round_filter(not default_on)
    if r.info()["round_filter"] != default_on:
        other, lab_o = timed(min(3, args.steps))
        other["labels_identical"] = bool(np.array_equal(lab_o, lab))
        other["headline_speedup"] = other["kernel_ms"] / out["kernel_ms"]
        other["note"] = ("the same steps with the spatial filter in the state the headline "
                         "does not use")
        out["other_filter_state"] = other
    r.set_round_filter(default_on)
    # the library's autotuner on this scene: it times every compiled launch
    # shape on the roadmap's own records (a pass of its first 32 present
    # boxes at their current poses, into its own accumulators) and keeps the
    # fastest.  The boxes go back to the scene's initial poses first: after
    # hundreds of random-walk updates the first 32 may have drifted out of
    # the robot's reach, and a pass of them would stand for nothing.  The
    # same steps then run at the chosen shape (absolute poses: the same final
    # state), and the labels must not change
    from paper_2603_28674_gb300 import rgg
    r.update_obstacles(np.arange(boxes.count), boxes.poses().astype(np.float32), stream)
    r.classify(stream)
    tuned = rgg.autotune([r], reps=3, stream=stream)
    if tuned:
        at, lab_a = timed(min(3, args.steps))
        at["chosen"] = tuned[0]
        at["shapes_timed"] = len(tuned)
        at["labels_identical"] = bool(np.array_equal(lab_a, lab))
        at["speedup_vs_default"] = out["kernel_ms"] / at["kernel_ms"]
        at["note"] = ("the same steps at the launch shape rgg_autotune picked for this scene; the "
                      "headline and the entries above run the library's default shape")
        out["autotuned"] = at
    r.check_status(stream)
    return out


def measure_persist(r, robot, m: int, stream) -> dict:
    """Save the roadmap to a temporary file and load it into a second roadmap
    (wall time of each call); the reloaded labels must equal the original's."""
    import tempfile
    from paper_2603_28674_gb300 import rgg
    info = r.info()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "roadmap.rgg")
        t0 = time.perf_counter()
        r.save(path, stream)
        t_save = time.perf_counter() - t0
        size = os.path.getsize(path)
        with rgg.Roadmap(robot.num_links, robot.inner_per_link, m) as b:
            t0 = time.perf_counter()
            b.load(path, stream)
            t_load = time.perf_counter() - t0
            same = bool(np.array_equal(b.fetch_labels(stream=stream), r.fetch_labels(stream=stream)))
    return {"file_gb": size / 1e9, "record_gb": info["record_bytes"] / 1e9,
            "save_s": t_save, "load_s": t_load, "save_gbs": size / t_save / 1e9,
            "load_gbs": size / t_load / 1e9, "labels_identical": same}


def measure_resolve(r, sc, factor: int, stream, with_oracle: bool) -> dict:
    """Time rgg_resolve_gray on the roadmap's current state (one warm-up, then
    three timed calls with CUDA events on the stream), and the oracle's dense
    clearance on a sample of the same gray edges."""
    import torch
    from paper_2603_28674_gb300 import rgg
    n = r.info()["num_edges"]
    out = torch.empty(n, dtype=torch.uint8, device=stream.device)
    clear = torch.empty(n, dtype=torch.float32, device=stream.device)
    st = rgg._ResolveStats()
    lib = rgg._lib()

    def call(stats):
        rgg._check("rgg_resolve_gray", lib.rgg_resolve_gray(
            r.handle, factor, out.data_ptr(), clear.data_ptr(), 1,
            ctypes.byref(st) if stats else None, int(stream.cuda_stream)))

    call(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        call(False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    res = {"factor": factor, "gray_edges": st.gray_edges, "resolved_red": st.resolved_red,
           "resolved_green": st.resolved_green, "evaluations": st.evaluations, "ms": ms,
           "gray_edges_per_s": st.gray_edges / (ms / 1e3),
           "evaluations_per_s": st.evaluations / (ms / 1e3)}
    if with_oracle and st.gray_edges:
        import oracle
        lazy = r.fetch_labels(stream=stream)
        gray = np.flatnonzero(lazy == rgg.GRAY)
        rng = np.random.default_rng(5)
        sample = rng.choice(gray, size=min(16, gray.size), replace=False)
        poses, present = r.fetch_boxes()
        t0 = time.perf_counter()
        for e in sample:
            oracle.edge_dense_clearance(sc.roadmap.robot, sc.roadmap.q_from[e],
                                        sc.roadmap.q_to[e], sc.roadmap.step, factor,
                                        poses.astype(np.float64), present=present)
        t = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": len(sample) / t, "unit": "gray edges/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"{len(sample)} gray edges, dense clearance over all "
                                         "present boxes, one thread"}
    return res


def run_geometry(args):
    """The paper's OBB / shortcut-spline geometry (Sec. 4.2, 4.3) against the
    sphere geometry on the same roadmap and update stream: classify time per
    update (the grid-filtered queries, and without the filter), the tests
    run, and the label mix each geometry reaches (gray fraction)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2603_28674_gb300 import build
    build.build()
    from paper_2603_28674_gb300 import rgg
    sc = make_scene(args.workload, n_updates=64)
    rm, robot = sc.roadmap, sc.roadmap.robot
    stream = torch.cuda.current_stream()
    dev = [torch.from_numpy(u.poses.astype(np.float32)).cuda() for u in sc.updates]
    out = {}
    with ClockSampler(0) as clocks:
        for name, geo, filt in (("spheres", rgg.GEOMETRY_SPHERES, True),
                                ("obb", rgg.GEOMETRY_OBB, True),
                                ("obb_unfiltered", rgg.GEOMETRY_OBB, False)):
            r = rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count,
                            geometry=geo)
            t0 = time.perf_counter()
            r.build_edges(robot, rm.q_from, rm.q_to, rm.step, stream)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
            if not filt:
                r.set_obb_filter(False)
            r.update_obstacles(np.arange(sc.boxes.count), sc.boxes.poses().astype(np.float32), stream)
            r.classify(stream)
            for i in range(args.warmup):
                k = i % len(sc.updates)
                r.update_obstacles(sc.updates[k].ids, dev[k], stream)
                r.classify(stream)
            torch.cuda.synchronize()
            if geo == rgg.GEOMETRY_OBB:
                r.obb_work()
            r.set_kernel_timing(True)
            r.kernel_time()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(args.steps):
                k = (args.warmup + i) % len(sc.updates)
                r.update_obstacles(sc.updates[k].ids, dev[k], stream)
                r.classify(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            k_ms, m_ms, n = r.kernel_time()
            info = r.info()
            lab = r.fetch_labels(stream=stream)
            mix = np.bincount(lab, minlength=3) / max(1, lab.size)
            res = {"ms_per_step": ms, "edges_per_s": info["num_edges"] / (ms / 1e3),
                   "classify_ms": k_ms / max(1, n), "merge_ms": m_ms / max(1, n),
                   "record_gb": info["record_bytes"] / 1e9, "build_s": build_s,
                   "labels": {"green": float(mix[0]), "gray": float(mix[1]), "red": float(mix[2])}}
            if geo == rgg.GEOMETRY_OBB:
                sat, seg = r.obb_work()
                res.update({"grid_cells": info["grid_cells"], "grid_items": info["grid_items"],
                            "spline_vertices": info["spline_vertices"],
                            "box_tests_per_step": sat / args.steps,
                            "segment_tests_per_step": seg / args.steps})
            r.check_status(stream)
            r.close()
            out[name] = res
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(2)
        idx = rng.choice(rm.num_edges, size=min(rm.num_edges, 2000), replace=False)
        t0 = time.perf_counter()
        oracle.classify_obb(robot, rm.q_from[idx], rm.q_to[idx], rm.step, sc.updates[0].poses)
        t = time.perf_counter() - t0
        cpu = {"value": len(idx) / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{len(idx)} random edges, OBB / spline labels against the "
                         f"{len(sc.updates[0].ids)} boxes one update moves (FP64, OpenMP)"}
    b = out["obb"]
    line = {
        "metric": METRIC, "value": b["edges_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload_config(args.workload, sc), geometry="obb (Sec. 4.2 boxes and "
                       "shortcut splines, grid-filtered queries)"),
        "geometries": out, "cpu_baseline": cpu,
        "gpu_launches": 5 * args.steps,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    return 0


def sjf_groups(sizes, n_groups: int):
    """Roadmap indices in shortest-job-first order (record bytes), cut into
    n_groups groups of (nearly) equal count: latency percentiles are taken
    over roadmaps, so equal counts put the median roadmap at the end of the
    middle group."""
    order = sorted(range(len(sizes)), key=lambda k: (sizes[k], k))
    n_groups = max(1, min(n_groups, len(order)))
    cuts = [round(g * len(order) / n_groups) for g in range(n_groups + 1)]
    return [order[a:b] for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def measure_batched(args, steps: int, warmup: int, n_roadmaps: int, n_groups: int = 8):
    """Workload 4: many independent roadmaps, each with its own robot, boxes
    and update per step; every roadmap's update is issued at the start of the
    step and its latency runs to its labels being ready (a CUDA event after
    its last launch).  Modes:
      plain        one launch sequence per roadmap, in arrival (index) order;
      plain_sjf    the same, smallest roadmap first;
      batched      roadmaps smallest first in n_groups persistent launches
                   (rgg_classify_many per group), an event after each group;
      one_launch   every roadmap's pass in one persistent launch;
      graph        the whole step (every update, then one persistent launch)
                   replayed as one captured CUDA graph.
    All run at the launch shape the library's autotuner picked, and all apply
    the same updates, so the final labels must agree."""
    import torch
    from paper_2603_28674_gb300 import rgg
    scenes = W.workload_batched(n_roadmaps=n_roadmaps, n_updates=8)
    stream = torch.cuda.current_stream()
    rms = []
    for sc in scenes:
        robot = sc.roadmap.robot
        r = rgg.Roadmap(robot.num_links, robot.inner_per_link, sc.boxes.count)
        r.build_edges(robot, sc.roadmap.q_from, sc.roadmap.q_to, sc.roadmap.step, stream)
        r.update_obstacles(np.arange(sc.boxes.count), sc.boxes.poses().astype(np.float32), stream)
        rms.append(r)
    rgg.classify_many(rms, stream)
    tuned = rgg.autotune(rms, reps=1, stream=stream)
    infos = [r.info() for r in rms]
    n_edges = sum(i["num_edges"] for i in infos)
    rec = sum(i["record_bytes"] for i in infos)
    dev = [[torch.from_numpy(u.poses.astype(np.float32)).cuda() for u in sc.updates]
           for sc in scenes]
    n_up = min(len(sc.updates) for sc in scenes)
    groups = sjf_groups([i["record_bytes"] for i in infos], n_groups)
    sjf = [k for g in groups for k in g]
    graphs = None

    def updates(step):
        for r, sc, d in zip(rms, scenes, dev):
            k = step % n_up
            r.update_obstacles(sc.updates[k].ids, d[k], stream)

    def event():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def run(mode, steps, warm):
        step_ms, lat = [], []
        for i in range(warm + steps):
            ends = [None] * len(rms)
            ev0 = event()
            if mode == "graph":
                graphs[i % n_up].launch(stream)
            else:
                updates(i)
                if mode == "one_launch":
                    rgg.classify_many(rms, stream)
                elif mode == "batched":
                    for g in groups:
                        rgg.classify_many([rms[k] for k in g], stream)
                        e = event()
                        for k in g:
                            ends[k] = e
                else:
                    for k in (sjf if mode == "plain_sjf" else range(len(rms))):
                        rms[k].classify(stream)
                        ends[k] = event()
            if ends[0] is None:
                # every roadmap's labels are ready when the shared launch ends
                e = event()
                ends = [e] * len(rms)
            last = event()
            torch.cuda.synchronize()
            if i >= warm:
                step_ms.append(ev0.elapsed_time(last))
                lat.extend(ev0.elapsed_time(e) for e in ends)
        return float(np.mean(step_ms)), np.array(lat), np.array(step_ms)

    out, final = {}, {}
    b_step = sum(algorithmic_bytes(i) for i in infos)
    for mode in ("plain", "plain_sjf", "batched", "one_launch", "graph"):
        if mode == "graph":
            # one graph per update index, reading the same device poses
            graphs = [rgg.StepGraph(rms, [(sc.updates[k].ids, d[k])
                                          for sc, d in zip(scenes, dev)])
                      for k in range(n_up)]
        ms, lat, st = run(mode, steps, warmup)
        final[mode] = [r.fetch_labels(stream=stream) for r in rms]
        out[mode] = {"ms_per_step": ms, "edges_per_s": n_edges / (ms / 1e3),
                     "step_ms_min_med_max": [float(np.min(st)), float(np.median(st)),
                                             float(np.max(st))],
                     "achieved_gbs": b_step / (ms / 1e3) / 1e9,
                     "latency_ms_p50": float(np.percentile(lat, 50)),
                     "latency_ms_p99": float(np.percentile(lat, 99))}
    ref = final["plain"]
    same = all(all(np.array_equal(a, b) for a, b in zip(ref, final[m])) for m in final)
    for r in rms:
        r.check_status(stream)
    nodes = graphs[0].nodes()
    for g in graphs:
        g.close()
    for r in rms:
        r.close()
    del dev
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    b, p = out["batched"], out["plain"]
    res = {"roadmaps": len(rms), "edges": n_edges, "record_gb": rec / 1e9,
           "dof": sorted({i["num_links"] for i in infos}), "moved_per_update": "1-16 per roadmap",
           "groups": len(groups), "graph_nodes": nodes,
           "autotune": {"chosen": tuned[0] if tuned else None, "shapes_timed": len(tuned)},
           "steps": steps, "warmup": warmup, "modes": out,
           "batched_vs_plain": {"throughput": b["edges_per_s"] / p["edges_per_s"],
                                "p50": p["latency_ms_p50"] / b["latency_ms_p50"],
                                "p99": p["latency_ms_p99"] / b["latency_ms_p99"]},
           "batched_vs_plain_sjf": {
               "throughput": b["edges_per_s"] / out["plain_sjf"]["edges_per_s"],
               "p50": out["plain_sjf"]["latency_ms_p50"] / b["latency_ms_p50"],
               "p99": out["plain_sjf"]["latency_ms_p99"] / b["latency_ms_p99"]},
           "labels_identical_across_modes": bool(same),
           # per step: one update kernel per roadmap; per launch group box
           # prep, classify and merge
           "gpu_launches_per_step": {"batched": len(rms) + 3 * len(groups),
                                     "plain": 4 * len(rms), "graph": len(rms) + 3}}
    return res


def run_batched(args):
    """Workload 4 on its own line (see measure_batched); the headline value is
    the CUDA-graph step's throughput."""
    import torch
    torch.cuda.set_device(0)
    from paper_2603_28674_gb300 import build
    build.build()
    peak, peak_kind = hbm_peak()
    with ClockSampler(0) as clocks:
        res = measure_batched(args, args.steps, args.warmup, args.roadmaps)
    g = res["modes"]["graph"]
    line = {
        "metric": METRIC, "value": g["edges_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batched {res['roadmaps']} roadmaps", "edges": res["edges"],
                   "record_gb": res["record_gb"], "dof": res["dof"],
                   "moved_per_update": "1-16 per roadmap", "l2": "records > L2; no flush needed"},
        "roofline": {"bound": "hbm", "achieved": g["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": g["achieved_gbs"] / peak, "traffic": None,
                     "peak_source": f"{peak_kind} HBM copy bandwidth",
                     "note": "whole step (updates + one launch per pass over all roadmaps, "
                             "replayed as one CUDA graph)"},
        "batched": res,
        "gpu_launches": args.steps * res["gpu_launches_per_step"]["graph"],
        "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    return 0 if res["labels_identical_across_modes"] else 1


def measure_serving(args, seconds: float, rate_hz: float = 2000.0):
    """Workload 5: a Poisson stream of obstacle-update requests against eight
    resident roadmaps, served with continuous batching and, for comparison,
    one request per classify launch.  Each mode starts from the same box
    state; the final labels of every roadmap must agree between the modes.
    The workload's rate is 2,000 requests/s; a higher rate shows the two
    modes once one request per launch can no longer keep up."""
    import torch
    from paper_2603_28674_gb300 import serve as SV
    scenes, reqs = W.workload_serving(rate_hz=rate_hz, duration_s=seconds)
    srv = SV.Server(device=torch.cuda.current_device())
    for sc in scenes:
        rm = sc.roadmap
        srv.add_roadmap(rm.robot, rm.q_from, rm.q_to, rm.step, np.arange(sc.boxes.count),
                        sc.boxes.poses())
    requests = [SV.ServeRequest(q.arrival_s, q.roadmap, q.update.ids.astype(np.uint32),
                                q.update.poses.astype(np.float32)) for q in reqs]
    init = [sc.boxes.poses().astype(np.float32) for sc in scenes]

    def reset():
        for r, p in zip(srv.roadmaps, init):
            r.update_obstacles(np.arange(len(p)), p, srv.stream)
            r.classify(srv.stream)
        srv.stream.synchronize()

    n_warm = min(len(requests), 300)
    warm = [SV.ServeRequest(q.arrival_s - requests[0].arrival_s, q.roadmap, q.ids, q.poses)
            for q in requests[:n_warm]]
    out, final = {}, {}
    for mode in ("one_at_a_time", "batched"):
        srv.serve(warm, mode)
        reset()
        out[mode] = srv.serve(requests, mode)
        final[mode] = [srv.labels(k) for k in range(len(srv.roadmaps))]
    same = all(np.array_equal(a, b) for a, b in zip(final["batched"], final["one_at_a_time"]))
    infos = [r.info() for r in srv.roadmaps]
    srv.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    b, p = out["batched"], out["one_at_a_time"]
    return {"roadmaps": len(scenes), "edges": [i["num_edges"] for i in infos],
            "record_gb": sum(i["record_bytes"] for i in infos) / 1e9,
            "requests": len(requests), "arrival_window_s": seconds, "rate_hz": rate_hz,
            "offered_req_s": b["offered_req_s"], "moved_per_request": "1-8",
            "batched": b, "one_at_a_time": p,
            "p50_speedup": p["latency_ms_p50"] / b["latency_ms_p50"],
            "p99_speedup": p["latency_ms_p99"] / b["latency_ms_p99"],
            "throughput_speedup": b["throughput_req_s"] / p["throughput_req_s"],
            "final_labels_identical": bool(same)}


def run_serve(args):
    """Workload 5 on its own line (see measure_serving)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2603_28674_gb300 import build
    build.build()
    with ClockSampler(0) as clocks:
        res = measure_serving(args, args.serve_seconds)
    b = res["batched"]
    line = {
        "metric": METRIC, "value": b["edges_per_s"], "unit": "request-edges/s", "n_gpus": 1,
        "steps": res["requests"], "warmup": 300,
        "ms_per_step": 1e3 / b["throughput_req_s"] if b["throughput_req_s"] else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving {res['roadmaps']} resident roadmaps",
                   "edges": res["edges"], "record_gb": res["record_gb"],
                   "offered_req_s": res["offered_req_s"], "boxes_per_roadmap": 64,
                   "moved_per_request": "1-8", "duration_s": args.serve_seconds,
                   "l2": "records > L2; no flush needed"},
        "serving": res,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    return 0 if res["final_labels_identical"] else 1


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.geometry == "obb":
        return run_geometry(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
