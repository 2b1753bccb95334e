"""Serving obstacle-update requests against device-resident roadmaps.

A request moves a few boxes of one roadmap (Sec. 4.3's online update) and
asks for that roadmap's labels once the move is applied.  The server keeps
every roadmap's records, box sets and labels on the GPU and runs a loop of
continuous batching:

  * requests join a FIFO queue when they arrive;
  * at each iteration the planner admits waiting requests while resources
    last: a request handle on its roadmap (the library's snapshot memory) and
    a page-locked host result slot.  Requests of one roadmap are admitted in
    arrival order; a request blocked on its own roadmap does not hold back
    the others;
  * the admitted requests' moves are staged with rgg_update_request, every
    roadmap with new requests is classified in one persistent launch per pass
    (rgg_classify_many: the moves of several requests on one roadmap share a
    pass and each request still gets its own labels), and each request's
    snapshot is copied to its host slot asynchronously;
  * up to `max_inflight` iterations are enqueued at once, so new arrivals are
    admitted while earlier ones are on the GPU, and slots and handles are
    freed as iterations complete.

Roadmaps are admitted by device memory: a roadmap whose records, per-edge
state and snapshot memory (the library's own estimate, rgg_estimate_bytes)
would not fit in the memory budget is refused.

Requests are admitted by queue length: with `max_queue` set, a request that
arrives while that many requests already wait is refused at once.  A request
may carry a cancellation time: if it is still waiting then, it leaves the
queue without being staged (a request already on the GPU completes).

The `one_at_a_time` mode serves the same stream with one request per
classify launch (the update-then-classify loop of a plain caller), with the
same pipelining depth, for comparison.

Completion times come from CUDA events on the serving stream, on the same
clock as the arrivals (the loop's start event is synchronised before the
first arrival), so a latency is arrival -> labels in host memory.
"""
from __future__ import annotations

import collections
import heapq
import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class ServeRequest:
    arrival_s: float      # seconds after the start of serving
    roadmap: int          # index returned by Server.add_roadmap
    ids: np.ndarray       # [m] uint32 box ids
    poses: np.ndarray     # [m, 15] float32 absolute poses
    cancel_s: Optional[float] = None  # withdrawn at this time if not yet admitted


class RequestQueue:
    """Waiting requests in arrival order (host logic only).

    ``arrive`` refuses a request when ``max_len`` requests already wait;
    ``sweep`` drops the waiting requests whose cancellation time has come.
    Refused and cancelled requests are recorded.  A sweep looks up the
    cancellation time of each arrival once and keeps the due times in a
    heap, so its cost does not grow with the queue."""

    def __init__(self, max_len: Optional[int] = None):
        self.items: collections.deque = collections.deque()
        self.max_len = max_len
        self.refused: list = []
        self.cancelled: list = []
        self._new: list = []   # arrivals the next sweep has not seen
        self._due: list = []   # heap of (cancellation time, arrival number, item)
        self._seq = 0

    def __len__(self) -> int:
        return len(self.items)

    def arrive(self, item) -> bool:
        if self.max_len is not None and len(self.items) >= self.max_len:
            self.refused.append(item)
            return False
        self.items.append(item)
        self._new.append(item)
        return True

    def sweep(self, now: float, cancel_at) -> None:
        for item in self._new:
            t = cancel_at(item)
            if t is not None:
                heapq.heappush(self._due, (t, self._seq, item))
                self._seq += 1
        self._new.clear()
        while self._due and self._due[0][0] <= now:
            item = heapq.heappop(self._due)[2]
            try:
                self.items.remove(item)    # still waiting (not admitted meanwhile)?
            except ValueError:
                continue
            self.cancelled.append(item)


class Planner:
    """Admission of queued requests (host logic only).

    ``admit`` walks the queue in arrival order and takes a request when its
    roadmap has a free handle, a host slot is free, and no earlier request of
    the same roadmap is still waiting; it returns the admitted requests in
    arrival order and removes them from the queue."""

    def __init__(self, n_roadmaps: int, handles_per_roadmap: int, host_slots: int):
        self.free_handles = [handles_per_roadmap] * n_roadmaps
        self.free_slots = host_slots

    def admit(self, queue: collections.deque, roadmap_of, limit: Optional[int] = None) -> list:
        # walk the queue only while a request can still be taken: a slot is
        # free, the limit is not reached and some roadmap has a free handle
        # (a roadmap without one blocks its later requests)
        taken, keep = [], []
        n_open = sum(1 for h in self.free_handles if h > 0)
        while queue and self.free_slots > 0 and n_open > 0 and (limit is None or len(taken) < limit):
            item = queue.popleft()
            k = roadmap_of(item)
            if self.free_handles[k] > 0:
                self.free_handles[k] -= 1
                self.free_slots -= 1
                if self.free_handles[k] == 0:
                    n_open -= 1
                taken.append(item)
            else:
                keep.append(item)
        queue.extendleft(reversed(keep))
        return taken

    def release(self, roadmap: int) -> None:
        self.free_handles[roadmap] += 1
        self.free_slots += 1


def roadmap_bytes(num_links: int, inner_per_link: int, max_obstacles: int, q_from, q_to,
                  step: float, device: int = 0) -> int:
    """Device bytes a roadmap will hold once built and serving requests: the
    library's estimate of the built roadmap plus the request snapshots."""
    from . import rgg
    n = int(np.asarray(q_from).reshape(-1, num_links).shape[0])
    return rgg.estimate_bytes(num_links, inner_per_link, max_obstacles, q_from, q_to, step,
                              device=device) + rgg.MAX_REQUESTS * n


class Server:
    def __init__(self, device: int = 0, memory_budget: Optional[int] = None,
                 max_inflight: int = 2, host_slots: int = 256):
        import torch

        from . import rgg

        self.torch, self.rgg = torch, rgg
        self.device = device
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            memory_budget = int(0.9 * free)
        self.memory_budget = memory_budget
        self.memory_used = 0
        self.max_inflight = max_inflight
        self.host_slots = host_slots
        self.roadmaps: List = []
        self.num_edges: List[int] = []
        self._slots = None

    # -- resident roadmaps ---------------------------------------------------
    def add_roadmap(self, robot, q_from, q_to, step: float, box_ids, box_poses,
                    max_obstacles: Optional[int] = None) -> int:
        """Build a roadmap's records on the GPU and place its boxes; refused
        with MemoryError when it does not fit in the memory budget."""
        rgg = self.rgg
        M = int(max_obstacles if max_obstacles is not None else len(box_ids))
        need = roadmap_bytes(robot.num_links, robot.inner_per_link, M, q_from, q_to, step,
                             self.device)
        if self.memory_used + need > self.memory_budget:
            raise MemoryError(f"roadmap needs {need} B; {self.memory_budget - self.memory_used}"
                              " B of the budget left")
        r = rgg.Roadmap(robot.num_links, robot.inner_per_link, M, device=self.device)
        r.build_edges(robot, q_from, q_to, step, self.stream)
        r.update_obstacles(box_ids, np.asarray(box_poses, np.float32), self.stream)
        r.classify(self.stream)
        r.check_status(self.stream)
        info = r.info()
        self.memory_used += max(need, int(info["device_bytes"]) +
                                rgg.MAX_REQUESTS * int(info["num_edges"]))
        self.roadmaps.append(r)
        self.num_edges.append(int(info["num_edges"]))
        self._slots = None
        return len(self.roadmaps) - 1

    def close(self) -> None:
        for r in self.roadmaps:
            r.close()
        self.roadmaps = []

    def labels(self, k: int) -> np.ndarray:
        self.stream.synchronize()
        return self.roadmaps[k].fetch_labels(stream=self.stream)

    # -- the serving loop ----------------------------------------------------
    def _host_slots(self):
        if self._slots is None:
            width = max(self.num_edges) if self.num_edges else 1
            self._slots = self.torch.empty((self.host_slots, max(width, 1)),
                                           dtype=self.torch.uint8, pin_memory=True)
        return self._slots

    def serve(self, requests: Sequence[ServeRequest], mode: str = "batched",
              keep_results: bool = False, max_queue: Optional[int] = None) -> Dict:
        """Serve `requests` (arrival times relative to the start of the call)
        and return latency and throughput statistics over the requests that
        completed; with keep_results the labels of every completed request
        are returned under "results" (None for refused or cancelled ones).
        With max_queue, arrivals beyond that many waiting requests are
        refused."""
        if mode not in ("batched", "one_at_a_time"):
            raise ValueError(f"unknown mode {mode}")
        torch, rgg = self.torch, self.rgg
        rms, s = self.roadmaps, self.stream
        n = len(requests)
        order = sorted(range(n), key=lambda i: requests[i].arrival_s)
        slots = self._host_slots()
        free_slots = list(range(self.host_slots))
        planner = Planner(len(rms), rgg.MAX_REQUESTS, self.host_slots)
        limit = 1 if mode == "one_at_a_time" else None
        done_s = np.full(n, np.nan)
        results: List[Optional[np.ndarray]] = [None] * n if keep_results else []
        rq_queue = RequestQueue(max_queue)
        inflight: collections.deque = collections.deque()
        batch_sizes, passes_roadmaps = [], []
        launches = 0

        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(s)
        s.synchronize()
        t0 = time.perf_counter()
        nxt, completed = 0, 0

        def retire(ev, batch):
            nonlocal completed
            t = ev0.elapsed_time(ev) / 1e3
            for (i, k, h, slot) in batch:
                done_s[i] = t
                if keep_results:
                    results[i] = slots[slot, :self.num_edges[k]].numpy().copy()
                rms[k].release_request(h)
                free_slots.append(slot)
                planner.release(k)
                completed += 1

        def settled():
            return completed + len(rq_queue.refused) + len(rq_queue.cancelled)

        while settled() < n:
            now = time.perf_counter() - t0
            while nxt < n and requests[order[nxt]].arrival_s <= now:
                rq_queue.arrive(order[nxt])
                nxt += 1
            rq_queue.sweep(now, lambda i: requests[i].cancel_s)
            queue = rq_queue.items
            while inflight and inflight[0][0].query():
                retire(*inflight.popleft())
            if queue and len(inflight) < self.max_inflight:
                taken = planner.admit(queue, lambda i: requests[i].roadmap, limit)
                if taken:
                    batch, touched = [], []
                    for i in taken:
                        rq = requests[i]
                        k = rq.roadmap
                        h = rms[k].update_request(rq.ids, rq.poses, s)
                        batch.append((i, k, h, free_slots.pop()))
                        if k not in touched:
                            touched.append(k)
                    if mode == "batched":
                        rgg.classify_many([rms[k] for k in touched], s)
                    else:
                        rms[touched[0]].classify(s)
                    launches += 1
                    for (i, k, h, slot) in batch:
                        rms[k].fetch_request_labels(h, out=slots[slot, :self.num_edges[k]],
                                                    stream=s)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(s)
                    inflight.append((ev, batch))
                    batch_sizes.append(len(batch))
                    passes_roadmaps.append(len(touched))
                    continue
            # nothing admitted: a full pipeline, or requests blocked on handles
            # or slots, or no arrival left, wait for the oldest batch; else
            # poll for the next arrival (sleeping when the GPU is idle)
            if inflight and (len(inflight) >= self.max_inflight or queue or nxt >= n):
                inflight[0][0].synchronize()
                continue
            if not inflight and nxt < n and not queue:
                wait = requests[order[nxt]].arrival_s - (time.perf_counter() - t0)
                if wait > 3e-4:
                    time.sleep(wait - 2e-4)
        for r in rms:
            r.check_status(s)
        arrivals = np.array([rq.arrival_s for rq in requests])
        ok = ~np.isnan(done_s)
        n_ok = int(ok.sum())
        lat = (done_s[ok] - arrivals[ok]) * 1e3
        span = float(np.nanmax(done_s) - arrivals.min()) if n_ok else 0.0
        edges = sum(self.num_edges[requests[i].roadmap] for i in np.flatnonzero(ok))
        out = {
            "mode": mode, "requests": n, "completed": n_ok,
            "refused": len(rq_queue.refused), "cancelled": len(rq_queue.cancelled),
            "latency_ms_p50": float(np.percentile(lat, 50)) if n_ok else 0.0,
            "latency_ms_p99": float(np.percentile(lat, 99)) if n_ok else 0.0,
            "latency_ms_max": float(lat.max()) if n_ok else 0.0,
            "latency_ms_mean": float(lat.mean()) if n_ok else 0.0,
            "throughput_req_s": n_ok / span if span > 0 else 0.0,
            "offered_req_s": (n / float(arrivals.max() - arrivals.min())
                              if n > 1 and arrivals.max() > arrivals.min() else 0.0),
            "edges_per_s": edges / span if span > 0 else 0.0,
            "span_s": span,
            "batches": len(batch_sizes),
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            "mean_roadmaps_per_launch": float(np.mean(passes_roadmaps)) if passes_roadmaps else 0.0,
            "classify_calls": launches,
        }
        if keep_results:
            out["results"] = results
        return out
