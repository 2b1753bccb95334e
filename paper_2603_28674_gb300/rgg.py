"""Python binding of librgg.so (include/rgg.h): argument marshalling only.

Every step of the classification runs in the library's CUDA kernels.  There
is no CPU fallback: if librgg.so has not been built, or no GPU is present,
the calls raise.

Streams: every call takes ``stream`` as a CUDA stream handle (int), a
``torch.cuda.Stream``, or None for torch's current stream on the roadmap's
device.  Device buffers are torch CUDA tensors; host buffers numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

GREEN, GRAY, RED = 0, 1, 2
GEOMETRY_SPHERES, GEOMETRY_OBB = 0, 1
RECORDS_LINK_ENDS, RECORDS_SPHERES = 0, 1
RGG_OK, RGG_ERR_INVALID, RGG_ERR_OOM, RGG_ERR_CUDA, RGG_ERR_TIMEOUT, RGG_ERR_STATE = \
    0, -1, -2, -3, -4, -5
RGG_ERR_CAPACITY = -6
RGG_ERR_IO = -7
NOALLOC_MAX_EDGES = 131072
NOALLOC_MAX_TILES = 16384
BOXES_PER_PASS = 32
NUM_VARIANTS = 13
MAX_REQUESTS = 64
PENDING_EXTRA = 4096

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librgg.so")

# Entry points declared in include/rgg.h (checked by the test suite).
EXPORTS = (
    "rgg_roadmap_create", "rgg_roadmap_destroy", "rgg_upload_edges", "rgg_build_edges",
    "rgg_update_obstacles", "rgg_classify", "rgg_classify_many", "rgg_fetch_labels",
    "rgg_fetch_box_sets", "rgg_fetch_records", "rgg_labels_device_ptr", "rgg_roadmap_info",
    "rgg_check_status", "rgg_set_kernel_timing", "rgg_kernel_time", "rgg_set_launch_shape",
    "rgg_status_string", "rgg_classify_noalloc", "rgg_update_request",
    "rgg_fetch_request_labels", "rgg_release_request", "rgg_autotune",
    "rgg_step_graph_create", "rgg_step_graph_launch", "rgg_step_graph_nodes",
    "rgg_step_graph_destroy", "rgg_save", "rgg_load", "rgg_resolve_gray", "rgg_fetch_boxes",
    "rgg_set_obb_filter", "rgg_obb_work", "rgg_fetch_obb_records", "rgg_set_round_filter",
    "rgg_streamed_bytes", "rgg_set_wait_limit", "rgg_inject_alloc_failure", "rgg_estimate_bytes",
    "rgg_set_work_counting", "rgg_work_counts", "rgg_check_guards",
)


class RGGError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = _lib().rgg_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{fn} failed: {msg} ({status})")


class _Desc(ctypes.Structure):
    _fields_ = [("num_links", ctypes.c_uint32), ("inner_per_link", ctypes.c_uint32),
                ("max_obstacles", ctypes.c_uint32), ("margin_m", ctypes.c_float),
                ("device", ctypes.c_int), ("geometry", ctypes.c_uint32),
                ("record_format", ctypes.c_uint32)]


class _Robot(ctypes.Structure):
    _fields_ = [("num_links", ctypes.c_uint32), ("a", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("d", ctypes.POINTER(ctypes.c_double)),
                ("radius", ctypes.POINTER(ctypes.c_double))]


class _NoallocArgs(ctypes.Structure):
    _fields_ = [("num_links", ctypes.c_uint32), ("inner_per_link", ctypes.c_uint32),
                ("num_edges", ctypes.c_uint64), ("num_samples", ctypes.c_uint64),
                ("sample_off", ctypes.c_void_p), ("inner_xyzr", ctypes.c_void_p),
                ("inner_stride", ctypes.c_uint64), ("outer_xyzr", ctypes.c_void_p),
                ("outer_stride", ctypes.c_uint64), ("num_boxes", ctypes.c_uint32),
                ("box_ids", ctypes.c_void_p), ("box_poses", ctypes.c_void_p),
                ("mask_words", ctypes.c_uint32), ("hit", ctypes.c_void_p),
                ("touch", ctypes.c_void_p), ("counts", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("margin_m", ctypes.c_float),
                ("regular_records", ctypes.c_uint32), ("status", ctypes.c_void_p),
                ("wait_limit_ns", ctypes.c_uint64)]


class _TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("consumer_warps", ctypes.c_uint32),
                ("classify_ms", ctypes.c_float), ("reserved", ctypes.c_float)]


class _ResolveStats(ctypes.Structure):
    _fields_ = [("gray_edges", ctypes.c_uint64), ("resolved_red", ctypes.c_uint64),
                ("resolved_green", ctypes.c_uint64), ("evaluations", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [("num_edges", ctypes.c_uint64), ("num_samples", ctypes.c_uint64),
                ("num_inner", ctypes.c_uint64), ("num_outer", ctypes.c_uint64),
                ("record_bytes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("num_links", ctypes.c_uint32), ("inner_per_link", ctypes.c_uint32),
                ("max_obstacles", ctypes.c_uint32), ("mask_words", ctypes.c_uint32),
                ("tile_samples", ctypes.c_uint32), ("num_tiles", ctypes.c_uint64),
                ("pending_boxes", ctypes.c_uint32), ("grid_ctas", ctypes.c_uint32),
                ("open_requests", ctypes.c_uint32), ("pending_capacity", ctypes.c_uint32),
                ("geometry", ctypes.c_uint32), ("grid_cells", ctypes.c_uint32),
                ("grid_items", ctypes.c_uint64), ("spline_vertices", ctypes.c_uint64),
                ("round_filter", ctypes.c_uint32), ("record_format", ctypes.c_uint32),
                ("variant", ctypes.c_uint32), ("last_variant", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    dbl = ctypes.c_double
    sig = {
        "rgg_roadmap_create": [ctypes.POINTER(_Desc), ctypes.POINTER(vp)],
        "rgg_roadmap_destroy": [vp],
        "rgg_upload_edges": [vp, u64, vp, vp, vp, i32, vp],
        "rgg_build_edges": [vp, ctypes.POINTER(_Robot), u64, vp, vp, dbl, vp],
        "rgg_update_obstacles": [vp, u32, vp, vp, i32, vp],
        "rgg_classify": [vp, vp],
        "rgg_classify_many": [ctypes.POINTER(vp), u32, vp],
        "rgg_fetch_labels": [vp, vp, u64, u64, i32, vp],
        "rgg_fetch_box_sets": [vp, vp, vp, u64, u64, i32, vp],
        "rgg_fetch_records": [vp, u64, u64, vp, vp, vp],
        "rgg_labels_device_ptr": [vp, ctypes.POINTER(vp)],
        "rgg_roadmap_info": [vp, ctypes.POINTER(Info)],
        "rgg_check_status": [vp, vp],
        "rgg_set_kernel_timing": [vp, i32],
        "rgg_kernel_time": [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(u64)],
        "rgg_set_launch_shape": [vp, u32, u32],
        "rgg_classify_noalloc": [ctypes.POINTER(_NoallocArgs), vp],
        "rgg_update_request": [vp, u32, vp, vp, i32, ctypes.POINTER(u32), vp],
        "rgg_fetch_request_labels": [vp, u32, vp, u64, u64, i32, vp],
        "rgg_release_request": [vp, u32],
        "rgg_autotune": [ctypes.POINTER(vp), u32, u32, ctypes.POINTER(_TuneResult), u32,
                         ctypes.POINTER(u32), vp],
        "rgg_step_graph_create": [ctypes.POINTER(vp), u32, ctypes.POINTER(u32),
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                  ctypes.POINTER(vp)],
        "rgg_step_graph_launch": [vp, vp],
        "rgg_step_graph_nodes": [vp, ctypes.POINTER(u64)],
        "rgg_step_graph_destroy": [vp],
        "rgg_save": [vp, ctypes.c_char_p, vp],
        "rgg_resolve_gray": [vp, u32, vp, vp, i32, ctypes.POINTER(_ResolveStats), vp],
        "rgg_fetch_boxes": [vp, vp, vp, vp],
        "rgg_set_obb_filter": [vp, i32],
        "rgg_set_round_filter": [vp, i32],
        "rgg_streamed_bytes": [vp, ctypes.POINTER(u64)],
        "rgg_obb_work": [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "rgg_fetch_obb_records": [vp, vp, vp, vp],
        "rgg_load": [vp, ctypes.c_char_p, vp],
        "rgg_set_wait_limit": [vp, u64],
        "rgg_set_work_counting": [vp, i32],
        "rgg_work_counts": [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "rgg_inject_alloc_failure": [u64],
        "rgg_check_guards": [ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "rgg_estimate_bytes": [ctypes.POINTER(_Desc), u64, vp, vp, dbl, ctypes.POINTER(u64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = i32
    lib.rgg_status_string.argtypes = [i32]
    lib.rgg_status_string.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def library_path() -> str:
    _lib()
    return LIB_PATH


def _check(fn: str, status: int) -> None:
    if status != RGG_OK:
        raise RGGError(fn, status)


def _stream(stream, device: int) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream(device).cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _host(arr, dtype) -> np.ndarray:
    return np.ascontiguousarray(arr, dtype=dtype)


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x) -> int:
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("torch buffers must be contiguous")
        return int(x.data_ptr())
    return int(x.ctypes.data)


def _dst_kind(out) -> int:
    """0 host (synchronous), 1 device, 2 page-locked torch CPU tensor (async)."""
    if _is_device(out):
        return 1
    if hasattr(out, "is_pinned") and out.is_pinned():
        return 2
    return 0


class Roadmap:
    """One resident roadmap (wraps an rgg_roadmap_t)."""

    def __init__(self, num_links: int, inner_per_link: int, max_obstacles: int,
                 margin: float = 2e-5, device: int = 0, geometry: int = GEOMETRY_SPHERES,
                 record_format: int = RECORDS_LINK_ENDS):
        lib = _lib()
        desc = _Desc(num_links, inner_per_link, max_obstacles, margin, device, geometry,
                     record_format)
        h = ctypes.c_void_p()
        _check("rgg_roadmap_create", lib.rgg_roadmap_create(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.device = device
        self.num_links = num_links
        self.inner_per_link = inner_per_link
        self.max_obstacles = max_obstacles
        self.margin = margin
        self.geometry = geometry

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib().rgg_roadmap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- offline records ----------------------------------------------------
    def build_edges(self, robot, q_from, q_to, step: float, stream=None) -> None:
        """Build the sphere records on the GPU from edge endpoints (rgg_build_edges)."""
        arrs = [_host(getattr(robot, k), np.float64) for k in ("a", "alpha", "d", "radius")]
        p = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs]
        rb = _Robot(len(arrs[0]), *p)
        qa = _host(q_from, np.float64).reshape(-1, self.num_links)
        qb = _host(q_to, np.float64).reshape(-1, self.num_links)
        if qa.shape != qb.shape:
            raise ValueError("q_from and q_to differ in shape")
        _check("rgg_build_edges", _lib().rgg_build_edges(
            self._h, ctypes.byref(rb), qa.shape[0], qa.ctypes.data, qb.ctypes.data, float(step),
            _stream(stream, self.device)))

    def upload_edges(self, sample_off, inner_xyzr, outer_xyzr, stream=None) -> None:
        """Upload caller-built records (rgg_upload_edges); inner/outer are [4, n]
        plane arrays, host numpy or device torch tensors."""
        soff = _host(sample_off, np.uint64)
        dev = _is_device(inner_xyzr)
        if dev != _is_device(outer_xyzr):
            raise ValueError("inner and outer records must both be host or both device")
        if not dev:
            inner_xyzr = _host(inner_xyzr, np.float32)
            outer_xyzr = _host(outer_xyzr, np.float32)
        _check("rgg_upload_edges", _lib().rgg_upload_edges(
            self._h, soff.shape[0] - 1, soff.ctypes.data, _ptr(inner_xyzr), _ptr(outer_xyzr),
            int(dev), _stream(stream, self.device)))

    # -- online update and classification -------------------------------------
    def update_obstacles(self, ids, poses, stream=None) -> None:
        """Move boxes ``ids`` to absolute ``poses`` [m, 15] (float32; host numpy
        or device tensor)."""
        ids = _host(ids, np.uint32).reshape(-1)
        dev = _is_device(poses)
        if not dev:
            poses = _host(poses, np.float32).reshape(-1, 15)
            if poses.shape[0] != ids.shape[0]:
                raise ValueError("one pose per id")
        _check("rgg_update_obstacles", _lib().rgg_update_obstacles(
            self._h, ids.shape[0], ids.ctypes.data, _ptr(poses), int(dev),
            _stream(stream, self.device)))

    def update_request(self, ids, poses, stream=None) -> int:
        """Versioned move (rgg_update_request): like update_obstacles, and the
        labels once this move is applied are kept under the returned handle."""
        ids = _host(ids, np.uint32).reshape(-1)
        dev = _is_device(poses)
        if not dev:
            poses = _host(poses, np.float32).reshape(-1, 15)
            if poses.shape[0] != ids.shape[0]:
                raise ValueError("one pose per id")
        h = ctypes.c_uint32()
        _check("rgg_update_request", _lib().rgg_update_request(
            self._h, ids.shape[0], ids.ctypes.data, _ptr(poses), int(dev), ctypes.byref(h),
            _stream(stream, self.device)))
        return int(h.value)

    def fetch_request_labels(self, handle: int, first: int = 0, count: Optional[int] = None,
                             out=None, stream=None):
        """Snapshot labels of request ``handle`` (numpy uint8, a device tensor,
        or a pinned CPU tensor filled asynchronously)."""
        if count is None:
            count = self.info()["num_edges"] - first
        if out is None:
            out = np.empty(count, dtype=np.uint8)
        _check("rgg_fetch_request_labels", _lib().rgg_fetch_request_labels(
            self._h, handle, _ptr(out), first, count, _dst_kind(out),
            _stream(stream, self.device)))
        return out

    def release_request(self, handle: int) -> None:
        _check("rgg_release_request", _lib().rgg_release_request(self._h, handle))

    def classify(self, stream=None) -> None:
        _check("rgg_classify", _lib().rgg_classify(self._h, _stream(stream, self.device)))

    # -- results --------------------------------------------------------------
    def fetch_labels(self, first: int = 0, count: Optional[int] = None, out=None,
                     stream=None):
        """Labels [first, first+count) into ``out`` (numpy uint8, a device
        tensor, or a pinned CPU tensor filled asynchronously), allocated as
        numpy when None."""
        if count is None:
            count = self.info()["num_edges"] - first
        if out is None:
            out = np.empty(count, dtype=np.uint8)
        _check("rgg_fetch_labels", _lib().rgg_fetch_labels(
            self._h, _ptr(out), first, count, _dst_kind(out), _stream(stream, self.device)))
        return out

    def fetch_box_sets(self, first: int = 0, count: Optional[int] = None, stream=None):
        """(hit, touch) box-id bitsets [count, mask_words] uint32, host."""
        info = self.info()
        if count is None:
            count = info["num_edges"] - first
        hit = np.empty((count, info["mask_words"]), dtype=np.uint32)
        touch = np.empty_like(hit)
        _check("rgg_fetch_box_sets", _lib().rgg_fetch_box_sets(
            self._h, hit.ctypes.data, touch.ctypes.data, first, count, 0,
            _stream(stream, self.device)))
        return hit, touch

    def fetch_records(self, first: int = 0, count: Optional[int] = None):
        """(inner [4, n_in], outer [4, n_out], sample_off [N+1]) of edges
        [first, first+count), host, in the rgg_upload_edges layout."""
        info = self.info()
        n = info["num_edges"]
        soff = np.empty(n + 1, dtype=np.uint64)
        _check("rgg_fetch_records", _lib().rgg_fetch_records(self._h, 0, 0, None, None,
                                                             soff.ctypes.data))
        if count is None:
            count = n - first
        s0, s1 = int(soff[first]), int(soff[first + count])
        L, K = self.num_links, self.inner_per_link
        inner = np.empty((4, K * L * (s1 - s0)), dtype=np.float32)
        outer = np.empty((4, L * (s1 - s0 - count)), dtype=np.float32)
        _check("rgg_fetch_records", _lib().rgg_fetch_records(
            self._h, first, count, inner.ctypes.data, outer.ctypes.data, None))
        return inner, outer, soff

    def fetch_boxes(self, stream=None):
        """(poses [M, 15] float32, present [M] uint8) of the box table."""
        poses = np.empty((self.max_obstacles, 15), dtype=np.float32)
        present = np.empty(self.max_obstacles, dtype=np.uint8)
        _check("rgg_fetch_boxes", _lib().rgg_fetch_boxes(self._h, poses.ctypes.data,
                                                         present.ctypes.data,
                                                         _stream(stream, self.device)))
        return poses, present

    def labels_device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check("rgg_labels_device_ptr", _lib().rgg_labels_device_ptr(self._h, ctypes.byref(p)))
        return int(p.value or 0)

    def info(self) -> dict:
        inf = Info()
        _check("rgg_roadmap_info", _lib().rgg_roadmap_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def check_status(self, stream=None) -> None:
        _check("rgg_check_status", _lib().rgg_check_status(self._h, _stream(stream, self.device)))

    def set_work_counting(self, enable: bool) -> None:
        """Count the classify kernel's executed work (rgg_set_work_counting)."""
        _check("rgg_set_work_counting", _lib().rgg_set_work_counting(self._h, int(enable)))

    def work_counts(self) -> dict:
        """Rounds examined, outer sphere-box tests and inner (configuration,
        box) pairs executed since the last call (rgg_work_counts)."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check("rgg_work_counts", _lib().rgg_work_counts(self._h, ctypes.byref(a), ctypes.byref(b),
                                                         ctypes.byref(c)))
        return {"rounds": int(a.value), "outer_tests": int(b.value), "inner_pairs": int(c.value)}

    def set_wait_limit(self, limit_ns: int) -> None:
        """Limit of the classify kernel's bounded waits, ns (rgg_set_wait_limit)."""
        _check("rgg_set_wait_limit", _lib().rgg_set_wait_limit(self._h, int(limit_ns)))

    def set_round_filter(self, enable: bool) -> None:
        """Sphere geometry: copy only the rounds of records the moved boxes may
        reach (default); off streams every record."""
        _check("rgg_set_round_filter", _lib().rgg_set_round_filter(self._h, int(enable)))

    def streamed_bytes(self) -> int:
        """Record bytes the classify launches copied since the last call."""
        v = ctypes.c_uint64()
        _check("rgg_streamed_bytes", _lib().rgg_streamed_bytes(self._h, ctypes.byref(v)))
        return int(v.value)

    def set_obb_filter(self, enable: bool) -> None:
        """OBB geometry: test only the grid cells the moved boxes meet (default)."""
        _check("rgg_set_obb_filter", _lib().rgg_set_obb_filter(self._h, int(enable)))

    def fetch_obb_records(self):
        """OBB geometry: (boxes [N, L, 16], spline offsets [N*L*K + 1],
        spline vertices [V, 4]) host copies (rgg_fetch_obb_records)."""
        info = self.info()
        n, L, K = info["num_edges"], self.num_links, self.inner_per_link
        obb = np.empty((n, L, 16), dtype=np.float32)
        off = np.empty(n * L * K + 1, dtype=np.uint64)
        v = np.empty((max(info["spline_vertices"], 1), 4), dtype=np.float32)
        _check("rgg_fetch_obb_records", _lib().rgg_fetch_obb_records(
            self._h, obb.ctypes.data, off.ctypes.data, v.ctypes.data))
        return obb, off, v[:info["spline_vertices"]]

    def obb_work(self):
        """OBB geometry: (box tests, spline-segment tests) since the last call."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check("rgg_obb_work", _lib().rgg_obb_work(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def resolve_gray(self, factor: int = 10, stream=None):
        """Non-lazy resolution of the gray edges (rgg_resolve_gray): returns
        (labels [N] uint8, clearance [N] float32, stats dict), host arrays."""
        n = self.info()["num_edges"]
        labels = np.empty(n, dtype=np.uint8)
        clear = np.empty(n, dtype=np.float32)
        st = _ResolveStats()
        _check("rgg_resolve_gray", _lib().rgg_resolve_gray(
            self._h, int(factor), labels.ctypes.data, clear.ctypes.data, 0, ctypes.byref(st),
            _stream(stream, self.device)))
        return labels, clear, {k: getattr(st, k) for k, _ in st._fields_}

    # -- persistence ----------------------------------------------------------
    def save(self, path, stream=None) -> None:
        """Write the records, per-edge state and boxes to `path` (rgg_save)."""
        _check("rgg_save", _lib().rgg_save(self._h, os.fsencode(path),
                                           _stream(stream, self.device)))

    def load(self, path, stream=None) -> None:
        """Replace edges and state with a file rgg_save wrote (rgg_load)."""
        _check("rgg_load", _lib().rgg_load(self._h, os.fsencode(path),
                                           _stream(stream, self.device)))

    # -- timing and launch shape ----------------------------------------------
    def set_kernel_timing(self, enable: bool) -> None:
        _check("rgg_set_kernel_timing", _lib().rgg_set_kernel_timing(self._h, int(enable)))

    def kernel_time(self):
        """(classify ms, merge ms, passes) of the timed passes since the last call."""
        cm, mm, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        _check("rgg_kernel_time", _lib().rgg_kernel_time(self._h, ctypes.byref(cm),
                                                         ctypes.byref(mm), ctypes.byref(n)))
        return cm.value, mm.value, n.value

    def set_launch_shape(self, variant: int = 0, consumer_warps: int = 0) -> None:
        """Pipeline shape of the classify kernel (see rgg_set_launch_shape)."""
        _check("rgg_set_launch_shape", _lib().rgg_set_launch_shape(self._h, variant,
                                                                   consumer_warps))


def classify_many(roadmaps: Sequence[Roadmap], stream=None) -> None:
    """One persistent launch per pass over all roadmaps (rgg_classify_many)."""
    if not roadmaps:
        return
    arr = (ctypes.c_void_p * len(roadmaps))(*[r.handle for r in roadmaps])
    _check("rgg_classify_many", _lib().rgg_classify_many(arr, len(roadmaps),
                                                         _stream(stream, roadmaps[0].device)))


def inject_alloc_failure(nth: int) -> None:
    """Make the nth device allocation of the library from now fail (0: off);
    a test hook (rgg_inject_alloc_failure)."""
    _check("rgg_inject_alloc_failure", _lib().rgg_inject_alloc_failure(int(nth)))


def check_guards() -> tuple:
    """(buffers checked, buffers whose guard bytes changed) over every live
    device buffer of the library (rgg_check_guards; synchronises the devices
    that hold them).  A changed guard means something wrote past the end of
    a buffer; it is reported in the count, not raised."""
    checked, bad = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = _lib().rgg_check_guards(ctypes.byref(checked), ctypes.byref(bad))
    if st not in (RGG_OK, RGG_ERR_STATE):
        _check("rgg_check_guards", st)
    return int(checked.value), int(bad.value)


def estimate_bytes(num_links: int, inner_per_link: int, max_obstacles: int, q_from, q_to,
                   step: float, margin: float = 2e-5, device: int = 0,
                   record_format: int = RECORDS_LINK_ENDS) -> int:
    """Device bytes a sphere-geometry roadmap holds after build_edges with
    these edges (rgg_estimate_bytes; host arithmetic, no GPU needed)."""
    desc = _Desc(num_links, inner_per_link, max_obstacles, margin, device, GEOMETRY_SPHERES,
                 record_format)
    qa = _host(q_from, np.float64).reshape(-1, num_links)
    qb = _host(q_to, np.float64).reshape(-1, num_links)
    if qa.shape != qb.shape:
        raise ValueError("q_from and q_to differ in shape")
    out = ctypes.c_uint64()
    _check("rgg_estimate_bytes", _lib().rgg_estimate_bytes(
        ctypes.byref(desc), qa.shape[0], qa.ctypes.data, qb.ctypes.data, float(step),
        ctypes.byref(out)))
    return int(out.value)


def classify_noalloc(*, num_links: int, inner_per_link: int, sample_off, num_samples: int,
                     inner, outer, box_ids, box_poses, mask_words: int, hit, touch, counts,
                     labels, margin: float = 2e-5, regular_records: bool = False, status=None,
                     wait_limit_ns: int = 0, stream=None) -> None:
    """One pass of rgg_classify_noalloc on caller-owned device buffers.

    ``sample_off`` (int64/uint64), ``inner`` / ``outer`` ([4, stride] float32
    planes), ``hit`` / ``touch`` ([N, mask_words] int32/uint32), ``counts``
    ([N] int32/uint32), ``labels`` ([N] uint8) and the optional ``status``
    ([1] int32) are CUDA tensors on the current device; ``box_ids`` /
    ``box_poses`` are host arrays.  ``regular_records``: the records are
    rgg_build_edges' (see include/rgg.h).  The call itself allocates nothing
    on the device."""
    ids = _host(box_ids, np.uint32).reshape(-1)
    poses = _host(box_poses, np.float32).reshape(-1, 15)
    if poses.shape[0] != ids.shape[0]:
        raise ValueError("one pose per id")
    args = _NoallocArgs(
        num_links, inner_per_link, int(labels.shape[0]), int(num_samples), _ptr(sample_off),
        _ptr(inner), int(inner.stride(0)), _ptr(outer), int(outer.stride(0)), ids.shape[0],
        ids.ctypes.data, poses.ctypes.data, mask_words, _ptr(hit), _ptr(touch), _ptr(counts),
        _ptr(labels), margin, int(bool(regular_records)),
        _ptr(status) if status is not None else None, int(wait_limit_ns))
    dev = inner.device.index if hasattr(inner, "device") else 0
    _check("rgg_classify_noalloc", _lib().rgg_classify_noalloc(ctypes.byref(args),
                                                               _stream(stream, dev)))


def autotune(roadmaps: Sequence[Roadmap], reps: int = 2, stream=None) -> list:
    """Time every supported launch shape on these roadmaps' own records and
    keep the fastest on all of them (rgg_autotune).  Returns the timed shapes,
    fastest first, as dicts."""
    if not roadmaps:
        return []
    arr = (ctypes.c_void_p * len(roadmaps))(*[r.handle for r in roadmaps])
    cap = 64
    res = (_TuneResult * cap)()
    cnt = ctypes.c_uint32()
    _check("rgg_autotune", _lib().rgg_autotune(arr, len(roadmaps), reps, res, cap,
                                               ctypes.byref(cnt),
                                               _stream(stream, roadmaps[0].device)))
    return [{"variant": res[i].variant, "consumer_warps": res[i].consumer_warps,
             "classify_ms": res[i].classify_ms} for i in range(min(cnt.value, cap))]


class StepGraph:
    """One captured update + classify step of several roadmaps (rgg_step_graph_*).

    ``moves`` is a list with one (ids, poses) pair per roadmap: ids a host
    array, poses a contiguous [m, 15] float32 CUDA tensor that every launch
    reads (write the next poses into it between launches).  Keep the tensors
    and the roadmaps alive while the graph exists."""

    def __init__(self, roadmaps: Sequence[Roadmap], moves):
        if len(moves) != len(roadmaps):
            raise ValueError("one (ids, poses) pair per roadmap")
        n = len(roadmaps)
        self._ids = [_host(ids, np.uint32).reshape(-1) for ids, _ in moves]
        self._poses = [p for _, p in moves]
        for ids, p in zip(self._ids, self._poses):
            if not _is_device(p) or tuple(p.shape) != (ids.shape[0], 15):
                raise ValueError("poses must be [m, 15] CUDA tensors, one row per id")
        self.roadmaps = list(roadmaps)
        arr = (ctypes.c_void_p * n)(*[r.handle for r in roadmaps])
        nid = (ctypes.c_uint32 * n)(*[ids.shape[0] for ids in self._ids])
        idp = (ctypes.c_void_p * n)(*[ids.ctypes.data for ids in self._ids])
        pp = (ctypes.c_void_p * n)(*[_ptr(p) for p in self._poses])
        h = ctypes.c_void_p()
        _check("rgg_step_graph_create", _lib().rgg_step_graph_create(arr, n, nid, idp, pp,
                                                                     ctypes.byref(h)))
        self._h = h
        self.device = roadmaps[0].device

    def launch(self, stream=None) -> None:
        _check("rgg_step_graph_launch", _lib().rgg_step_graph_launch(
            self._h, _stream(stream, self.device)))

    def nodes(self) -> int:
        n = ctypes.c_uint64()
        _check("rgg_step_graph_nodes", _lib().rgg_step_graph_nodes(self._h, ctypes.byref(n)))
        return int(n.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib().rgg_step_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

