"""Python access to the FP64 CPU oracle (oracle/rgg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg call this; the product path never does.  The
oracle shares no code with the CUDA library.  Every function computes in
FP64 from the robot, the edge endpoints and the box poses.

Conventions (paper sections in brackets):
  robot    any object with DH arrays ``a, alpha, d, radius`` ([L] float64) and
           ``inner_per_link`` (K) [Sec. 3.2, 4.2]
  edges    ``qa, qb``: [N, L] float64 joint-space endpoints; ``step``: the
           resolution eps [Sec. 3.2]
  boxes    [M, 15] float64 poses: centre(3), R(9 row-major, columns are the box
           axes), half-extents(3); ``present``: [M] bool, absent boxes ignored
  labels   0 = GREEN, 1 = GRAY, 2 = RED [Sec. 4.1]
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build_oracle

GREEN, GRAY, RED = 0, 1, 2

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_oracle.build())
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.or_set_threads.argtypes = [i32]
    lib.or_max_threads.restype = i32
    lib.or_num_samples.argtypes = [i32, _D, _D, dbl]
    lib.or_num_samples.restype = i64
    lib.or_forward_kinematics.argtypes = [i32, _D, _D, _D, _D, _D]
    lib.or_box_distance.argtypes = [_D, _D]
    lib.or_box_distance.restype = dbl
    lib.or_edge_spheres.argtypes = [i32, _D, _D, _D, _D, i32, _D, _D, dbl, i64, _D, _D]
    lib.or_edge_spheres.restype = i64
    lib.or_classify.argtypes = [i32, _D, _D, _D, _D, i32, i64, _D, _D, dbl, i64, i32, _D,
                                _U8, _U8, _D, _D, _D, _U32, _U32]
    lib.or_classify.restype = i32
    _I64 = ctypes.POINTER(ctypes.c_int64)
    lib.or_classify_spheres.argtypes = [i64, _I64, _D, _I64, _D, i32, _D, _U8, _U8, _D,
                                        _U32, _U32]
    lib.or_classify_spheres.restype = i32
    lib.or_segment_point_distance.argtypes = [_D, _D, _D]
    lib.or_segment_point_distance.restype = dbl
    lib.or_obb_separation.argtypes = [_D, _D]
    lib.or_obb_separation.restype = dbl
    lib.or_edge_obbs.argtypes = [i32, _D, _D, _D, _D, _D, _D, dbl, _D]
    lib.or_edge_obbs.restype = i64
    lib.or_edge_splines.argtypes = [i32, _D, _D, _D, _D, i32, _D, _D, dbl, i64, _D, _I64]
    lib.or_edge_splines.restype = i64
    lib.or_classify_obb.argtypes = [i32, _D, _D, _D, _D, i32, i64, _D, _D, dbl, i64, i32, _D,
                                    _U8, _U8, _D, _U32, _U32]
    lib.or_classify_obb.restype = i32
    lib.or_segment_box_distance.argtypes = [_D, _D, _D]
    lib.or_segment_box_distance.restype = dbl
    lib.or_edge_dense_clearance.argtypes = [i32, _D, _D, _D, _D, _D, _D, dbl, i32, i32, _D,
                                            _U8, _D]
    lib.or_edge_dense_clearance.restype = dbl
    _lib = lib
    return lib


def _d(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return x, x.ctypes.data_as(_D)


def _robot(robot):
    arrs = [np.ascontiguousarray(getattr(robot, k), dtype=np.float64)
            for k in ("a", "alpha", "d", "radius")]
    return arrs, [a.ctypes.data_as(_D) for a in arrs], int(arrs[0].shape[0]), \
        int(robot.inner_per_link)


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_max_threads())


def num_samples(qa, qb, step: float) -> int:
    """Configurations of one edge, max(2, ceil(|qb - qa|_inf / step) + 1)."""
    qa, pa = _d(qa)
    qb, pb = _d(qb)
    return int(_load().or_num_samples(qa.shape[0], pa, pb, float(step)))


def forward_kinematics(robot, q) -> np.ndarray:
    """Frame origins o_0..o_L, [L+1, 3]."""
    keep, ptrs, L, _ = _robot(robot)
    q, pq = _d(q)
    out = np.zeros((L + 1, 3))
    _load().or_forward_kinematics(L, *ptrs[:3], pq, out.ctypes.data_as(_D))
    return out


def box_distance(box, x) -> float:
    box, pb = _d(box)
    x, px = _d(x)
    return float(_load().or_box_distance(pb, px))


def edge_spheres(robot, qa, qb, step: float):
    """(inner [n, L, K, 4], outer [n-1, L, 4]) for one edge, (x, y, z, r)."""
    keep, ptrs, L, K = _robot(robot)
    n = num_samples(qa, qb, step)
    qa, pa = _d(qa)
    qb, pb = _d(qb)
    inner = np.zeros((n, L, K, 4))
    outer = np.zeros((max(n - 1, 0), L, 4))
    got = _load().or_edge_spheres(L, *ptrs, K, pa, pb, float(step), n,
                                  inner.ctypes.data_as(_D), outer.ctypes.data_as(_D))
    assert got == n
    return inner, outer


def classify(robot, qa, qb, step: float, boxes, present=None, bits: bool = False):
    """Plain-definition labels of every edge against every present box.

    Returns a dict with ``labels`` [N] uint8, ``kappa``, ``h_in``, ``h_out``
    [N] float64 and, with ``bits``, ``hit`` / ``touch`` [N, ceil(M/32)] uint32.
    """
    keep, ptrs, L, K = _robot(robot)
    qa, pa = _d(np.asarray(qa).reshape(-1, L))
    qb, pb = _d(np.asarray(qb).reshape(-1, L))
    n_edges = qa.shape[0]
    boxes, pbx = _d(np.asarray(boxes, dtype=np.float64).reshape(-1, 15))
    m = boxes.shape[0]
    pres = None
    if present is not None:
        pres = np.ascontiguousarray(present, dtype=np.uint8)
    max_s = 2
    if n_edges:
        dq = np.abs(qb - qa).max(axis=1)
        max_s = int(np.ceil(dq.max() / step)) + 3
    out = {k: np.zeros(n_edges) for k in ("kappa", "h_in", "h_out")}
    out["labels"] = np.zeros(n_edges, dtype=np.uint8)
    w = (m + 31) // 32
    hit = np.zeros((n_edges, max(w, 1)), dtype=np.uint32) if bits else None
    touch = np.zeros((n_edges, max(w, 1)), dtype=np.uint32) if bits else None
    rc = _load().or_classify(
        L, *ptrs, K, n_edges, pa, pb, float(step), max_s, m, pbx,
        pres.ctypes.data_as(_U8) if pres is not None else None,
        out["labels"].ctypes.data_as(_U8),
        out["kappa"].ctypes.data_as(_D), out["h_in"].ctypes.data_as(_D),
        out["h_out"].ctypes.data_as(_D),
        hit.ctypes.data_as(_U32) if bits else None,
        touch.ctypes.data_as(_U32) if bits else None)
    if rc != 0:
        raise ValueError("oracle classify rejected its arguments")
    if bits:
        out["hit"], out["touch"] = hit[:, :w], touch[:, :w]
    return out


def classify_spheres(in_off, inner, out_off, outer, boxes, present=None, bits: bool = False):
    """Labels of edges given their sphere sets (or_classify_spheres): edge e
    owns inner[in_off[e]:in_off[e+1]] and outer[out_off[e]:out_off[e+1]],
    rows (x, y, z, r).  Returns ``labels``, ``kappa`` and, with ``bits``,
    ``hit`` / ``touch``."""
    _I64 = ctypes.POINTER(ctypes.c_int64)
    io = np.ascontiguousarray(in_off, dtype=np.int64)
    oo = np.ascontiguousarray(out_off, dtype=np.int64)
    n_edges = io.shape[0] - 1
    if oo.shape[0] != n_edges + 1:
        raise ValueError("one offset table entry per edge for both sphere sets")
    inner, pi = _d(np.asarray(inner, dtype=np.float64).reshape(-1, 4))
    outer, po = _d(np.asarray(outer, dtype=np.float64).reshape(-1, 4))
    if io[-1] > inner.shape[0] or oo[-1] > outer.shape[0]:
        raise ValueError("offsets beyond the sphere arrays")
    boxes, pbx = _d(np.asarray(boxes, dtype=np.float64).reshape(-1, 15))
    m = boxes.shape[0]
    pres = None if present is None else np.ascontiguousarray(present, dtype=np.uint8)
    w = max((m + 31) // 32, 1)
    out = {"labels": np.zeros(n_edges, dtype=np.uint8), "kappa": np.zeros(n_edges)}
    hit = np.zeros((n_edges, w), dtype=np.uint32)
    touch = np.zeros((n_edges, w), dtype=np.uint32)
    rc = _load().or_classify_spheres(
        n_edges, io.ctypes.data_as(_I64), pi, oo.ctypes.data_as(_I64), po, m, pbx,
        pres.ctypes.data_as(_U8) if pres is not None else None,
        out["labels"].ctypes.data_as(_U8), out["kappa"].ctypes.data_as(_D),
        hit.ctypes.data_as(_U32), touch.ctypes.data_as(_U32))
    if rc != 0:
        raise ValueError("oracle classify_spheres rejected its arguments")
    if bits:
        out["hit"], out["touch"] = hit, touch
    return out


def segment_point_distance(p0, p1, x) -> float:
    p0, a = _d(p0)
    p1, b = _d(p1)
    x, c = _d(x)
    return float(_load().or_segment_point_distance(a, b, c))


def obb_separation(A, B) -> float:
    """Largest separation of two boxes (15 doubles each) over the 15 SAT axes:
    > 0 disjoint, <= 0 they meet."""
    A, pa = _d(np.asarray(A, dtype=np.float64).reshape(15))
    B, pb = _d(np.asarray(B, dtype=np.float64).reshape(15))
    return float(_load().or_obb_separation(pa, pb))


def edge_obbs(robot, qa, qb, step: float):
    """[L, 15] boxes of the edge's bodies (or_edge_obbs)."""
    keep, ptrs, L, K = _robot(robot)
    qa, pa = _d(qa)
    qb, pb = _d(qb)
    out = np.zeros((L, 15))
    n = _load().or_edge_obbs(L, *ptrs, pa, pb, float(step), out.ctypes.data_as(_D))
    if n < 0:
        raise ValueError("oracle edge_obbs rejected its arguments")
    return out


def edge_splines(robot, qa, qb, step: float):
    """Kept spline vertices per (body, sphere): a list of L lists of K arrays
    [count, 3] (or_edge_splines)."""
    _I64 = ctypes.POINTER(ctypes.c_int64)
    keep, ptrs, L, K = _robot(robot)
    qa, pa = _d(qa)
    qb, pb = _d(qb)
    n = num_samples(qa, qb, step)
    verts = np.zeros((L, K, n, 3))
    counts = np.zeros((L, K), dtype=np.int64)
    got = _load().or_edge_splines(L, *ptrs, K, pa, pb, float(step), n, verts.ctypes.data_as(_D),
                                  counts.ctypes.data_as(_I64))
    if got < 0:
        raise ValueError("oracle edge_splines rejected its arguments")
    return [[verts[i, s, :counts[i, s]] for s in range(K)] for i in range(L)]


def classify_obb(robot, qa, qb, step: float, boxes, present=None, bits: bool = False):
    """Labels with the paper's OBB / spline primitives (or_classify_obb):
    ``labels``, ``kappa`` and, with ``bits``, ``hit`` / ``touch``."""
    keep, ptrs, L, K = _robot(robot)
    qa, pa = _d(np.asarray(qa).reshape(-1, L))
    qb, pb = _d(np.asarray(qb).reshape(-1, L))
    n_edges = qa.shape[0]
    boxes, pbx = _d(np.asarray(boxes, dtype=np.float64).reshape(-1, 15))
    m = boxes.shape[0]
    pres = None if present is None else np.ascontiguousarray(present, dtype=np.uint8)
    max_s = 2
    if n_edges:
        max_s = int(np.ceil(np.abs(qb - qa).max(axis=1).max() / step)) + 3
    w = max((m + 31) // 32, 1)
    out = {"labels": np.zeros(n_edges, dtype=np.uint8), "kappa": np.zeros(n_edges)}
    hit = np.zeros((n_edges, w), dtype=np.uint32)
    touch = np.zeros((n_edges, w), dtype=np.uint32)
    rc = _load().or_classify_obb(
        L, *ptrs, K, n_edges, pa, pb, float(step), max_s, m, pbx,
        pres.ctypes.data_as(_U8) if pres is not None else None,
        out["labels"].ctypes.data_as(_U8), out["kappa"].ctypes.data_as(_D),
        hit.ctypes.data_as(_U32), touch.ctypes.data_as(_U32))
    if rc != 0:
        raise ValueError("oracle classify_obb rejected its arguments")
    if bits:
        out["hit"], out["touch"] = hit[:, :(m + 31) // 32], touch[:, :(m + 31) // 32]
    return out


def segment_box_distance(p0, p1, box) -> float:
    p0, a = _d(p0)
    p1, b = _d(p1)
    box, c = _d(box)
    return float(_load().or_segment_box_distance(a, b, c))


def edge_dense_clearance(robot, qa, qb, step: float, factor: int, boxes, present=None):
    """Minimum over a `factor`-times finer resampling of the edge, links and
    present boxes of (capsule-axis-to-box distance - R); <= 0 means the robot
    collides there.  Returns (clearance, edge fraction where it occurs)."""
    keep, ptrs, L, K = _robot(robot)
    qa, pa = _d(qa)
    qb, pb = _d(qb)
    boxes, pbx = _d(np.asarray(boxes, dtype=np.float64).reshape(-1, 15))
    pres = None if present is None else np.ascontiguousarray(present, dtype=np.uint8)
    t = ctypes.c_double(-1.0)
    v = _load().or_edge_dense_clearance(
        L, ptrs[0], ptrs[1], ptrs[2], ptrs[3], pa, pb, float(step), int(factor),
        boxes.shape[0], pbx, pres.ctypes.data_as(_U8) if pres is not None else None,
        ctypes.byref(t))
    return float(v), float(t.value)
