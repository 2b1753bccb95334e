/*
 * rgg.h -- C ABI of the GB300 Red-Green-Gray edge-classification library
 * (librgg.so).
 *
 * The library keeps a roadmap's serialized edge approximations resident in
 * GPU memory and, after obstacles move, labels every edge RED (an inner
 * sphere certainly hits a box), GREEN (no outer sphere touches any box) or
 * GRAY (needs a full check).  The calls follow the paper's statement of the
 * problem:
 *   - the approximations are built once, offline, and stored persistently on
 *     the GPU (Sec. 4.3, "Offline storage")          -> rgg_upload_edges,
 *                                                       rgg_build_edges
 *   - after an obstacle moves only its new transform is uploaded and its
 *     rows are updated in place (Sec. 4.3, "Online updates"; Algorithm 1's
 *     input is an obstacle and its transformation)   -> rgg_update_obstacles
 *   - intersection tests over the serialized data certify red and green and
 *     leave the rest gray (Sec. 4.1; Sec. 4.3, "Intersection queries";
 *     Algorithm 1, lazy mode)                        -> rgg_classify
 *   - labels stay on the device until asked for      -> rgg_fetch_labels
 *
 * Geometry (the approximations this library classifies with):
 *   inner  K spheres per link inscribed in the link's capsule at every
 *          configuration of the edge (the vertices of the paper's splines
 *          L_{e,i}, Sec. 4.2);
 *   outer  one sphere per link per sample interval enclosing the link's sweep
 *          over that interval (stands in for the paper's per-edge OBB);
 *   boxes  each obstacle is an exact oriented box, used as both its inner
 *          and its outer approximation.
 * With margin delta, a box b is HIT by an edge if some inner sphere (c, r)
 * has dist(c, b) <= r - delta and TOUCHED if some outer sphere has
 * dist(c, b) <= r + delta.  An edge is RED if any present box hits it,
 * GREEN if no present box touches it, GRAY otherwise.  The library keeps,
 * per edge, the set of boxes that hit it and the set that touch it (the
 * per-component intersection lists of Algorithm 1), so an update only
 * re-tests the moved boxes and the label always equals the label against
 * the current pose of every box.
 *
 * Conventions
 *   - Every call returns an rgg_status (0 = RGG_OK, negative = error) unless
 *     stated otherwise.  A failed call leaves the roadmap unchanged unless
 *     stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is stream-ordered; calls on one roadmap must
 *     be issued on one stream or ordered by the caller.
 *   - The caller owns every buffer it passes; the library copies what it
 *     needs and never keeps a caller pointer after the call returns (for
 *     pinned host or device sources the copy is stream-ordered: keep the
 *     source alive and unchanged until the stream reaches it).
 *   - Each roadmap lives on one CUDA device (rgg_roadmap_desc.device); calls
 *     switch to that device and restore the caller's current device.
 *   - Errors that only the device can see (a bounded wait that ran out,
 *     see rgg_set_wait_limit) are latched in the roadmap's device status
 *     word and returned by the next rgg_fetch_labels / rgg_fetch_box_sets
 *     with a host destination or rgg_check_status as RGG_ERR_TIMEOUT.  While
 *     an error is latched every classify pass of the roadmap is skipped on
 *     the device (its kernels return at once and leave the box sets and
 *     labels as they were), so a stream of enqueued passes cannot pile up
 *     one time-out after another.  Reporting the error recovers: the word is
 *     cleared, every present box is queued again (the next rgg_classify
 *     re-tests all of them, so the labels become those of the current poses)
 *     and every open request handle is marked lost (rgg_fetch_request_labels
 *     returns RGG_ERR_TIMEOUT for it; release it).
 */
#ifndef RGG_H_
#define RGG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rgg_roadmap* rgg_roadmap_t;

enum rgg_status {
  RGG_OK = 0,
  RGG_ERR_INVALID = -1,  /* bad argument, size, layout or id               */
  RGG_ERR_OOM = -2,      /* device or pinned-host allocation failed        */
  RGG_ERR_CUDA = -3,     /* a CUDA runtime call failed                     */
  RGG_ERR_TIMEOUT = -4,  /* a bounded device-side wait ran out             */
  RGG_ERR_STATE = -5,    /* call not valid in the roadmap's current state  */
  RGG_ERR_CAPACITY = -6, /* over a fixed capacity: rgg_classify_noalloc's     */
                         /* scratch, pending entries or open requests        */
  RGG_ERR_IO = -7        /* a file could not be opened, read or written      */
};

/* Geometry of a roadmap's approximations (rgg_roadmap_desc.geometry):
 *   SPHERES   inner spheres per configuration and outer spheres per interval
 *             (the default; every record streamed each pass);
 *   OBB       the paper's own primitives (Sec. 4.2, 4.3): one oriented box
 *             per (edge, body) as the outer approximation, tested against the
 *             moved boxes by the separating-axis test, and shortcut splines
 *             through the inscribed spheres' centres as the inner
 *             approximation, tested against each obstacle's inscribed sphere;
 *             a uniform grid over the edge boxes limits each pass to the cells
 *             the moved boxes meet (Sec. 4.3, spatial filtering). */
enum rgg_geometry { RGG_GEOMETRY_SPHERES = 0, RGG_GEOMETRY_OBB = 1 };

/* How rgg_build_edges stores a sphere-geometry roadmap's inner spheres
 * (rgg_roadmap_desc.record_format):
 *   LINK_ENDS  per (edge, link, configuration) only the far end of the link
 *              (12 B); the near end is the previous link's far end (the base,
 *              the world origin, for link 0) and the K inner spheres are
 *              interpolated on the GPU at fractions (j + 1/2)/K of the
 *              segment, radius R_i.  The default; it needs margin_m >= 1e-5 m
 *              (the interpolation adds under 1e-6 m of error), and a roadmap
 *              with a smaller margin stores SPHERES.
 *   SPHERES    every inner sphere (16 B each, K per link and configuration).
 * Uploaded records are always SPHERES. */
enum rgg_record_format { RGG_RECORDS_LINK_ENDS = 0, RGG_RECORDS_SPHERES = 1 };

/* Edge labels (Sec. 4.1): valid, unknown, invalid. */
enum rgg_label { RGG_GREEN = 0, RGG_GRAY = 1, RGG_RED = 2 };

/* Largest supported values. */
enum {
  RGG_MAX_LINKS = 32,          /* num_links                                    */
  RGG_MAX_INNER = 16,          /* inner_per_link                               */
  RGG_MAX_OBSTACLES = 4096,    /* max_obstacles                                */
  RGG_BOXES_PER_PASS = 32,     /* moved boxes tested per streaming pass        */
  RGG_NUM_VARIANTS = 13,       /* compiled pipeline shapes (rgg_set_launch_shape) */
  RGG_MAX_REQUESTS = 64,       /* open requests per roadmap (rgg_update_request) */
  RGG_PENDING_EXTRA = 4096,    /* pending entries beyond max_obstacles          */
  RGG_MAX_RESOLVE_FACTOR = 100, /* rgg_resolve_gray: resampling factor           */
  RGG_NOALLOC_MAX_EDGES = 131072,  /* rgg_classify_noalloc: edges per call          */
  RGG_NOALLOC_MAX_TILES = 16384    /* rgg_classify_noalloc: tiles of up to 527      */
                                   /* configurations x links per call               */
};

typedef struct {
  uint32_t num_links;       /* L: robot links (= joints), 1..RGG_MAX_LINKS        */
  uint32_t inner_per_link;  /* K: inner spheres per link, 1..RGG_MAX_INNER        */
  uint32_t max_obstacles;   /* M: box ids are 0..M-1, 1..RGG_MAX_OBSTACLES        */
  float margin_m;           /* delta in metres, >= 0 (2e-5 is the documented      */
                            /* default; it must exceed the FP32 rounding error)   */
  int device;               /* CUDA device ordinal                                */
  uint32_t geometry;        /* enum rgg_geometry (0 = spheres)                    */
  uint32_t record_format;   /* enum rgg_record_format (0 = link ends)             */
} rgg_roadmap_desc;

/* A serial arm in standard Denavit-Hartenberg form, for rgg_build_edges.
 * Joint i applies Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i); link i is the segment
 * between frame origins i and i+1 (the base frame is the world frame), a
 * capsule of radius radius[i].  Host arrays of num_links doubles. */
typedef struct {
  uint32_t num_links;
  const double* a;
  const double* alpha;
  const double* d;
  const double* radius;
} rgg_robot_desc;

/* Sizes of the resident data (rgg_roadmap_info). */
typedef struct {
  uint64_t num_edges;       /* N                                                  */
  uint64_t num_samples;     /* S = sum over edges of n_e (configurations)         */
  uint64_t num_inner;       /* K * L * S inner spheres                            */
  uint64_t num_outer;       /* L * (S - N) outer spheres                          */
  uint64_t record_bytes;    /* 16 * (num_inner + num_outer), or with link-end     */
                            /* records 12 * L * S + 16 * num_outer                */
  uint64_t device_bytes;    /* all device memory held by the roadmap              */
  uint32_t num_links, inner_per_link, max_obstacles, mask_words;
  uint32_t tile_samples;    /* configurations per streaming tile                  */
  uint64_t num_tiles;
  uint32_t pending_boxes;   /* pending entries (moved boxes not yet classified)   */
  uint32_t grid_ctas;       /* CTAs of the classify launch                        */
  uint32_t open_requests;   /* request handles in use (rgg_update_request)        */
  uint32_t pending_capacity;/* max_obstacles + RGG_PENDING_EXTRA                  */
  uint32_t geometry;        /* enum rgg_geometry                                  */
  uint32_t grid_cells;      /* OBB geometry: cells of the uniform grid            */
  uint64_t grid_items;      /* OBB geometry: (box, cell) incidences               */
  uint64_t spline_vertices; /* OBB geometry: kept spline vertices                 */
  uint32_t round_filter;    /* 1: the spatial filter is on and active (see below)  */
  uint32_t record_format;   /* enum rgg_record_format of the resident records     */
  uint32_t variant;         /* the roadmap's launch variant (rgg_set_launch_shape) */
  uint32_t last_variant;    /* the variant its last classify launch ran            */
} rgg_info;

/* ------------------------------------------------------------------------ */
/* Create an empty roadmap on desc->device: no edges, no boxes present (every
 * label GREEN once edges exist).  *out receives the handle; free it with
 * rgg_roadmap_destroy.  RGG_ERR_INVALID for a NULL or out-of-range desc,
 * RGG_ERR_OOM / RGG_ERR_CUDA if the device state cannot be allocated. */
int rgg_roadmap_create(const rgg_roadmap_desc* desc, rgg_roadmap_t* out);

/* Free every device and host resource of the roadmap (synchronises the
 * device first).  NULL is accepted and ignored. */
int rgg_roadmap_destroy(rgg_roadmap_t r);

/* ------------------------------------------------------------------------ */
/* Upload serialized edge approximations built by the caller (Sec. 4.3,
 * "Offline storage": built once, kept on the GPU).  Replaces any edges the
 * roadmap had and resets every label to GREEN and every per-edge box set
 * to empty; every box already placed keeps its pose and becomes pending, so
 * the next rgg_classify labels the new edges against all present boxes.
 *
 *   num_edges    N (0 allowed: an empty roadmap)
 *   sample_off   N+1 host uint64: edge e has n_e = sample_off[e+1] -
 *                sample_off[e] >= 2 configurations; sample_off[0] = 0.
 *                Always a host array.
 *   inner_xyzr   4 planes of K*L*S floats each (x plane, then y, z, radius),
 *                S = sample_off[N].  Sphere (e, link i, sample k, sphere j)
 *                is element K*(L*sample_off[e] + i*n_e + k) + j of each plane.
 *   outer_xyzr   4 planes of L*(S-N) floats each.  Sphere (e, link i,
 *                interval k), 0 <= k < n_e - 1, is element
 *                L*(sample_off[e] - e) + i*(n_e - 1) + k of each plane.
 *   src_is_device  0: inner/outer are host pointers; 1: device pointers.
 * Every radius must be >= 0 and every value finite (checked for host
 * sources only).  The method assumes inner inside outer: each inner sphere
 * of configuration k must lie inside the union of the outer spheres of the
 * intervals next to k (k-1..k and k..k+1), because inner spheres are tested
 * only against boxes those outer spheres touch.
 * Host-source records whose inner spheres of every configuration share one
 * radius and sit at equal steps on a segment (within 1e-6 m, as
 * rgg_build_edges writes them) are tested with interpolated centres when
 * margin_m >= 1e-5; all others sphere by sphere.  RGG_ERR_INVALID on a bad
 * layout; RGG_ERR_OOM if the records do not fit in device memory. */
int rgg_upload_edges(rgg_roadmap_t r, uint64_t num_edges, const uint64_t* sample_off,
                     const float* inner_xyzr, const float* outer_xyzr, int src_is_device,
                     void* stream);

/* Build the serialized approximations on the GPU from the edges themselves
 * (the offline preprocessing of Sec. 4.2 / 4.3), in FP64, stored as FP32
 * (inner radii rounded down, outer radii rounded up; link ends rounded to
 * nearest), in the roadmap's record format.  Same effect on the roadmap
 * state as rgg_upload_edges.
 *
 *   robot        the arm; robot->num_links must equal the roadmap's L.
 *   q_from, q_to N x L host doubles (row-major): edge e goes from q_from[e]
 *                to q_to[e] in joint space.
 *   step         resolution eps > 0 in radians.  Edge e gets
 *                n_e = max(2, ceil(max_j |q_to[e][j] - q_from[e][j]| / step) + 1)
 *                configurations q_k = q_from + (k / (n_e - 1)) (q_to - q_from)
 *                (Sec. 3.2's cfg(e), endpoints included).
 * Inner sphere j of link i at configuration q_k: centre at fraction
 * (j + 1/2)/K of the link segment, radius radius[i].  Outer sphere of link i
 * over [q_k, q_{k+1}]: centre = midpoint of link i at (q_k + q_{k+1})/2,
 * radius = l_i/2 + R_i + 1/2 sum_{j<=i} |dq_j| sum_{m=j..i} l_m with
 * l_m = sqrt(a_m^2 + d_m^2) and dq = q_{k+1} - q_k, which encloses every
 * point of the link's capsule over the whole interval.
 * RGG_ERR_INVALID for bad robot/edges/step; RGG_ERR_OOM if the records do
 * not fit in device memory. */
int rgg_build_edges(rgg_roadmap_t r, const rgg_robot_desc* robot, uint64_t num_edges,
                    const double* q_from, const double* q_to, double step, void* stream);

/* ------------------------------------------------------------------------ */
/* Move (or place for the first time) obstacles: box ids[m] takes the
 * absolute pose pose[15*m .. 15*m+14] = centre(3), R(9, row-major; its
 * columns are the box axes in world coordinates), half-extents(3), metres.
 * The box table row is overwritten in place on the stream (Sec. 4.3,
 * "Online updates"); the ids join the roadmap's pending set, tested by the
 * next rgg_classify.  Moving a box twice before classifying keeps the last
 * pose.  A box never moved is absent and affects no label.
 *   n_changed    number of ids (0 allowed)
 *   ids          host array, each < max_obstacles, no repeats within a call
 *   pose         n_changed * 15 floats, host (src_is_device = 0) or device
 *                (src_is_device = 1).  Host poses are checked: finite,
 *                half-extents >= 0, R orthonormal with det +1 to 1e-3.
 * RGG_ERR_INVALID on a bad id or pose (nothing is changed). */
int rgg_update_obstacles(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                         const float* pose, int src_is_device, void* stream);
/* Pending entries: the moved boxes wait, in the order they were moved, as
 * entries (box id, staged pose).  A move of a box that already has an entry
 * since the last request boundary (see rgg_update_request) replaces that
 * entry's pose; otherwise it appends an entry.  At most max_obstacles +
 * RGG_PENDING_EXTRA entries wait at once: a call that would exceed it
 * returns RGG_ERR_CAPACITY and changes nothing (classify first). */

/* A versioned move: the same as rgg_update_obstacles, and in addition the
 * labels as they stand once this move (and every earlier one) is applied
 * are kept as a snapshot under a request handle.  Several requests on one
 * roadmap may wait together: the next rgg_classify (or rgg_classify_many)
 * applies their moves in order in the same streaming passes, and request h's
 * snapshot equals the labels that classifying after h's own moves alone
 * would give.  (Sec. 4.3's online update, one obstacle change per request;
 * the paper has no request handles: they let a server fuse the updates of
 * many requests into one pass.)
 *   n_changed    >= 1 ids (same rules as rgg_update_obstacles)
 *   *handle      receives the request handle, 0 .. RGG_MAX_REQUESTS-1
 * The first request after edges are set allocates RGG_MAX_REQUESTS x N bytes
 * of snapshot memory.  RGG_ERR_STATE before edges exist; RGG_ERR_CAPACITY
 * when all RGG_MAX_REQUESTS handles are open or the pending entries are
 * full; RGG_ERR_INVALID as for rgg_update_obstacles.  Replacing the edges
 * (rgg_upload_edges / rgg_build_edges) closes every open handle. */
int rgg_update_request(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                       const float* pose, int src_is_device, uint32_t* handle, void* stream);

/* Copy request `handle`'s snapshot labels [first, first+count) to `out` (host,
 * device or asynchronous page-locked host, as in rgg_fetch_labels).  Valid once a classify call has been
 * enqueued after the request: the copy is ordered after it on `stream`.
 * RGG_ERR_STATE if the handle is not open or its classify has not been
 * enqueued yet. */
int rgg_fetch_request_labels(rgg_roadmap_t r, uint32_t handle, uint8_t* out, uint64_t first,
                             uint64_t count, int dst_is_device, void* stream);

/* Close a request handle whose classify has been enqueued, so that a later
 * request may reuse its snapshot memory.  Host-side only: a later classify
 * that reuses the handle overwrites the snapshot in stream order, so enqueue
 * (or finish) every copy of it before that classify on the same stream.
 * RGG_ERR_STATE if the handle is not open or not yet classified. */
int rgg_release_request(rgg_roadmap_t r, uint32_t handle);

/* Classify every edge against the pending moved boxes and merge with the
 * per-edge box sets, so that each label equals the label against the
 * current pose of every present box (Algorithm 1, lazy mode).  Streams all
 * resident records once per RGG_BOXES_PER_PASS pending boxes.  Asynchronous:
 * labels stay on the device.  Clears the pending set.  With no pending box
 * it launches nothing.  RGG_ERR_STATE before any edges were set. */
int rgg_classify(rgg_roadmap_t r, void* stream);

/* Classify several roadmaps (each with its own edges, robot and pending
 * boxes) in one persistent launch per pass over a shared work queue.  The
 * labels are the same as rgg_classify on each roadmap alone.  All roadmaps
 * must live on the same device; repeats are not allowed. */
int rgg_classify_many(rgg_roadmap_t* roadmaps, uint32_t n, void* stream);
/* (All roadmaps must also share the launch variant, see rgg_set_launch_shape.) */

/* Copy labels [first, first+count) (uint8, enum rgg_label) to `out`:
 *   dst_is_device = 0  a host buffer: the call waits for the stream and then
 *                      reports any latched device error;
 *                   1  a device buffer (asynchronous);
 *                   2  a page-locked host buffer, asynchronous: the caller
 *                      waits on the stream and then calls rgg_check_status.
 * RGG_ERR_INVALID if the range exceeds the edge count. */
int rgg_fetch_labels(rgg_roadmap_t r, uint8_t* out, uint64_t first, uint64_t count,
                     int dst_is_device, void* stream);

/* Copy the per-edge box sets of edges [first, first+count): hit[e][w] and
 * touch[e][w], w < mask_words = ceil(max_obstacles/32), bit b of word b/32
 * for box id b (Algorithm 1's intersection lists).  Either pointer may be
 * NULL.  Host or device destination as in rgg_fetch_labels. */
int rgg_fetch_box_sets(rgg_roadmap_t r, uint32_t* hit, uint32_t* touch, uint64_t first,
                       uint64_t count, int dst_is_device, void* stream);

/* Copy the resident records of edges [first, first+count) to host buffers in
 * the rgg_upload_edges layout restricted to that range (inner: 4 planes of
 * K*L*(sample_off[first+count]-sample_off[first]) floats; outer: 4 planes of
 * L*(samples - count) floats), and the N+1 sample offsets (host, may be NULL).
 * With link-end records the inner spheres are the ones the records stand
 * for: centres interpolated in FP64 from the stored FP32 link ends, then
 * rounded; radii R_i rounded down.  Synchronous.  For inspection and tests. */
int rgg_fetch_records(rgg_roadmap_t r, uint64_t first, uint64_t count, float* inner_xyzr,
                      float* outer_xyzr, uint64_t* sample_off);

/* Copy the box table: pose[15*b .. 15*b+14] (centre, R row-major,
 * half-extents; the last pose given to the box, pending or not) and
 * present[b] (1 once the box has been placed) for every box id b <
 * max_obstacles, to host arrays (either may be NULL).  Waits for `stream`. */
int rgg_fetch_boxes(rgg_roadmap_t r, float* pose, uint8_t* present, void* stream);

/* Device pointer to the label array (N bytes, valid until the edges are
 * replaced or the roadmap destroyed), for zero-copy use on the device. */
int rgg_labels_device_ptr(rgg_roadmap_t r, const uint8_t** out);

/* Sizes of the resident data. */
int rgg_roadmap_info(rgg_roadmap_t r, rgg_info* out);

/* Wait for the stream and report any latched device-side error
 * (RGG_ERR_TIMEOUT), clearing it and recovering as described at the top. */
int rgg_check_status(rgg_roadmap_t r, void* stream);

/* Limit, in nanoseconds of wall time, of every bounded wait in the classify
 * kernel (a worker warp waiting for its tile's records or for the box
 * records, a refilling warp waiting for the stage's prefetched tile
 * metadata).  A wait that runs out ends the launch with
 * RGG_ERR_TIMEOUT latched (see the top).  The default, 4 s, is far above any
 * wait of a healthy launch (microseconds); very small limits exist to test
 * the failure path.  RGG_ERR_INVALID for 0. */
int rgg_set_wait_limit(rgg_roadmap_t r, uint64_t limit_ns);

/* Fault injection for tests of the host's error paths: the nth device
 * allocation the library makes from now on (any roadmap, any call) fails as
 * if the device were out of memory, and the call that made it returns
 * RGG_ERR_OOM with the roadmap unchanged.  0 turns it off; it also turns off
 * by itself once it has fired.  The paper has no counterpart. */
int rgg_inject_alloc_failure(uint64_t nth);

/* Guard bytes, a check for writes past the end of a buffer where no memory
 * checker can run: every device buffer the library allocates is followed by
 * 64 bytes of a fixed pattern (0xA5) at its requested size rounded up to
 * 16 B.  rgg_check_guards synchronises each device that holds library buffers
 * (so it waits for all work on them), reads every live buffer's guard and
 * stores, when the pointers are not NULL, the number of buffers checked and
 * the number whose guard changed.  Returns RGG_OK when every guard is intact,
 * RGG_ERR_STATE when one changed (a kernel or copy wrote past a buffer's end)
 * and RGG_ERR_CUDA when a synchronisation or read failed.  Buffers are
 * listed from allocation to release, so a call made while another thread
 * creates or destroys roadmaps sees each buffer either whole or not at all.
 * A debugging aid; the paper has no counterpart. */
int rgg_check_guards(uint64_t* n_checked, uint64_t* n_bad);

/* Device bytes a sphere-geometry roadmap created with `desc` holds once
 * rgg_build_edges(num_edges, q_from, q_to, step) has run: record planes,
 * tile tables of the default launch shape, per-edge state, kept endpoints
 * the default spatial filter's round data (link-end records) and the fixed
 * per-roadmap tables, i.e. rgg_roadmap_info's device_bytes
 * after the build (the first rgg_update_request adds RGG_MAX_REQUESTS x N
 * bytes).  Host-only arithmetic: the configuration counts follow
 * rgg_build_edges' rule; the tile size uses desc->device's SM count (152 if
 * the device cannot be queried; it matters only for roadmaps too small to
 * give each SM two tiles).  RGG_ERR_INVALID for bad arguments (as for
 * rgg_roadmap_create / rgg_build_edges), RGG_ERR_STATE for the OBB geometry,
 * whose spline sizes are only known once built. */
int rgg_estimate_bytes(const rgg_roadmap_desc* desc, uint64_t num_edges, const double* q_from,
                       const double* q_to, double step, uint64_t* bytes);

/* Kernel timing: when enabled, rgg_classify records CUDA events on its stream
 * around each pass's streaming classify launch and its merge launch;
 * rgg_kernel_time returns the summed durations (ms) of each since the last
 * call and the number of passes timed, and resets them (it synchronises on
 * the events). */
int rgg_set_kernel_timing(rgg_roadmap_t r, int enable);
int rgg_kernel_time(rgg_roadmap_t r, double* classify_ms, double* merge_ms, uint64_t* launches);

/* Work counting: while enabled, rgg_classify runs the classify kernel's
 * counting instance (compiled for the two default launch shapes; other
 * shapes and rgg_classify_many count nothing), which adds up the work it
 * executes.  rgg_work_counts returns the totals since the last call (each
 * pointer may be NULL), waits for the device and resets them:
 *   rounds       rounds of 31 configurations examined (the spatial filter
 *                skips the others)
 *   outer_tests  outer sphere-box tests executed after the warp's bounding-
 *                sphere cull (the logical count is outer spheres x moved
 *                boxes)
 *   inner_pairs  (configuration, box) pairs given the inner test, each up to
 *                K sphere-box tests
 * The paper has no counterpart; it measures what the culling saves. */
int rgg_set_work_counting(rgg_roadmap_t r, int enable);
int rgg_work_counts(rgg_roadmap_t r, uint64_t* rounds, uint64_t* outer_tests,
                    uint64_t* inner_pairs);

/* Launch shape of the streaming classify kernel: `variant` picks one of the
 * compiled pipeline shapes (shared-memory ring depth x stage size x rounds of
 * 31 configurations per tile; RGG_NUM_VARIANTS in all, 0 = smallest tiles,
 * 5 the default for sphere records, 10 for link-end records; the spatial
 * filter runs with variants 5, 7, 10, 11 and 12 only; 12 is 10's tiles with
 * 3 rounds per work item, which a roadmap of at least 262,144 tiles left on
 * its default shape runs for a pass whose previous pass listed at least 95%
 * of its tiles) and `consumer_warps` the
 * warps per CTA that test records (0 = the format's default, 24 for sphere
 * records and 27 for link ends; 1..27).  With edges present the tiles are rebuilt for the new shape (the
 * call synchronises the device).  Roadmaps classified together by
 * rgg_classify_many must share the variant.  RGG_ERR_INVALID for an
 * unsupported shape (nothing changes). */
int rgg_set_launch_shape(rgg_roadmap_t r, uint32_t variant, uint32_t consumer_warps);

/* ------------------------------------------------------------------------ */
/* Non-lazy resolution of gray edges (Algorithm 1 with lazy = false: gray
 * edges are validated by a full check).  For every edge whose current label
 * is GRAY, the robot's link capsules (segment between consecutive frame
 * origins, radius R_i) are checked at (n_e - 1) * factor + 1 configurations
 * q(t) = q_from + t (q_to - q_from), t = c / ((n_e - 1) factor), which
 * include the edge's own configurations, against the boxes of the edge's
 * touch set (only boxes an outer sphere touched can meet a capsule).  The
 * clearance is the minimum over those configurations, links and boxes of
 * (distance from the capsule axis to the box - R_i), computed exactly per
 * (configuration, link, box) in FP32.  With thr = max(margin_m, 1e-5 m)
 * (the FP32 error stays below 5e-6 m):
 *   clearance <= -thr: RED (the robot collides at some checked configuration)
 *   clearance >= thr:  GREEN (it is free at every checked configuration)
 *   otherwise:         GRAY (too close to decide in FP32).
 * Edges that are not gray keep their label.  The roadmap's own labels and
 * box sets are not changed (the next classify works on the lazy state).
 *   factor         1 .. RGG_MAX_RESOLVE_FACTOR
 *   labels_out     N resolved labels (may be NULL)
 *   clearance_out  N floats: the gray edges' clearance (NaN for edges that
 *                  were not gray; a RED edge reports the first clearance
 *                  below -thr found, not the minimum) (may be NULL)
 *   dst_is_device  0: host buffers (the call waits); 1: device buffers
 *   stats          counts of gray edges, resolved red / green edges and
 *                  capsule-box evaluations (may be NULL; the call then
 *                  waits for the stream)
 * Needs edges built by rgg_build_edges (the robot and the endpoints are
 * kept) and no pending moves: RGG_ERR_STATE otherwise. */
typedef struct {
  uint64_t gray_edges;
  uint64_t resolved_red;
  uint64_t resolved_green;
  uint64_t evaluations;
} rgg_resolve_stats;

int rgg_resolve_gray(rgg_roadmap_t r, uint32_t factor, uint8_t* labels_out, float* clearance_out,
                     int dst_is_device, rgg_resolve_stats* stats, void* stream);

/* ------------------------------------------------------------------------ */
/* Persistence: the resident roadmap to and from a file (Sec. 1: serialized
 * roadmap data is stored and reloaded between planning iterations; Sec. 4.3:
 * the serialized matrices are built once and kept).
 *
 * rgg_save writes the records, the per-edge state (box sets, counts,
 * labels), the box table and which boxes are present.  The roadmap must have
 * edges and no pending moves (RGG_ERR_STATE otherwise), so that the saved
 * labels are those of the saved boxes.  It waits for `stream` first, then
 * copies through a 64 MB page-locked buffer.
 *
 * rgg_load replaces the roadmap's edges and state with a saved file's.  The
 * roadmap must have the file's num_links, inner_per_link and max_obstacles
 * (RGG_ERR_INVALID otherwise, nothing changed); the margin and launch shape
 * stay the roadmap's own.  Pending moves are dropped and open request
 * handles closed.  After the call the labels, box sets and boxes equal the
 * saved ones, and later updates classify as they would have on the saved
 * roadmap.  Synchronous.
 *
 * File layout (little-endian): a 96-byte header ("RGGSAVE1", version, L, K,
 * M, mask words, margin, flags, N, S, inner and outer counts), then
 * sample_off[N+1] (uint64), inner planes (4 x K*L*S float; with link-end
 * records, flag bit 1, 3 x L*S float followed by 32 link radii), outer
 * planes (4 x L*(S-N) float), hit and touch sets (2 x N x mask words
 * uint32), counts[N] (uint32), labels[N] (uint8), box table (M x 16 float),
 * present[M] (uint8), and a 64-bit checksum of everything before it.  A
 * roadmap loads either record format.
 * RGG_ERR_IO if the file cannot be opened, read or written; RGG_ERR_INVALID
 * for a header that does not match, a truncated file or a checksum
 * mismatch. */
int rgg_save(rgg_roadmap_t r, const char* path, void* stream);
int rgg_load(rgg_roadmap_t r, const char* path, void* stream);

/* Sphere geometry only: the spatial filter (Sec. 4.3, "spatially filtered
 * many-to-many checking", here over the streamed records).  By default it is
 * on for link-end records (where the classify kernel is bound by its work per
 * round, and skipping rounds no moved box can reach pays) and off for sphere
 * records; rgg_set_round_filter(r, 0 or 1) overrides the default.
 * While it is on, every round of 31 configurations of a tile
 * (rgg_info.tile_samples configurations per tile) has a bounding sphere of
 * its outer spheres and every tile a sphere holding its rounds' spheres
 * (computed when it is switched on and whenever the tiles change).  Before
 * each pass a small kernel tests those spheres against the pass's moved
 * boxes (exact box distance, radius plus margin, FP32 slack 1e-5 m) and lists
 * the tiles some box may reach; the classify kernel takes only the listed
 * tiles, copies only their runs of rounds some box may reach, and tests only
 * the boxes that may reach each round.  Labels and box sets are the same with
 * and without it (a round no box reaches holds no touch).  It applies with
 * the default launch shape only (rgg_info.round_filter reports whether it is
 * active).  Its data take 24 B per round slot (32 per tile) plus 20 B per
 * tile.
 * rgg_set_round_filter synchronises the device.  RGG_ERR_STATE on an
 * OBB-geometry roadmap.
 * rgg_streamed_bytes returns the record bytes (inner and outer planes, with
 * the 16-byte rounding of each copy) the filtered classify launches of this
 * roadmap copied since the last call, and resets the count; it waits for the
 * device.  Launches without the filter copy every record (record_bytes plus
 * the rounding) and are not counted, nor are the autotuner's. */
int rgg_set_round_filter(rgg_roadmap_t r, int enable);
int rgg_streamed_bytes(rgg_roadmap_t r, uint64_t* record_bytes);

/* OBB geometry only.  rgg_set_obb_filter(r, 0) makes every pass test the
 * moved boxes against the boxes of every non-empty grid cell instead of the
 * cells they meet (same bits; for measuring the filter).  rgg_obb_work
 * returns the separating-axis tests and spline-segment tests run since the
 * last call, and resets them (it waits for the device).  RGG_ERR_STATE on a
 * sphere-geometry roadmap. */
int rgg_set_obb_filter(rgg_roadmap_t r, int enable);
/* Copy the OBB geometry's records to host arrays (any may be NULL):
 *   obb      N*L boxes of 16 floats: centre (3), 0, then for k = 1..3 the
 *            axis u_k (3) and its half-extent -- box (e, body i) at e*L + i
 *   spl_off  N*L*K + 1 offsets: spline (e, i, s) at (e*L + i)*K + s owns
 *            vertices [spl_off[k], spl_off[k+1])
 *   spl_v    spline_vertices (rgg_info) vertices of 4 floats (x, y, z, 0).
 * Synchronous.  RGG_ERR_STATE without edges or for the sphere geometry. */
int rgg_fetch_obb_records(rgg_roadmap_t r, float* obb, uint64_t* spl_off, float* spl_v);
int rgg_obb_work(rgg_roadmap_t r, uint64_t* sat_tests, uint64_t* segment_tests);

/* ------------------------------------------------------------------------ */
/* Autotuner of the classify launch shape (the paper has none: its batched
 * pass has fixed sizes).  Times one streaming classify launch over the given
 * roadmaps at every supported shape -- each compiled pipeline variant (ring
 * depth x tile size, i.e. records per block) with 16, 20, 24 and 27 consumer
 * warps -- on their own resident records and their first 32 present boxes
 * (warm-up launch, then `reps` launches each timed by its own CUDA events on
 * `stream`; the median counts), and sets the fastest shape on every roadmap.  Labels, box sets and pending
 * moves are not changed: the timed launches accumulate into scratch memory
 * the call allocates and frees.  Synchronous; it synchronises the device
 * whenever the tiles are rebuilt.
 *   roadmaps, n  1 <= n <= 128 distinct roadmaps with edges, one device
 *   reps         timed launches per shape (clamped to 1..100)
 *   results      up to max_results entries, fastest first (may be NULL when
 *                max_results is 0); *n_results (may be NULL) = shapes timed.
 * With no present box on any roadmap nothing is timed and the shapes stay.
 * RGG_ERR_STATE before edges exist. */
typedef struct {
  uint32_t variant;         /* pipeline variant (rgg_set_launch_shape)          */
  uint32_t consumer_warps;  /* consumer warps per CTA                          */
  float classify_ms;        /* median duration of the timed launches, ms       */
  float reserved;
} rgg_tune_result;

int rgg_autotune(rgg_roadmap_t* roadmaps, uint32_t n, uint32_t reps, rgg_tune_result* results,
                 uint32_t max_results, uint32_t* n_results, void* stream);

/* ------------------------------------------------------------------------ */
/* Step graphs: one update-and-classify step of several roadmaps captured once
 * into a CUDA graph and replayed by a single launch (the paper launches each
 * step's work from the host).  The captured step moves, for each roadmap i,
 * the n_ids[i] boxes ids[i] to the poses read at each launch from the DEVICE
 * pointer poses[i] (n_ids[i] x 15 floats, same layout as
 * rgg_update_obstacles; the caller refreshes them between launches), then
 * classifies every roadmap as rgg_classify_many does.  Creating the graph
 * records the step's effect on the roadmaps' host-side state (boxes become
 * present), enqueues no work, and returns the handle in *out.
 * Rules:
 *   - at creation and at every launch the roadmaps must have no pending
 *     moves (RGG_ERR_STATE otherwise): the step uses the pending entries'
 *     staging rows;
 *   - replacing a roadmap's edges or changing its launch variant invalidates
 *     the graph (its launch returns RGG_ERR_STATE);
 *   - destroy the graph before any of its roadmaps.
 * Launches are asynchronous on `stream`; labels equal those of the same
 * update + rgg_classify_many issued call by call.  n_ids[i] may be 0 (the
 * roadmap is only classified when it has pending boxes, i.e. not at all). */
typedef struct rgg_step_graph* rgg_step_graph_t;

int rgg_step_graph_create(rgg_roadmap_t* roadmaps, uint32_t n, const uint32_t* n_ids,
                          const uint32_t* const* ids, const float* const* poses,
                          rgg_step_graph_t* out);
int rgg_step_graph_launch(rgg_step_graph_t g, void* stream);
/* Number of nodes in the captured graph (kernel launches and memsets). */
int rgg_step_graph_nodes(rgg_step_graph_t g, uint64_t* nodes);
int rgg_step_graph_destroy(rgg_step_graph_t g);

/* ------------------------------------------------------------------------ */
/* One classification pass that allocates nothing.  (The paper has no
 * counterpart: this entry point exists for callers of this library that may
 * not allocate device memory -- a real-time loop that must not wait on the
 * driver's allocator, a host whose memory manager owns every device byte, or
 * a plugin that may only launch work on buffers it is handed.)
 *
 * The caller owns the serialized records and the per-edge state, in device
 * memory, laid out as below; the call tests every edge against the given
 * moved boxes and merges the results into the per-edge state as
 * rgg_classify does: the same kernels, and with regular_records set as
 * rgg_classify would set it for the same records, the same labels and box
 * sets bit for bit.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch (tile tables, per-edge
 * accumulators, box records; about 3.7 MB) is a fixed array inside the
 * library, held by every device that loads the library until the process
 * exits.  On each device the first call looks up that array's address; make
 * that first call before any stream capture.  All calls share the array and
 * clear what must start at zero, so calls that overlap on the GPU (on
 * different streams, or from several threads) race: order them.  The call
 * works on the current device and stream; it returns once the work is
 * enqueued.
 *
 * Layout (all pointers device, except box_ids / box_poses which are host):
 *   sample_off   N+1 uint64 configuration offsets, as for rgg_upload_edges
 *                (n_e >= 2); num_samples must equal sample_off[N]
 *   inner_xyzr   4 planes at inner_xyzr + p*inner_stride (floats), each with
 *                K*L*num_samples spheres in the rgg_upload_edges order;
 *                16-byte aligned, stride a multiple of 4 and >= count + 4
 *   outer_xyzr   likewise, L*(num_samples - N) spheres per plane
 *   box_ids      num_boxes (<= 32) distinct ids, each < 32*mask_words
 *   box_poses    num_boxes x 15 floats: centre, R (row-major), half-extents
 *   hit, touch   N x mask_words uint32 box sets (in/out), bit b of word b/32
 *   counts       N uint32: hit-set size | touch-set size << 16 (in/out);
 *                zero together with the sets before the first call
 *   labels       N uint8 (out), enum rgg_label
 *   regular_records  1 if every configuration's K inner spheres share one
 *                radius and sit at equal steps on a segment, as
 *                rgg_build_edges writes them (records read back with
 *                rgg_fetch_records from such a roadmap are); the inner test
 *                then interpolates the centres when margin_m >= 1e-5, as
 *                rgg_classify does.  0: sphere by sphere.  The library cannot
 *                check device records: set it only for such records.
 *   status       optional device int (may be NULL): 0 once the pass has
 *                finished, else the code of a bounded wait that ran out, in
 *                which case hit, touch, counts and labels were left as they
 *                were (run the call again)
 *   wait_limit_ns  limit of the kernel's bounded waits (0: 4 s), as
 *                rgg_set_wait_limit
 * Limits: N <= RGG_NOALLOC_MAX_EDGES and at most RGG_NOALLOC_MAX_TILES tiles
 * (tiles hold up to 527 configurations x links, fewer for robots with few
 * links); larger inputs return RGG_ERR_CAPACITY and nothing is launched.
 * RGG_ERR_INVALID for bad sizes, alignment, ids or poses.  A sample_off that
 * breaks its rules gives undefined labels but no out-of-bounds access. */
typedef struct {
  uint32_t num_links, inner_per_link;
  uint64_t num_edges, num_samples;
  const uint64_t* sample_off;
  const float* inner_xyzr;
  uint64_t inner_stride;
  const float* outer_xyzr;
  uint64_t outer_stride;
  uint32_t num_boxes;
  const uint32_t* box_ids;
  const float* box_poses;
  uint32_t mask_words;
  uint32_t* hit;
  uint32_t* touch;
  uint32_t* counts;
  uint8_t* labels;
  float margin_m;
  uint32_t regular_records;
  int* status;
  uint64_t wait_limit_ns;
} rgg_noalloc_args;

int rgg_classify_noalloc(const rgg_noalloc_args* args, void* stream);

/* Static description of a status code (never NULL). */
const char* rgg_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RGG_H_ */
