// Internal header of the host side: the per-roadmap state and the helpers the
// host translation units share (not part of the C ABI).
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rgg.h"
#include "rgg_kernels.h"

namespace rgg_host {

using namespace rgg;

// A named NVTX range around a C-ABI call, for timeline tools (Nsight Systems,
// ncu --nvtx): without a tool attached the calls do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RGG_OK;
  cudaGetLastError();  // clear sticky-free errors so the next call starts clean
  return e == cudaErrorMemoryAllocation ? RGG_ERR_OOM : RGG_ERR_CUDA;
}

#define RGG_CK(call)                         \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// Every device allocation of the library goes through here, so that a test
// can make the n-th one fail (rgg_inject_alloc_failure) and so that each
// buffer carries guard bytes after its end (rgg_check_guards).  Buffers from
// device_alloc are released with device_free.
cudaError_t device_alloc(void** p, size_t bytes);
void device_free(void* p);

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return device_alloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// Smallest margin for which interpolated inner centres are used (their error
// is below 2e-6 m, the FP32 tests' below 1e-6 m).
constexpr float kRegularMinMargin = 1e-5f;

// Streaming tile geometry of one roadmap (see the classify kernel): each
// stage buffer holds a header, the tile's edge table, 4 inner planes (or 3
// link-end planes) and 4 outer planes.
struct Tiling {
  uint32_t S = 0, max_edges = 0;
  uint32_t off_in = 0, off_out = 0, in_cap = 0, out_cap = 0;
};

inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }
inline uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

// A window of S consecutive global samples meets at most S/(2L) + 2 edges
// (every edge has at least 2L samples); one more entry of slack.  Link-end
// planes hold the tile's S entries, up to max_n halo entries before them
// (the longest edge's configuration count bounds a link's run) and the
// 16-byte rounding of the copy.
inline bool tiling_for(uint32_t L, uint32_t K, uint32_t S, uint32_t stage_bytes, bool joints,
                       uint32_t max_n, Tiling* t) {
  t->S = S;
  t->max_edges = S / (2 * L) + 3;
  t->off_in = align16(kStageEtabOff + 16 * t->max_edges);
  t->in_cap = joints ? round4(S + max_n + 8) : round4(K * S + 8);
  t->off_out = t->off_in + (joints ? 12 : 16) * t->in_cap;
  t->out_cap = round4(S + 1 + 8);
  return t->max_edges <= (uint32_t)kMaxTileEdges &&
         (uint64_t)t->off_out + 16ull * t->out_cap <= (uint64_t)stage_bytes;
}

// Tiles of 31*rounds samples (full rounds) when they fit a stage, else the
// largest that does; smaller only for roadmaps too small to give every CTA of
// a launch two tiles (big tiles keep the producer warp's per-tile cost low).
// S = 0 when nothing fits (link-end records of an edge longer than a stage).
inline Tiling choose_tiling(uint32_t L, uint32_t K, uint64_t G, uint32_t warps, int variant,
                            bool joints = false, uint32_t max_n = 0) {
  // `warps`: how many tiles the roadmap should at least be cut into
  const VariantShape v = variant_shape(variant);
  uint32_t smax = 31 * v.rounds;
  Tiling t;
  while (smax > 1 && !tiling_for(L, K, smax, v.stage_bytes, joints, max_n, &t)) --smax;
  if (!tiling_for(L, K, smax, v.stage_bytes, joints, max_n, &t)) return Tiling();
  const uint64_t want = (G + warps - 1) / std::max<uint32_t>(warps, 1);
  uint32_t s = (uint32_t)std::min<uint64_t>(smax, std::max<uint64_t>(want, 31));
  s = std::max<uint32_t>(1, std::min(s, smax));
  tiling_for(L, K, s, v.stage_bytes, joints, max_n, &t);
  return t;
}

struct EdgeState {
  uint64_t N = 0, S_tot = 0, G = 0, n_inner = 0, n_outer = 0;
  uint64_t in_stride = 0, out_stride = 0;
  std::vector<uint64_t> h_soff;
  uint64_t* d_soff = nullptr;
  float* d_inner = nullptr;
  float* d_outer = nullptr;
  TileDesc* d_tiles = nullptr;
  int4* d_etab = nullptr;
  uint64_t T = 0, n_etab = 0;
  Tiling tiling;
  uint32_t* d_red = nullptr;
  uint32_t* d_touch = nullptr;
  uint32_t* d_counts = nullptr;
  uint8_t* d_labels = nullptr;
  uint32_t* d_edge_acc = nullptr;
  uint8_t* d_hist = nullptr;   // [RGG_MAX_REQUESTS][N] request snapshots, allocated on first use
  double* d_qa = nullptr;      // [N][L] edge endpoints (edges built by rgg_build_edges only)
  double* d_qb = nullptr;
  uint8_t* d_resolved = nullptr;  // [N] labels of the last gray resolution
  float* d_clear = nullptr;       // [N] its clearances
  uint32_t* d_gray = nullptr;     // [N] the gray edges a resolution lists
  // OBB / spline geometry (Sec. 4.2): boxes per (edge, body), spline CSR,
  // the uniform grid over the boxes, and the per-pass work list
  float4* d_obb = nullptr;        // [N * L][4]
  uint64_t* d_spl_off = nullptr;  // [N * L * K + 1]
  float4* d_spl_v = nullptr;      // spline vertices
  uint64_t n_obb = 0, n_spl = 0, n_spl_v = 0;
  GridSpec grid{};
  uint32_t n_cells = 0;
  uint64_t n_items = 0;
  uint32_t* d_cell_off = nullptr;   // [cells + 1]
  float4* d_cell_items = nullptr;   // 2 per item: AABB low corner + index, high corner
  uint2* d_pairs = nullptr;         // [pair_cap]
  uint32_t pair_cap = 0;
  uint32_t* d_qcnt = nullptr;       // [2] query counters
  // spatial filter of the sphere geometry: per (tile, round) bounding sphere,
  // outer-record range and this pass's candidate boxes (see rgg_device.cuh)
  float4* d_rsph = nullptr;
  uint32_t* d_rout = nullptr;
  uint32_t* d_rcand = nullptr;
  uint32_t* d_tlist = nullptr;   // [T] this pass's listed tiles, then their count
  uint64_t device_bytes = 0;
  bool regular = false;        // inner spheres equally spaced with one radius per sample
  // link-end records (3 planes, see rgg_device.cuh) instead of inner spheres,
  // with per-tile halo counts; max_n = the longest edge's configurations
  bool joints = false;
  uint32_t* d_tile_halo = nullptr;
  uint32_t max_n = 0;

  void release() {
    device_free(d_soff);
    device_free(d_inner);
    device_free(d_outer);
    device_free(d_tiles);
    device_free(d_etab);
    device_free(d_red);
    device_free(d_touch);
    device_free(d_counts);
    device_free(d_labels);
    device_free(d_edge_acc);
    device_free(d_hist);
    device_free(d_qa);
    device_free(d_qb);
    device_free(d_resolved);
    device_free(d_clear);
    device_free(d_gray);
    device_free(d_obb);
    device_free(d_spl_off);
    device_free(d_spl_v);
    device_free(d_cell_off);
    device_free(d_cell_items);
    device_free(d_pairs);
    device_free(d_qcnt);
    device_free(d_rsph);
    device_free(d_rout);
    device_free(d_rcand);
    device_free(d_tlist);
    device_free(d_tile_halo);
    *this = EdgeState();
  }
};

}  // namespace rgg_host

struct rgg_roadmap {
  using EdgeState = rgg_host::EdgeState;
  int device = 0;
  uint32_t L = 0, K = 0, M = 0, Wm = 0;
  float margin = 2e-5f;
  int num_sms = 0;
  uint32_t ctas_per_sm = 1, consumer_warps = rgg::kDefaultConsumerWarps;
  int variant = rgg::kDefaultVariant;
  bool shape_set = false;      // the caller or the autotuner chose the launch shape
  int last_variant = -1;       // the variant the last classify launch ran
  // the spatial filter's listed-tile count of the last single-roadmap pass,
  // copied to page-locked memory after the pass (read back one pass later,
  // so it may be a pass old; it only picks between variants 10 and 12)
  uint32_t* h_listed = nullptr;
  uint32_t* d_listed = nullptr;  // its device address
  bool has_edges = false;
  uint64_t gen = 0;            // bumped whenever tiles or edges are replaced
  uint32_t geometry = RGG_GEOMETRY_SPHERES;
  bool obb_filter = true;      // spatial grid filtering of the OBB queries
  // spatial filtering of the sphere geometry's records: -1 the default (on
  // for link-end records, off for sphere records), 0 off, 1 on
  int round_filter_mode = -1;
  unsigned long long* d_streamed = nullptr;  // [1] record bytes the classify launches copied
  unsigned long long* d_obbwork = nullptr;  // [2] SAT tests, spline-segment tests
  // the robot of edges built by rgg_build_edges (for the gray resolution)
  bool has_robot = false;
  double dh_a[RGG_MAX_LINKS], dh_alpha[RGG_MAX_LINKS], dh_d[RGG_MAX_LINKS], dh_radius[RGG_MAX_LINKS];
  unsigned long long* d_work = nullptr;  // [6] resolution counters and the gray list's cursors
  unsigned long long* d_count = nullptr; // [3] classify work counters (rgg_work_counts)
  bool counting = false;
  EdgeState es;
  float* d_table = nullptr;    // [M][16] box poses
  float* d_stage = nullptr;    // [stage_rows][16] staged pose of each pending entry
  uint32_t stage_rows = 0;
  float* d_changed = nullptr;  // box area: [32][24] derived records of the pass, link radii
  uint32_t record_format = 0;  // 0: link-end records for built edges when the margin allows
  int* d_status = nullptr;          // [0] status word, [1] classify work counter
  uint64_t wait_ns = 4000000000ull; // limit of the classify kernel's bounded waits
  std::vector<uint8_t> present;
  // Pending entries in application order.  Entry i stages its pose in row
  // `row` of d_stage; `snap` >= 0 marks the last entry of a request whose
  // snapshot is taken right after it.  The trailing run is the entries after
  // the last snapshot; within it a box has at most one entry (run_idx[b]).
  struct Entry {
    uint32_t id, row;
    int32_t snap;
  };
  std::vector<Entry> pending;
  std::vector<int32_t> run_idx;
  size_t run_start = 0;
  // request handles: 0 free, 1 waiting for a classify, 2 classified, 3 lost
  // to a device error (its snapshot is not valid; release it)
  std::vector<uint8_t> req_state;
  // kernel timing: events before classify, between classify and merge, after merge
  bool timing = false;
  std::vector<std::array<cudaEvent_t, 3>> events;
  size_t events_used = 0;
};

namespace rgg_host {

// rgg_api.cu
uint32_t launch_ctas(const rgg_roadmap* r);
bool build_tiles(uint32_t L, uint64_t N, const std::vector<uint64_t>& soff, uint64_t G, uint32_t S,
                 std::vector<TileDesc>* tiles, std::vector<int4>* etab,
                 std::vector<uint32_t>* halo = nullptr);
int set_tiles(rgg_roadmap* r, EdgeState* es, cudaStream_t s);
int alloc_edges(rgg_roadmap* r, EdgeState* es, uint64_t N, std::vector<uint64_t>&& soff,
                cudaStream_t s, bool joints = false);
bool use_joints(const rgg_roadmap* r);
void default_shape(rgg_roadmap* r, bool joints);
// Puts the launch shape back unless `keep` is set: new edges take their
// format's default shape, but a call that fails keeps the old edges, whose
// tiles belong to the old shape.
struct ShapeRestore {
  rgg_roadmap* r;
  int variant;
  uint32_t warps;
  bool keep = false;
  explicit ShapeRestore(rgg_roadmap* rm);
  ~ShapeRestore();
};
bool tiles_fit(const rgg_roadmap* r, int variant);
int set_link_radii(rgg_roadmap* r, const double* radius, cudaStream_t s);
void clear_pending(rgg_roadmap* r);
int requeue_present(rgg_roadmap* r, cudaStream_t s);
uint64_t fixed_device_bytes(const rgg_roadmap* r);
int install_edges(rgg_roadmap* r, EdgeState&& es, cudaStream_t s);
uint64_t round_data_bytes(uint64_t T);
void release_rounds(EdgeState* es);
int compute_rounds(rgg_roadmap* r, EdgeState* es, cudaStream_t s);
bool filter_active(const rgg_roadmap* r);
bool filter_wanted(const rgg_roadmap* r, const EdgeState* es);
bool valid_soff(const uint64_t* soff, uint64_t N, uint32_t L);
bool finite_planes(const float* p, uint64_t count, bool radius_plane);
bool regular_inner(const float* inner, uint64_t n_in, uint32_t K);
bool valid_pose(const float* p);
cudaEvent_t* next_events(rgg_roadmap* r);
ClassifyJob make_job(rgg_roadmap* r, uint32_t C, uint64_t tile_base);
MergeJob make_merge_job(rgg_roadmap* r, size_t lo, uint32_t C, bool ordered, uint64_t edge_base);
bool shape_ok(uint32_t variant, uint32_t cw);
int apply_shape(rgg_roadmap* r, int variant, uint32_t cw);
int check_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
                int src_is_device, uint32_t* new_entries);
int stage_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
                int src_is_device, cudaStream_t s);
int classify_group(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s);
int check_status_locked(rgg_roadmap_t r, cudaStream_t s);

// rgg_obb_host.cu
int build_obb(rgg_roadmap* r, EdgeState* es, const rgg_robot_desc* robot, const double* d_qa,
              const double* d_qb, cudaStream_t s);
int classify_group_obb(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s);

}  // namespace rgg_host
