// Host side of the C ABI declared in include/rgg.h: argument checks, device
// memory, tiling of the record stream, and kernel launches.  Every step of
// the classification runs in the kernels of rgg_kernels.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <utility>
#include <vector>

#include "rgg.h"
#include "rgg_kernels.h"

using namespace rgg;

namespace {

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

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RGG_OK;
  cudaGetLastError();  // clear sticky-free errors so the next call starts clean
  return e == cudaErrorMemoryAllocation ? RGG_ERR_OOM : RGG_ERR_CUDA;
}

#define RGG_CK(call)                         \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// Smallest margin for which interpolated inner centres are used (their error
// is below 2e-6 m, the FP32 tests' below 1e-6 m).
constexpr float kRegularMinMargin = 1e-5f;

// Streaming tile geometry of one roadmap (see the classify kernel): each
// stage buffer holds a header, the tile's edge table, 4 inner planes and 4
// outer planes.
struct Tiling {
  uint32_t S = 0, max_edges = 0;
  uint32_t off_in = 0, off_out = 0, in_cap = 0, out_cap = 0;
};

uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }
uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

// A window of S consecutive global samples meets at most S/(2L) + 2 edges
// (every edge has at least 2L samples); one more entry of slack.
bool tiling_for(uint32_t L, uint32_t K, uint32_t S, uint32_t stage_bytes, Tiling* t) {
  t->S = S;
  t->max_edges = S / (2 * L) + 3;
  t->off_in = align16(kStageEtabOff + 16 * t->max_edges);
  t->in_cap = round4(K * S + 8);
  t->off_out = t->off_in + 16 * t->in_cap;
  t->out_cap = round4(S + 1 + 8);
  return t->max_edges <= (uint32_t)kMaxTileEdges &&
         (uint64_t)t->off_out + 16ull * t->out_cap <= (uint64_t)stage_bytes;
}

// Tiles of 31*rounds samples (full rounds) when they fit a stage, else the
// largest that does; smaller only for roadmaps too small to give every CTA of
// a launch two tiles (big tiles keep the producer warp's per-tile cost low).
Tiling choose_tiling(uint32_t L, uint32_t K, uint64_t G, uint32_t warps, int variant) {
  // `warps`: how many tiles the roadmap should at least be cut into
  const VariantShape v = variant_shape(variant);
  uint32_t smax = 31 * v.rounds;
  Tiling t;
  while (smax > 1 && !tiling_for(L, K, smax, v.stage_bytes, &t)) --smax;
  const uint64_t want = (G + warps - 1) / std::max<uint32_t>(warps, 1);
  uint32_t s = (uint32_t)std::min<uint64_t>(smax, std::max<uint64_t>(want, 31));
  s = std::max<uint32_t>(1, std::min(s, smax));
  tiling_for(L, K, s, v.stage_bytes, &t);
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
  uint64_t device_bytes = 0;
  bool regular = false;        // inner spheres equally spaced with one radius per sample

  void release() {
    cudaFree(d_soff);
    cudaFree(d_inner);
    cudaFree(d_outer);
    cudaFree(d_tiles);
    cudaFree(d_etab);
    cudaFree(d_red);
    cudaFree(d_touch);
    cudaFree(d_counts);
    cudaFree(d_labels);
    cudaFree(d_edge_acc);
    cudaFree(d_hist);
    cudaFree(d_qa);
    cudaFree(d_qb);
    cudaFree(d_resolved);
    cudaFree(d_clear);
    cudaFree(d_obb);
    cudaFree(d_spl_off);
    cudaFree(d_spl_v);
    cudaFree(d_cell_off);
    cudaFree(d_cell_items);
    cudaFree(d_pairs);
    cudaFree(d_qcnt);
    *this = EdgeState();
  }
};

}  // namespace

struct rgg_roadmap {
  int device = 0;
  uint32_t L = 0, K = 0, M = 0, Wm = 0;
  float margin = 2e-5f;
  int num_sms = 0;
  uint32_t ctas_per_sm = 1, consumer_warps = kDefaultConsumerWarps;
  int variant = kDefaultVariant;
  bool has_edges = false;
  uint64_t gen = 0;            // bumped whenever tiles or edges are replaced
  uint32_t geometry = RGG_GEOMETRY_SPHERES;
  bool obb_filter = true;      // spatial grid filtering of the OBB queries
  unsigned long long* d_obbwork = nullptr;  // [2] SAT tests, spline-segment tests
  // the robot of edges built by rgg_build_edges (for the gray resolution)
  bool has_robot = false;
  double dh_a[RGG_MAX_LINKS], dh_alpha[RGG_MAX_LINKS], dh_d[RGG_MAX_LINKS], dh_radius[RGG_MAX_LINKS];
  unsigned long long* d_work = nullptr;  // [4] resolution counters
  EdgeState es;
  float* d_table = nullptr;    // [M][16] box poses
  float* d_stage = nullptr;    // [stage_rows][16] staged pose of each pending entry
  uint32_t stage_rows = 0;
  float* d_changed = nullptr;  // [32][24] derived records of the current pass
  int* d_status = nullptr;          // [0] status word, [1] classify work counter
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
  // request handles: 0 free, 1 waiting for a classify, 2 classified
  std::vector<uint8_t> req_state;
  // kernel timing: events before classify, between classify and merge, after merge
  bool timing = false;
  std::vector<std::array<cudaEvent_t, 3>> events;
  size_t events_used = 0;
};

namespace {

uint32_t launch_ctas(const rgg_roadmap* r) { return (uint32_t)r->num_sms * r->ctas_per_sm; }

// Tile descriptors and per-tile edge tables of a roadmap (see
// rgg_device.cuh): tile t covers global samples [t*S, min((t+1)*S, G)).
bool build_tiles(uint32_t L, uint64_t N, const std::vector<uint64_t>& soff, uint64_t G,
                 uint32_t S, std::vector<TileDesc>* tiles, std::vector<int4>* etab) {
  const uint64_t T = (G + S - 1) / S;
  tiles->resize(T);
  etab->clear();
  etab->reserve(N + T);
  uint64_t ef = 0;  // edge holding the tile's first sample
  for (uint64_t t = 0; t < T; ++t) {
    const uint64_t g0 = t * S, g1 = std::min<uint64_t>(g0 + S, G);
    while ((uint64_t)L * soff[ef + 1] <= g0) ++ef;
    uint64_t el = ef;
    while ((uint64_t)L * soff[el + 1] < g1) ++el;
    const uint64_t so_f = soff[ef], n_f = soff[ef + 1] - so_f;
    const uint64_t so_l = soff[el], n_l = soff[el + 1] - so_l;
    // first interval: the halo before the first sample when the tile starts
    // inside a link's run, else the run's first interval
    const uint64_t rf = g0 - L * so_f, i_f = rf / n_f, k_f = rf - i_f * n_f;
    const uint64_t o0 = L * (so_f - ef) + i_f * (n_f - 1) + (k_f > 0 ? k_f - 1 : 0);
    // last interval: the one after the last sample, or before it at a run's end
    const uint64_t rl = g1 - 1 - L * so_l, i_l = rl / n_l, k_l = rl - i_l * n_l;
    const uint64_t o1 = L * (so_l - el) + i_l * (n_l - 1) + std::min(k_l, n_l - 2) + 1;
    const uint64_t n_edges = el - ef + 1;
    if (n_edges > kMaxTileEdges || o1 - o0 > 0xffff || o0 >= (1ull << 40) ||
        etab->size() >= 0xffffffffull || el >= 0xffffffffull)
      return false;
    (*tiles)[t].packed = o0 | ((o1 - o0) << 40) | (n_edges << 56);
    (*tiles)[t].etab = (uint32_t)etab->size();
    (*tiles)[t].e_first = (uint32_t)ef;
    for (uint64_t e = ef; e <= el; ++e) {
      const int64_t estart = (int64_t)(L * soff[e]) - (int64_t)g0;
      const int64_t ostart = (int64_t)(L * (soff[e] - e)) - (int64_t)o0;
      const uint64_t n = soff[e + 1] - soff[e];
      float inv = 1.0f / (float)n;
      int inv_bits;
      std::memcpy(&inv_bits, &inv, sizeof(inv_bits));
      etab->push_back(make_int4((int)estart, (int)n, (int)ostart, inv_bits));
    }
  }
  return true;
}

// (Re)build the tile descriptors and edge tables of `es` for the roadmap's
// current launch shape and copy them to the device (synchronous).
int set_tiles(rgg_roadmap* r, EdgeState* es, cudaStream_t s) {
  Tiling tiling = choose_tiling(r->L, r->K, es->G, 2 * launch_ctas(r), r->variant);
  std::vector<TileDesc> h_tiles;
  std::vector<int4> h_etab;
  if (es->N && !build_tiles(r->L, es->N, es->h_soff, es->G, tiling.S, &h_tiles, &h_etab))
    return RGG_ERR_INVALID;
  TileDesc* d_tiles = nullptr;
  int4* d_etab = nullptr;
  cudaError_t e = dalloc(&d_tiles, h_tiles.size());
  if (e == cudaSuccess) e = dalloc(&d_etab, h_etab.size());
  if (e == cudaSuccess && !h_tiles.empty())
    e = cudaMemcpyAsync(d_tiles, h_tiles.data(), h_tiles.size() * sizeof(TileDesc),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !h_etab.empty())
    e = cudaMemcpyAsync(d_etab, h_etab.data(), h_etab.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s);
  // the host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(d_tiles);
    cudaFree(d_etab);
    return cuda_status(e);
  }
  es->device_bytes -= es->T * sizeof(TileDesc) + es->n_etab * sizeof(int4);
  cudaFree(es->d_tiles);
  cudaFree(es->d_etab);
  es->d_tiles = d_tiles;
  es->d_etab = d_etab;
  es->T = h_tiles.size();
  es->n_etab = h_etab.size();
  es->tiling = tiling;
  es->device_bytes += es->T * sizeof(TileDesc) + es->n_etab * sizeof(int4);
  return RGG_OK;
}

// Allocate the per-edge state and record planes for N edges with per-edge
// sample offsets h_soff (host), into `es` (not yet visible to the roadmap).
int alloc_edges(rgg_roadmap* r, EdgeState* es, uint64_t N, std::vector<uint64_t>&& soff,
                cudaStream_t s) {
  const bool spheres = r->geometry == RGG_GEOMETRY_SPHERES;
  es->N = N;
  es->h_soff = std::move(soff);
  es->S_tot = es->h_soff[N];
  es->G = (uint64_t)r->L * es->S_tot;
  es->n_inner = spheres ? (uint64_t)r->K * es->G : 0;
  es->n_outer = spheres ? (uint64_t)r->L * (es->S_tot - N) : 0;
  // plane stride: count + 4 floats of tail slack for 16-byte rounding of the
  // bulk copies, rounded to 64 floats (256 B) to keep planes aligned
  es->in_stride = ((es->n_inner + 4 + 63) / 64) * 64;
  es->out_stride = ((es->n_outer + 4 + 63) / 64) * 64;
  cudaError_t e = cudaSuccess;
#define RGG_AL(ptr, cnt)                 \
  if (e == cudaSuccess) {                \
    e = dalloc(&(ptr), (cnt));           \
    es->device_bytes += (cnt) * sizeof(*(ptr)); \
  }
  RGG_AL(es->d_soff, N + 1);
  if (spheres) {
    RGG_AL(es->d_inner, 4 * es->in_stride);
    RGG_AL(es->d_outer, 4 * es->out_stride);
  }
  RGG_AL(es->d_red, N * r->Wm);
  RGG_AL(es->d_touch, N * r->Wm);
  RGG_AL(es->d_counts, N);
  RGG_AL(es->d_labels, N);
  RGG_AL(es->d_edge_acc, 2 * N);
#undef RGG_AL
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(es->d_soff, es->h_soff.data(), (N + 1) * sizeof(uint64_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && N) {
    e = cudaMemsetAsync(es->d_red, 0, N * r->Wm * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_touch, 0, N * r->Wm * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_counts, 0, N * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_labels, RGG_GREEN, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_edge_acc, 0, 2 * N * 4, s);
  }
  if (e == cudaSuccess && spheres) {
    const int rc = set_tiles(r, es, s);
    if (rc != RGG_OK) {
      es->release();
      return rc;
    }
  }
  if (e == cudaSuccess && N && spheres) {
    // zero the padded tails so that the rounded bulk copies read defined data
    e = cudaMemsetAsync(es->d_inner, 0, 4 * es->in_stride * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_outer, 0, 4 * es->out_stride * sizeof(float), s);
  }
  if (e != cudaSuccess) {
    es->release();
    return cuda_status(e);
  }
  return RGG_OK;
}

void clear_pending(rgg_roadmap* r) {
  for (size_t i = r->run_start; i < r->pending.size(); ++i) r->run_idx[r->pending[i].id] = -1;
  r->pending.clear();
  r->run_start = 0;
}

// Swap in freshly built edges: labels GREEN, box sets empty, open requests
// closed, and every present box pending (its staged pose copied from the
// box table) so that the next classify tests it against the new edges.
int install_edges(rgg_roadmap* r, EdgeState&& es, cudaStream_t s) {
  r->es.release();
  r->es = std::move(es);
  r->has_edges = true;
  ++r->gen;
  clear_pending(r);
  std::fill(r->req_state.begin(), r->req_state.end(), 0);
  BoxUpdateParams p;
  p.n = 0;
  p.table = r->d_table;
  p.stage = r->d_stage;
  p.dev_pose = nullptr;
  p.from_table = 1;
  for (uint32_t b = 0; b < r->M; ++b) {
    if (!r->present[b]) continue;
    const uint32_t row = (uint32_t)r->pending.size();
    r->run_idx[b] = (int32_t)row;
    r->pending.push_back({b, row, -1});
    p.ids[p.n] = b;
    p.rows[p.n] = row;
    if (++p.n == kMaxUpdateBoxes) {
      RGG_CK(launch_box_update(p, s));
      p.n = 0;
    }
  }
  RGG_CK(launch_box_update(p, s));
  return RGG_OK;
}

// n_e >= 2 per edge; L*n_e and the edge count fit the 32-bit tile tables.
bool valid_soff(const uint64_t* soff, uint64_t N, uint32_t L) {
  if (!soff || soff[0] != 0 || N >= 0xffffffffull) return false;
  for (uint64_t e = 0; e < N; ++e) {
    if (soff[e + 1] < soff[e] + 2) return false;
    if ((soff[e + 1] - soff[e]) * (uint64_t)L > 0x7fffffffull) return false;
  }
  return true;
}

bool finite_planes(const float* p, uint64_t count, bool radius_plane) {
  for (uint64_t i = 0; i < count; ++i) {
    const float v = p[i];
    if (!std::isfinite(v) || (radius_plane && v < 0.0f)) return false;
  }
  return true;
}

// True when every sample's K inner spheres (consecutive in each plane) share
// one radius and their centres lie, within 1e-6 m per coordinate, at equal
// steps on the segment from the first centre to the last.
bool regular_inner(const float* inner, uint64_t n_in, uint32_t K) {
  const float* X = inner;
  const float* Y = inner + n_in;
  const float* Z = inner + 2 * n_in;
  const float* R = inner + 3 * n_in;
  for (uint64_t s = 0; s + K <= n_in; s += K) {
    for (uint32_t j = 1; j < K; ++j)
      if (R[s + j] != R[s]) return false;
    for (uint32_t j = 1; j + 1 < K; ++j) {
      const double t = (double)j / (double)(K - 1);
      const float* P[3] = {X, Y, Z};
      for (const float* c : P) {
        const double want = (double)c[s] + t * ((double)c[s + K - 1] - (double)c[s]);
        if (std::fabs((double)c[s + j] - want) > 1e-6) return false;
      }
    }
  }
  return true;
}

bool valid_pose(const float* p) {
  for (int c = 0; c < 15; ++c)
    if (!std::isfinite(p[c])) return false;
  for (int c = 12; c < 15; ++c)
    if (p[c] < 0.0f) return false;
  const float* R = p + 3;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double dot = 0;
      for (int m = 0; m < 3; ++m) dot += (double)R[3 * m + a] * R[3 * m + b];
      if (std::fabs(dot - (a == b ? 1.0 : 0.0)) > 1e-3) return false;
    }
  const double det = (double)R[0] * (R[4] * R[8] - R[5] * R[7]) -
                     (double)R[1] * (R[3] * R[8] - R[5] * R[6]) +
                     (double)R[2] * (R[3] * R[7] - R[4] * R[6]);
  return std::fabs(det - 1.0) <= 1e-3;
}

cudaEvent_t* next_events(rgg_roadmap* r) {
  if (r->events_used == r->events.size()) {
    std::array<cudaEvent_t, 3> ev{};
    for (int i = 0; i < 3; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
        return nullptr;
      }
    r->events.push_back(ev);
  }
  return r->events[r->events_used++].data();
}

ClassifyJob make_job(rgg_roadmap* r, uint32_t C, uint64_t tile_base) {
  ClassifyJob j{};
  const EdgeState& es = r->es;
  j.inner = es.d_inner;
  j.outer = es.d_outer;
  j.in_stride = es.in_stride;
  j.out_stride = es.out_stride;
  j.tiles = es.d_tiles;
  j.etab = es.d_etab;
  j.boxes = r->d_changed;
  j.edge_acc = es.d_edge_acc;
  j.G = es.G;
  j.tile_base = tile_base;
  j.num_tiles = es.T;
  j.L = r->L;
  j.K = r->K;
  j.S = es.tiling.S;
  j.C = C;
  j.off_in = es.tiling.off_in;
  j.off_out = es.tiling.off_out;
  j.in_cap = es.tiling.in_cap;
  j.out_cap = es.tiling.out_cap;
  j.margin = r->margin;
  // interpolated inner centres add up to ~2e-6 m of error on top of the FP32
  // rounding; the margin must cover both
  j.regular = (es.regular && r->margin >= kRegularMinMargin) ? 1u : 0u;
  j.inv_k = 1.0f / (float)r->K;
  j.inv_km1 = r->K > 1 ? 1.0f / (float)(r->K - 1) : 0.0f;
  return j;
}

// Merge job of entries [lo, lo+C) of the pending list.  `ordered` applies
// them one by one and takes the requests' snapshots; otherwise their ids are
// distinct and ascending.
MergeJob make_merge_job(rgg_roadmap* r, size_t lo, uint32_t C, bool ordered, uint64_t edge_base) {
  MergeJob m{};
  const EdgeState& es = r->es;
  m.red = es.d_red;
  m.touch = es.d_touch;
  m.counts = es.d_counts;
  m.labels = es.d_labels;
  m.edge_acc = es.d_edge_acc;
  m.num_edges = es.N;
  m.edge_base = edge_base;
  m.Wm = r->Wm;
  m.C = C;
  m.ordered = ordered ? 1u : 0u;
  m.hist = es.d_hist;
  for (uint32_t b = 0; b < C; ++b) {
    const auto& en = r->pending[lo + b];
    m.ids[b] = en.id;
    if (en.snap >= 0) {
      m.snap_mask |= 1u << b;
      m.snap_slot[b] = (uint8_t)en.snap;
    }
  }
  return m;
}

// A launch shape every kernel instance supports: threads within the launch
// bounds, the batched kernel's shared memory within the opt-in limit, and no
// more consumer warps than work items in the ring (so that the ring's phase
// parity stays unambiguous).
bool shape_ok(uint32_t variant, uint32_t cw) {
  if (variant >= (uint32_t)kNumVariants || cw < 1 || 32 * (cw + 1) > (uint32_t)kMaxClassifyThreads)
    return false;
  if (classify_smem_bytes((int)variant, cw) > 232448) return false;
  const VariantShape vs = variant_shape((int)variant);
  return (uint64_t)cw <=
         (uint64_t)vs.stages * ((vs.rounds + vs.rounds_per_item - 1) / vs.rounds_per_item);
}

// Switch a roadmap to a checked shape; the tiles depend on the variant only
// and are rebuilt when it changes (after the device has drained).
int apply_shape(rgg_roadmap* r, int variant, uint32_t cw) {
  const int old_v = r->variant;
  const uint32_t old_cw = r->consumer_warps;
  r->variant = variant;
  r->consumer_warps = cw;
  if (variant != old_v && r->has_edges && r->es.N && r->geometry == RGG_GEOMETRY_SPHERES) {
    cudaDeviceSynchronize();  // no launch may still read the old tiles
    const int rc = set_tiles(r, &r->es, nullptr);
    if (rc != RGG_OK) {
      r->variant = old_v;
      r->consumer_warps = old_cw;
      return rc;
    }
    ++r->gen;  // captured step graphs hold the old tiles
  }
  return RGG_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* rgg_status_string(int s) {
  switch (s) {
    case RGG_OK: return "ok";
    case RGG_ERR_INVALID: return "invalid argument";
    case RGG_ERR_OOM: return "out of memory";
    case RGG_ERR_CUDA: return "CUDA runtime error";
    case RGG_ERR_TIMEOUT: return "device-side wait timed out";
    case RGG_ERR_STATE: return "call not valid in the current state";
    case RGG_ERR_CAPACITY: return "over a fixed capacity (no-alloc scratch, pending entries, open requests)";
    case RGG_ERR_IO: return "file could not be opened, read or written";
    default: return "unknown status";
  }
}

int rgg_roadmap_create(const rgg_roadmap_desc* desc, rgg_roadmap_t* out) {
  if (!desc || !out) return RGG_ERR_INVALID;
  *out = nullptr;
  if (desc->num_links < 1 || desc->num_links > RGG_MAX_LINKS || desc->inner_per_link < 1 ||
      desc->inner_per_link > RGG_MAX_INNER || desc->max_obstacles < 1 ||
      desc->max_obstacles > RGG_MAX_OBSTACLES || !(desc->margin_m >= 0.0f) ||
      !std::isfinite(desc->margin_m) || desc->geometry > RGG_GEOMETRY_OBB)
    return RGG_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return RGG_ERR_CUDA;
  }
  if (desc->device < 0 || desc->device >= ndev) return RGG_ERR_INVALID;
  DeviceGuard g(desc->device);
  if (!g.ok) return RGG_ERR_CUDA;
  rgg_roadmap* r = new (std::nothrow) rgg_roadmap();
  if (!r) return RGG_ERR_OOM;
  r->device = desc->device;
  r->L = desc->num_links;
  r->K = desc->inner_per_link;
  r->M = desc->max_obstacles;
  r->Wm = (r->M + 31) / 32;
  r->margin = desc->margin_m;
  r->geometry = desc->geometry;
  r->present.assign(r->M, 0);
  r->run_idx.assign(r->M, -1);
  r->req_state.assign(RGG_MAX_REQUESTS, 0);
  r->stage_rows = r->M + RGG_PENDING_EXTRA;
  cudaError_t e = cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, r->device);
  if (e == cudaSuccess) e = dalloc(&r->d_table, (size_t)r->M * 16);
  if (e == cudaSuccess) e = dalloc(&r->d_stage, (size_t)r->stage_rows * 16);
  if (e == cudaSuccess) e = dalloc(&r->d_changed, (size_t)kBoxesPerPass * kBoxRecFloats);
  if (e == cudaSuccess) e = dalloc(&r->d_status, 4);
  if (e == cudaSuccess) e = dalloc(&r->d_work, 4);
  if (e == cudaSuccess) e = dalloc(&r->d_obbwork, 2);
  if (e == cudaSuccess) e = cudaMemset(r->d_obbwork, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(r->d_table, 0, (size_t)r->M * 16 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(r->d_status, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(r->d_table);
    cudaFree(r->d_stage);
    cudaFree(r->d_changed);
    cudaFree(r->d_status);
    cudaFree(r->d_work);
    cudaFree(r->d_obbwork);
    delete r;
    return cuda_status(e);
  }
  *out = r;
  return RGG_OK;
}

int rgg_roadmap_destroy(rgg_roadmap_t r) {
  if (!r) return RGG_OK;
  DeviceGuard g(r->device);
  cudaDeviceSynchronize();
  r->es.release();
  cudaFree(r->d_table);
  cudaFree(r->d_stage);
  cudaFree(r->d_changed);
  cudaFree(r->d_status);
  cudaFree(r->d_work);
  cudaFree(r->d_obbwork);
  for (auto& ev : r->events)
    for (cudaEvent_t x : ev) cudaEventDestroy(x);
  delete r;
  return RGG_OK;
}

int rgg_upload_edges(rgg_roadmap_t r, uint64_t num_edges, const uint64_t* sample_off,
                     const float* inner_xyzr, const float* outer_xyzr, int src_is_device,
                     void* stream) {
  if (!r || !sample_off) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;  // boxes and splines are built here
  if (!valid_soff(sample_off, num_edges, r->L)) return RGG_ERR_INVALID;
  if (num_edges && (!inner_xyzr || !outer_xyzr)) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t S_tot = sample_off[num_edges];
  const uint64_t n_in = (uint64_t)r->K * r->L * S_tot;
  const uint64_t n_out = (uint64_t)r->L * (S_tot - num_edges);
  if (!src_is_device && num_edges) {
    for (int p = 0; p < 4; ++p)
      if (!finite_planes(inner_xyzr + p * n_in, n_in, p == 3) ||
          !finite_planes(outer_xyzr + p * n_out, n_out, p == 3))
        return RGG_ERR_INVALID;
  }
  EdgeState es;
  std::vector<uint64_t> soff(sample_off, sample_off + num_edges + 1);
  int rc = alloc_edges(r, &es, num_edges, std::move(soff), s);
  if (rc != RGG_OK) return rc;
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 4 && e == cudaSuccess && num_edges; ++p) {
    e = cudaMemcpyAsync(es.d_inner + p * es.in_stride, inner_xyzr + p * n_in, n_in * 4, kind, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(es.d_outer + p * es.out_stride, outer_xyzr + p * n_out, n_out * 4, kind, s);
  }
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  // device-resident uploads are not inspected: they take the exact
  // per-sphere path
  es.regular = !src_is_device && num_edges && regular_inner(inner_xyzr, n_in, r->K);
  r->has_robot = false;
  return install_edges(r, std::move(es), s);
}

// OBB geometry (Sec. 4.2, 4.3): per (edge, body) boxes and shortcut splines
// built on the GPU in FP64 (spline vertices counted, then written at their
// offsets), then the uniform grid over the boxes: cells of about the boxes'
// mean largest AABB side, at most 32 per axis, each listing the boxes whose
// AABB meets it.
static int build_obb(rgg_roadmap* r, EdgeState* es, const rgg_robot_desc* robot, const double* d_qa,
                     const double* d_qb, cudaStream_t s) {
  const uint64_t N = es->N;
  const uint32_t L = r->L, K = r->K;
  es->n_obb = N * L;
  es->n_spl = N * L * K;
  uint64_t max_n = 2;
  for (uint64_t e = 0; e < N; ++e) max_n = std::max<uint64_t>(max_n, es->h_soff[e + 1] - es->h_soff[e]);
  const uint64_t per_warp = max_n * 3 * (L + 1);
  if (per_warp * sizeof(double) > (256ull << 20)) return RGG_ERR_CAPACITY;
  uint64_t warps = std::min<uint64_t>(std::max<uint64_t>(N, 1), (uint64_t)r->num_sms * 32);
  while (warps > 8 && warps * per_warp * sizeof(double) > (1ull << 30)) warps /= 2;
  double* scratch = nullptr;
  uint32_t* d_count = nullptr;
  cudaError_t e = cudaSuccess;
  auto done = [&](int rc) {
    cudaFree(scratch);
    cudaFree(d_count);
    return rc;
  };
#define RGG_OB(ptr, cnt)                        \
  if (e == cudaSuccess) {                       \
    e = dalloc(&(ptr), (cnt));                  \
    es->device_bytes += (cnt) * sizeof(*(ptr)); \
  }
  RGG_OB(es->d_obb, 4 * es->n_obb);
  RGG_OB(es->d_spl_off, es->n_spl + 1);
  if (e == cudaSuccess) e = dalloc(&scratch, warps * per_warp);
  if (e == cudaSuccess) e = dalloc(&d_count, std::max<uint64_t>(es->n_spl, 1));
  if (e != cudaSuccess) return done(cuda_status(e));
  ObbBuildParams bp{};
  bp.L = L;
  bp.K = K;
  for (uint32_t i = 0; i < L; ++i) {
    bp.a[i] = robot->a[i];
    bp.alpha[i] = robot->alpha[i];
    bp.d[i] = robot->d[i];
    bp.radius[i] = robot->radius[i];
  }
  bp.qa = d_qa;
  bp.qb = d_qb;
  bp.soff = es->d_soff;
  bp.n_edges = N;
  bp.scratch = scratch;
  bp.scratch_per_warp = per_warp;
  bp.obb = es->d_obb;
  bp.spl_count = d_count;
  bp.pass = 0;
  e = launch_obb_build(bp, (uint32_t)warps, s);
  std::vector<uint32_t> count(es->n_spl);
  if (e == cudaSuccess && es->n_spl)
    e = cudaMemcpyAsync(count.data(), d_count, es->n_spl * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_status(e));
  std::vector<uint64_t> off(es->n_spl + 1, 0);
  for (uint64_t k = 0; k < es->n_spl; ++k) off[k + 1] = off[k] + count[k];
  es->n_spl_v = off[es->n_spl];
  RGG_OB(es->d_spl_v, std::max<uint64_t>(es->n_spl_v, 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(es->d_spl_off, off.data(), off.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  bp.spl_off = es->d_spl_off;
  bp.spl_v = es->d_spl_v;
  bp.pass = 1;
  if (e == cudaSuccess) e = launch_obb_build(bp, (uint32_t)warps, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_status(e));
  cudaFree(scratch);
  scratch = nullptr;
  // ---- the grid
  GridSpec g{};
  g.gx = g.gy = g.gz = 1;
  g.cell = 1.0f;
  if (es->n_obb) {
    const uint32_t blocks = (uint32_t)std::min<uint64_t>(1024, (es->n_obb + 255) / 256);
    float* d_part = nullptr;
    e = dalloc(&d_part, (size_t)blocks * 8);
    std::vector<float> part((size_t)blocks * 8);
    if (e == cudaSuccess) e = launch_obb_bounds(es->d_obb, es->n_obb, d_part, blocks, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(part.data(), d_part, part.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_part);
    if (e != cudaSuccess) return done(cuda_status(e));
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double side = 0.0;
    for (uint32_t b = 0; b < blocks; ++b) {
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], part[8 * b + k]);
        hi[k] = std::max(hi[k], part[8 * b + 3 + k]);
      }
      side += part[8 * b + 6];
    }
    if (!(std::isfinite(lo[0]) && std::isfinite(hi[0]) && std::isfinite(lo[1]) &&
          std::isfinite(hi[1]) && std::isfinite(lo[2]) && std::isfinite(hi[2])))
      return done(RGG_ERR_INVALID);
    const float ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    float cell = (float)(side / (double)es->n_obb);
    cell = std::max(cell, std::max(ext / 32.0f, 1e-3f));
    g.ox = lo[0];
    g.oy = lo[1];
    g.oz = lo[2];
    g.cell = cell;
    g.gx = std::min<uint32_t>(32, std::max<uint32_t>(1, (uint32_t)std::ceil((hi[0] - lo[0]) / cell)));
    g.gy = std::min<uint32_t>(32, std::max<uint32_t>(1, (uint32_t)std::ceil((hi[1] - lo[1]) / cell)));
    g.gz = std::min<uint32_t>(32, std::max<uint32_t>(1, (uint32_t)std::ceil((hi[2] - lo[2]) / cell)));
  }
  es->grid = g;
  es->n_cells = g.gx * g.gy * g.gz;
  uint32_t* d_cc = nullptr;
  e = dalloc(&d_cc, es->n_cells);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cc, 0, es->n_cells * sizeof(uint32_t), s);
  ObbGridParams gp{};
  gp.obb = es->d_obb;
  gp.n_obb = es->n_obb;
  gp.g = g;
  gp.cell_count = d_cc;
  gp.pass = 0;
  if (e == cudaSuccess) e = launch_obb_grid(gp, s);
  std::vector<uint32_t> cc(es->n_cells);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cc.data(), d_cc, cc.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(d_cc);
    return done(cuda_status(e));
  }
  std::vector<uint32_t> coff(es->n_cells + 1, 0);
  uint64_t items = 0;
  for (uint32_t c = 0; c < es->n_cells; ++c) {
    items += cc[c];
    if (items > 0xffffffffull) {
      cudaFree(d_cc);
      return done(RGG_ERR_CAPACITY);
    }
    coff[c + 1] = (uint32_t)items;
  }
  es->n_items = items;
  RGG_OB(es->d_cell_off, (uint64_t)es->n_cells + 1);
  RGG_OB(es->d_cell_items, 2 * std::max<uint64_t>(items, 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(es->d_cell_off, coff.data(), coff.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cc, 0, es->n_cells * sizeof(uint32_t), s);
  gp.cell_off = es->d_cell_off;
  gp.cell_cursor = d_cc;
  gp.cell_items = es->d_cell_items;
  gp.pass = 1;
  if (e == cudaSuccess) e = launch_obb_grid(gp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_cc);
  // every moved box may list every chunk of every cell
  es->pair_cap = (uint32_t)std::min<uint64_t>(
      0xffffffffull, (uint64_t)kBoxesPerPass * (es->n_cells + items / kObbChunk + 1));
  RGG_OB(es->d_pairs, es->pair_cap);
  RGG_OB(es->d_qcnt, 2);
#undef RGG_OB
  if (e != cudaSuccess) return done(cuda_status(e));
  return done(RGG_OK);
}

int rgg_build_edges(rgg_roadmap_t r, const rgg_robot_desc* robot, uint64_t num_edges,
                    const double* q_from, const double* q_to, double step, void* stream) {
  if (!r || !robot || robot->num_links != r->L || !robot->a || !robot->alpha || !robot->d ||
      !robot->radius)
    return RGG_ERR_INVALID;
  if (!(step > 0.0) || !std::isfinite(step)) return RGG_ERR_INVALID;
  if (num_edges && (!q_from || !q_to)) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < r->L; ++i)
    if (!std::isfinite(robot->a[i]) || !std::isfinite(robot->alpha[i]) ||
        !std::isfinite(robot->d[i]) || !std::isfinite(robot->radius[i]) || robot->radius[i] < 0)
      return RGG_ERR_INVALID;
  if (num_edges >= 0xffffffffull) return RGG_ERR_INVALID;  // tile table holds 32-bit edge ids
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t qn = num_edges * r->L;
  double *d_qa = nullptr, *d_qb = nullptr;
  uint64_t* d_counts = nullptr;
  int* d_bad = nullptr;
  std::vector<uint64_t> counts(num_edges);
  cudaError_t e = dalloc(&d_qa, qn);
  if (e == cudaSuccess) e = dalloc(&d_qb, qn);
  if (e == cudaSuccess) e = dalloc(&d_counts, num_edges);
  if (e == cudaSuccess) e = dalloc(&d_bad, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (e == cudaSuccess && qn) e = cudaMemcpyAsync(d_qa, q_from, qn * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && qn) e = cudaMemcpyAsync(d_qb, q_to, qn * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_count_samples(d_qa, d_qb, num_edges, r->L, step, d_counts, d_bad, s);
  int bad = 0;
  if (e == cudaSuccess && num_edges)
    e = cudaMemcpyAsync(counts.data(), d_counts, num_edges * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  auto cleanup = [&]() {
    cudaFree(d_qa);
    cudaFree(d_qb);
    cudaFree(d_counts);
    cudaFree(d_bad);
  };
  if (e != cudaSuccess) {
    cleanup();
    return cuda_status(e);
  }
  if (bad) {
    cleanup();
    return RGG_ERR_INVALID;
  }
  std::vector<uint64_t> soff(num_edges + 1, 0);
  for (uint64_t i = 0; i < num_edges; ++i) soff[i + 1] = soff[i] + counts[i];
  EdgeState es;
  int rc = alloc_edges(r, &es, num_edges, std::move(soff), s);
  if (rc != RGG_OK) {
    cleanup();
    return rc;
  }
  if (r->geometry == RGG_GEOMETRY_OBB) {
    rc = build_obb(r, &es, robot, d_qa, d_qb, s);
    if (rc != RGG_OK) {
      cleanup();
      es.release();
      return rc;
    }
  } else {
    BuildParams bp{};
    bp.L = r->L;
    bp.K = r->K;
    for (uint32_t i = 0; i < r->L; ++i) {
      bp.a[i] = robot->a[i];
      bp.alpha[i] = robot->alpha[i];
      bp.d[i] = robot->d[i];
      bp.radius[i] = robot->radius[i];
    }
    bp.qa = d_qa;
    bp.qb = d_qb;
    bp.soff = es.d_soff;
    bp.inner = es.d_inner;
    bp.outer = es.d_outer;
    bp.in_stride = es.in_stride;
    bp.out_stride = es.out_stride;
    bp.n_edges = num_edges;
    e = launch_build_records(bp, r->num_sms, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_counts);
  cudaFree(d_bad);
  if (e != cudaSuccess) {
    cudaFree(d_qa);
    cudaFree(d_qb);
    es.release();
    return cuda_status(e);
  }
  // the endpoints stay for the gray resolution
  es.d_qa = d_qa;
  es.d_qb = d_qb;
  es.device_bytes += 2 * qn * sizeof(double);
  es.regular = r->geometry == RGG_GEOMETRY_SPHERES;  // centres at (j + 1/2)/K, one radius per link
  rc = install_edges(r, std::move(es), s);
  if (rc == RGG_OK) {
    r->has_robot = true;
    for (uint32_t i = 0; i < r->L; ++i) {
      r->dh_a[i] = robot->a[i];
      r->dh_alpha[i] = robot->alpha[i];
      r->dh_d[i] = robot->d[i];
      r->dh_radius[i] = robot->radius[i];
    }
  }
  return rc;
}

// Checks a move's ids and host poses; counts the entries it would append.
static int check_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
                       int src_is_device, uint32_t* new_entries) {
  std::vector<uint8_t> seen(r->M, 0);
  uint32_t fresh = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (ids[i] >= r->M || seen[ids[i]]) return RGG_ERR_INVALID;
    seen[ids[i]] = 1;
    if (!src_is_device && !valid_pose(pose + 15 * (size_t)i)) return RGG_ERR_INVALID;
    if (r->run_idx[ids[i]] < 0) ++fresh;
  }
  *new_entries = fresh;
  return RGG_OK;
}

// Writes the poses into the box table and into the staging rows of the
// boxes' entries in the trailing run (appending entries where needed).
static int stage_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
                       int src_is_device, cudaStream_t s) {
  for (uint32_t base = 0; base < n; base += kMaxUpdateBoxes) {
    BoxUpdateParams p;
    p.n = std::min(kMaxUpdateBoxes, n - base);
    p.table = r->d_table;
    p.stage = r->d_stage;
    p.from_table = 0;
    p.dev_pose = src_is_device ? pose + 15 * (size_t)base : nullptr;
    for (uint32_t i = 0; i < p.n; ++i) {
      const uint32_t b = ids[base + i];
      if (r->run_idx[b] < 0) {
        r->run_idx[b] = (int32_t)r->pending.size();
        r->pending.push_back({b, (uint32_t)r->pending.size(), -1});
      }
      p.ids[i] = b;
      p.rows[i] = r->pending[r->run_idx[b]].row;
      r->present[b] = 1;
      if (!src_is_device) std::memcpy(p.pose[i], pose + 15 * (size_t)(base + i), 15 * sizeof(float));
    }
    RGG_CK(launch_box_update(p, s));
  }
  return RGG_OK;
}

int rgg_update_obstacles(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                         const float* pose, int src_is_device, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  if (n_changed == 0) return RGG_OK;
  if (!ids || !pose) return RGG_ERR_INVALID;
  uint32_t fresh = 0;
  int rc = check_moves(r, n_changed, ids, pose, src_is_device, &fresh);
  if (rc != RGG_OK) return rc;
  if (r->pending.size() + fresh > r->stage_rows) return RGG_ERR_CAPACITY;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  return stage_moves(r, n_changed, ids, pose, src_is_device, static_cast<cudaStream_t>(stream));
}

int rgg_update_request(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                       const float* pose, int src_is_device, uint32_t* handle, void* stream) {
  if (!r || !handle || n_changed == 0 || !ids || !pose) return RGG_ERR_INVALID;
  if (!r->has_edges) return RGG_ERR_STATE;
  uint32_t fresh = 0;
  int rc = check_moves(r, n_changed, ids, pose, src_is_device, &fresh);
  if (rc != RGG_OK) return rc;
  if (r->pending.size() + fresh > r->stage_rows) return RGG_ERR_CAPACITY;
  uint32_t h = 0;
  while (h < RGG_MAX_REQUESTS && r->req_state[h] != 0) ++h;
  if (h == RGG_MAX_REQUESTS) return RGG_ERR_CAPACITY;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  EdgeState& es = r->es;
  if (!es.d_hist && es.N) {
    cudaError_t e = dalloc(&es.d_hist, (size_t)RGG_MAX_REQUESTS * es.N);
    if (e != cudaSuccess) return cuda_status(e);
    es.device_bytes += (uint64_t)RGG_MAX_REQUESTS * es.N;
  }
  rc = stage_moves(r, n_changed, ids, pose, src_is_device, static_cast<cudaStream_t>(stream));
  if (rc != RGG_OK) return rc;
  // the request ends the trailing run: its snapshot follows the run's last entry
  r->pending.back().snap = (int32_t)h;
  for (size_t i = r->run_start; i < r->pending.size(); ++i) r->run_idx[r->pending[i].id] = -1;
  r->run_start = r->pending.size();
  r->req_state[h] = 1;
  *handle = h;
  return RGG_OK;
}

// One streaming pass per group of <= 32 pending entries; for several
// roadmaps, pass p of every roadmap that has one goes into the same
// persistent launch.  Without requests the entries (distinct boxes) are
// sorted so that each pass's ids ascend, for the merge kernel's word-grouped
// update; with requests they keep their order and merge one by one.
static int classify_group(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s) {
  uint32_t max_passes = 0;
  std::vector<uint8_t> ordered(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    auto& pend = rs[i]->pending;
    for (const auto& en : pend)
      if (en.snap >= 0) ordered[i] = 1;
    if (!ordered[i])
      std::sort(pend.begin(), pend.end(), [](const rgg_roadmap::Entry& a,
                                             const rgg_roadmap::Entry& b) { return a.id < b.id; });
    max_passes = std::max<uint32_t>(
        max_passes, (uint32_t)((rs[i]->pending.size() + kBoxesPerPass - 1) / kBoxesPerPass));
  }
  std::unique_ptr<BoxPrepParams> bpp(new (std::nothrow) BoxPrepParams);
  std::unique_ptr<ClassifyParams<kMaxJobs>> cpp;
  std::unique_ptr<MergeParams<kMaxJobs>> mpp;
  if (n > 1) {
    cpp.reset(new (std::nothrow) ClassifyParams<kMaxJobs>);
    mpp.reset(new (std::nothrow) MergeParams<kMaxJobs>);
  }
  if (!bpp || (n > 1 && (!cpp || !mpp))) return RGG_ERR_OOM;
  for (uint32_t pass = 0; pass < max_passes; ++pass) {
    BoxPrepParams& bp = *bpp;
    bp.njobs = 0;
    ClassifyParams<1> cp1;
    MergeParams<1> mp1;
    uint32_t nj = 0;
    uint64_t tiles = 0, edges = 0;
    rgg_roadmap* timed = nullptr;
    for (uint32_t i = 0; i < n; ++i) {
      rgg_roadmap* r = rs[i];
      const size_t lo = (size_t)pass * kBoxesPerPass;
      if (lo >= r->pending.size()) continue;
      const uint32_t C = (uint32_t)std::min<size_t>(kBoxesPerPass, r->pending.size() - lo);
      BoxPrepJob& pj = bp.job[bp.njobs++];
      pj.stage = r->d_stage;
      pj.out = r->d_changed;
      pj.C = C;
      for (uint32_t b = 0; b < C; ++b) {
        pj.ids[b] = r->pending[lo + b].id;
        pj.rows[b] = (uint16_t)r->pending[lo + b].row;
      }
      if (r->es.N == 0) continue;
      const ClassifyJob job = make_job(r, C, tiles);
      const MergeJob mj = make_merge_job(r, lo, C, ordered[i] != 0, edges);
      if (n == 1) {
        cp1.job[0] = job;
        mp1.job[0] = mj;
      } else {
        cpp->job[nj] = job;
        mpp->job[nj] = mj;
      }
      ++nj;
      tiles += r->es.T;
      edges += r->es.N;
      if (r->timing && !timed) timed = r;
    }
    RGG_CK(launch_box_prep(bp, s));
    if (nj == 0) continue;
    rgg_roadmap* r0 = rs[0];
    ClassifyLaunch lc;
    lc.consumer_warps = r0->consumer_warps;
    lc.variant = r0->variant;
    lc.grid = (uint32_t)std::min<uint64_t>((tiles + 1) / 2, launch_ctas(r0));
    lc.grid = std::max<uint32_t>(lc.grid, 1);
    uint32_t* counter = reinterpret_cast<uint32_t*>(r0->d_status + 1);
    RGG_CK(cudaMemsetAsync(counter, 0, sizeof(uint32_t), s));
    cudaEvent_t* ev = timed ? next_events(timed) : nullptr;
    if (ev) RGG_CK(cudaEventRecord(ev[0], s));
    if (n == 1) {
      cp1.njobs = 1;
      cp1.total_tiles = tiles;
      cp1.status = r0->d_status;
      cp1.work_counter = counter;
      RGG_CK(launch_classify_single(cp1, lc, s));
    } else {
      cpp->njobs = nj;
      cpp->total_tiles = tiles;
      cpp->status = r0->d_status;
      cpp->work_counter = counter;
      RGG_CK(launch_classify_batched(*cpp, lc, s));
    }
    if (ev) RGG_CK(cudaEventRecord(ev[1], s));
    if (n == 1) {
      mp1.njobs = 1;
      mp1.total_edges = edges;
      RGG_CK(launch_merge_single(mp1, s));
    } else {
      mpp->njobs = nj;
      mpp->total_edges = edges;
      RGG_CK(launch_merge_batched(*mpp, s));
    }
    if (ev) RGG_CK(cudaEventRecord(ev[2], s));
  }
  for (uint32_t i = 0; i < n; ++i) {
    for (const auto& en : rs[i]->pending)
      if (en.snap >= 0) rs[i]->req_state[en.snap] = 2;
    clear_pending(rs[i]);
  }
  return RGG_OK;
}

// OBB geometry: each roadmap's passes in turn.  Per pass: the moved boxes'
// records, the (box, cell) work list and the box / spline tests (Sec. 4.3
// queries with the spatial filter), then the same merge as the sphere path.
static int classify_group_obb(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s) {
  std::unique_ptr<BoxPrepParams> bpp(new (std::nothrow) BoxPrepParams);
  if (!bpp) return RGG_ERR_OOM;
  for (uint32_t i = 0; i < n; ++i) {
    rgg_roadmap* r = rs[i];
    auto& pend = r->pending;
    bool ordered = false;
    for (const auto& en : pend)
      if (en.snap >= 0) ordered = true;
    if (!ordered)
      std::sort(pend.begin(), pend.end(), [](const rgg_roadmap::Entry& a,
                                             const rgg_roadmap::Entry& b) { return a.id < b.id; });
    for (size_t lo = 0; lo < pend.size(); lo += kBoxesPerPass) {
      const uint32_t C = (uint32_t)std::min<size_t>(kBoxesPerPass, pend.size() - lo);
      BoxPrepParams& bp = *bpp;
      bp.njobs = 1;
      BoxPrepJob& pj = bp.job[0];
      pj.stage = r->d_stage;
      pj.out = r->d_changed;
      pj.C = C;
      for (uint32_t b = 0; b < C; ++b) {
        pj.ids[b] = pend[lo + b].id;
        pj.rows[b] = (uint16_t)pend[lo + b].row;
      }
      RGG_CK(launch_box_prep(bp, s));
      const EdgeState& es = r->es;
      if (es.N == 0) continue;
      ObbQueryParams q{};
      q.L = r->L;
      q.K = r->K;
      q.C = C;
      q.margin = r->margin;
      q.g = es.grid;
      q.obb = es.d_obb;
      q.spl_off = es.d_spl_off;
      q.spl_v = es.d_spl_v;
      q.cell_off = es.d_cell_off;
      q.cell_items = es.d_cell_items;
      q.boxes = r->d_changed;
      q.edge_acc = es.d_edge_acc;
      q.pairs = es.d_pairs;
      q.counters = es.d_qcnt;
      q.pair_cap = es.pair_cap;
      q.filter = r->obb_filter ? 1u : 0u;
      q.work = r->d_obbwork;
      RGG_CK(cudaMemsetAsync(es.d_qcnt, 0, 2 * sizeof(uint32_t), s));
      cudaEvent_t* ev = r->timing ? next_events(r) : nullptr;
      if (ev) RGG_CK(cudaEventRecord(ev[0], s));
      RGG_CK(launch_obb_query(q, r->num_sms, s));
      if (ev) RGG_CK(cudaEventRecord(ev[1], s));
      MergeParams<1> mp;
      mp.job[0] = make_merge_job(r, lo, C, ordered, 0);
      mp.njobs = 1;
      mp.total_edges = es.N;
      RGG_CK(launch_merge_single(mp, s));
      if (ev) RGG_CK(cudaEventRecord(ev[2], s));
    }
    for (const auto& en : pend)
      if (en.snap >= 0) r->req_state[en.snap] = 2;
    clear_pending(r);
  }
  return RGG_OK;
}

int rgg_classify(rgg_roadmap_t r, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges) return RGG_ERR_STATE;
  if (r->pending.empty()) return RGG_OK;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  if (r->geometry == RGG_GEOMETRY_OBB) return classify_group_obb(&r, 1, static_cast<cudaStream_t>(stream));
  return classify_group(&r, 1, static_cast<cudaStream_t>(stream));
}

int rgg_classify_many(rgg_roadmap_t* rs, uint32_t n, void* stream) {
  if (!rs && n) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < n; ++i) {
    if (!rs[i]) return RGG_ERR_INVALID;
    if (!rs[i]->has_edges) return RGG_ERR_STATE;
    if (rs[i]->device != rs[0]->device || rs[i]->variant != rs[0]->variant ||
        rs[i]->geometry != rs[0]->geometry)
      return RGG_ERR_INVALID;
    for (uint32_t j = 0; j < i; ++j)
      if (rs[j] == rs[i]) return RGG_ERR_INVALID;
  }
  if (n == 0) return RGG_OK;
  DeviceGuard g(rs[0]->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rs[0]->geometry == RGG_GEOMETRY_OBB) return classify_group_obb(rs, n, s);
  for (uint32_t base = 0; base < n; base += kMaxJobs) {
    int rc = classify_group(rs + base, std::min<uint32_t>(kMaxJobs, n - base), s);
    if (rc != RGG_OK) return rc;
  }
  return RGG_OK;
}

static int check_status_locked(rgg_roadmap_t r, cudaStream_t s) {
  int st = 0;
  RGG_CK(cudaMemcpyAsync(&st, r->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  RGG_CK(cudaStreamSynchronize(s));
  if (st != 0) {
    RGG_CK(cudaMemsetAsync(r->d_status, 0, sizeof(int), s));
    RGG_CK(cudaStreamSynchronize(s));
    return RGG_ERR_TIMEOUT;
  }
  return RGG_OK;
}

int rgg_fetch_labels(rgg_roadmap_t r, uint8_t* out, uint64_t first, uint64_t count,
                     int dst_is_device, void* stream) {
  if (!r || (!out && count) || dst_is_device < 0 || dst_is_device > 2) return RGG_ERR_INVALID;
  if (!r->has_edges && count) return RGG_ERR_STATE;
  if (first > r->es.N || count > r->es.N - first) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (count)
    RGG_CK(cudaMemcpyAsync(out, r->es.d_labels + first, count,
                           dst_is_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (dst_is_device == 0) return check_status_locked(r, s);
  return RGG_OK;
}

int rgg_fetch_request_labels(rgg_roadmap_t r, uint32_t handle, uint8_t* out, uint64_t first,
                             uint64_t count, int dst_is_device, void* stream) {
  if (!r || handle >= RGG_MAX_REQUESTS || (!out && count) || dst_is_device < 0 ||
      dst_is_device > 2)
    return RGG_ERR_INVALID;
  if (!r->has_edges || r->req_state[handle] != 2) return RGG_ERR_STATE;
  if (first > r->es.N || count > r->es.N - first) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (count)
    RGG_CK(cudaMemcpyAsync(out, r->es.d_hist + (size_t)handle * r->es.N + first, count,
                           dst_is_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (dst_is_device == 0) return check_status_locked(r, s);
  return RGG_OK;
}

int rgg_release_request(rgg_roadmap_t r, uint32_t handle) {
  if (!r || handle >= RGG_MAX_REQUESTS) return RGG_ERR_INVALID;
  if (r->req_state[handle] != 2) return RGG_ERR_STATE;
  r->req_state[handle] = 0;
  return RGG_OK;
}

int rgg_fetch_box_sets(rgg_roadmap_t r, uint32_t* hit, uint32_t* touch, uint64_t first,
                       uint64_t count, int dst_is_device, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges && count) return RGG_ERR_STATE;
  if (first > r->es.N || count > r->es.N - first) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t bytes = count * r->Wm * sizeof(uint32_t);
  if (hit && count) RGG_CK(cudaMemcpyAsync(hit, r->es.d_red + first * r->Wm, bytes, kind, s));
  if (touch && count) RGG_CK(cudaMemcpyAsync(touch, r->es.d_touch + first * r->Wm, bytes, kind, s));
  if (!dst_is_device) return check_status_locked(r, s);
  return RGG_OK;
}

int rgg_fetch_records(rgg_roadmap_t r, uint64_t first, uint64_t count, float* inner_xyzr,
                      float* outer_xyzr, uint64_t* sample_off) {
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges || r->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;
  const EdgeState& es = r->es;
  if (first > es.N || count > es.N - first) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  RGG_CK(cudaDeviceSynchronize());
  if (sample_off) std::memcpy(sample_off, es.h_soff.data(), (es.N + 1) * sizeof(uint64_t));
  if (count == 0) return RGG_OK;
  const uint64_t s0 = es.h_soff[first], s1 = es.h_soff[first + count];
  const uint64_t i0 = (uint64_t)r->K * r->L * s0, ni = (uint64_t)r->K * r->L * (s1 - s0);
  const uint64_t o0 = (uint64_t)r->L * (s0 - first), no = (uint64_t)r->L * (s1 - s0 - count);
  for (int p = 0; p < 4; ++p) {
    if (inner_xyzr)
      RGG_CK(cudaMemcpy(inner_xyzr + p * ni, es.d_inner + p * es.in_stride + i0, ni * 4,
                        cudaMemcpyDeviceToHost));
    if (outer_xyzr && no)
      RGG_CK(cudaMemcpy(outer_xyzr + p * no, es.d_outer + p * es.out_stride + o0, no * 4,
                        cudaMemcpyDeviceToHost));
  }
  return RGG_OK;
}

int rgg_fetch_boxes(rgg_roadmap_t r, float* pose, uint8_t* present, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pose) {
    std::vector<float> rows((size_t)r->M * 16);
    RGG_CK(cudaMemcpyAsync(rows.data(), r->d_table, rows.size() * sizeof(float),
                           cudaMemcpyDeviceToHost, s));
    RGG_CK(cudaStreamSynchronize(s));
    for (uint32_t b = 0; b < r->M; ++b)
      std::memcpy(pose + 15 * (size_t)b, rows.data() + 16 * (size_t)b, 15 * sizeof(float));
  }
  if (present) std::memcpy(present, r->present.data(), r->M);
  return RGG_OK;
}

int rgg_labels_device_ptr(rgg_roadmap_t r, const uint8_t** out) {
  if (!r || !out) return RGG_ERR_INVALID;
  if (!r->has_edges) return RGG_ERR_STATE;
  *out = r->es.d_labels;
  return RGG_OK;
}

int rgg_roadmap_info(rgg_roadmap_t r, rgg_info* out) {
  if (!r || !out) return RGG_ERR_INVALID;
  const EdgeState& es = r->es;
  out->num_edges = es.N;
  out->num_samples = es.S_tot;
  out->num_inner = es.n_inner;
  out->num_outer = es.n_outer;
  out->record_bytes = 16 * (es.n_inner + es.n_outer);
  out->device_bytes = es.device_bytes + (uint64_t)r->M * 64 + (uint64_t)r->stage_rows * 64 +
                      kBoxesPerPass * kBoxRecFloats * 4 + 16;
  out->num_links = r->L;
  out->inner_per_link = r->K;
  out->max_obstacles = r->M;
  out->mask_words = r->Wm;
  out->tile_samples = es.tiling.S;
  out->num_tiles = es.T;
  out->pending_boxes = (uint32_t)r->pending.size();
  out->open_requests = (uint32_t)std::count_if(r->req_state.begin(), r->req_state.end(),
                                                [](uint8_t x) { return x != 0; });
  out->pending_capacity = r->stage_rows;
  out->geometry = r->geometry;
  out->grid_cells = es.n_cells;
  out->grid_items = es.n_items;
  out->spline_vertices = es.n_spl_v;
  if (r->geometry == RGG_GEOMETRY_OBB) {
    // boxes, spline vertices and spline offsets
    out->num_inner = es.n_spl_v;
    out->num_outer = es.n_obb;
    out->record_bytes = 64 * es.n_obb + 16 * es.n_spl_v + 8 * (es.n_spl + 1);
  }
  out->grid_ctas = (uint32_t)std::min<uint64_t>(es.T, launch_ctas(r));
  return RGG_OK;
}

int rgg_check_status(rgg_roadmap_t r, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  return check_status_locked(r, static_cast<cudaStream_t>(stream));
}

int rgg_set_kernel_timing(rgg_roadmap_t r, int enable) {
  if (!r) return RGG_ERR_INVALID;
  r->timing = enable != 0;
  r->events_used = 0;
  return RGG_OK;
}

int rgg_kernel_time(rgg_roadmap_t r, double* classify_ms, double* merge_ms,
                    uint64_t* launches) {
  if (!r || !classify_ms || !merge_ms || !launches) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  double tc = 0.0, tm = 0.0;
  for (size_t i = 0; i < r->events_used; ++i) {
    RGG_CK(cudaEventSynchronize(r->events[i][2]));
    float a = 0.f, b = 0.f;
    RGG_CK(cudaEventElapsedTime(&a, r->events[i][0], r->events[i][1]));
    RGG_CK(cudaEventElapsedTime(&b, r->events[i][1], r->events[i][2]));
    tc += a;
    tm += b;
  }
  *classify_ms = tc;
  *merge_ms = tm;
  *launches = r->events_used;
  r->events_used = 0;
  return RGG_OK;
}

int rgg_set_obb_filter(rgg_roadmap_t r, int enable) {
  if (!r) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_OBB) return RGG_ERR_STATE;
  r->obb_filter = enable != 0;
  return RGG_OK;
}

int rgg_fetch_obb_records(rgg_roadmap_t r, float* obb, uint64_t* spl_off, float* spl_v) {
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges || r->geometry != RGG_GEOMETRY_OBB) return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  const EdgeState& es = r->es;
  RGG_CK(cudaDeviceSynchronize());
  if (obb && es.n_obb)
    RGG_CK(cudaMemcpy(obb, es.d_obb, es.n_obb * 4 * sizeof(float4), cudaMemcpyDeviceToHost));
  if (spl_off) RGG_CK(cudaMemcpy(spl_off, es.d_spl_off, (es.n_spl + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (spl_v && es.n_spl_v)
    RGG_CK(cudaMemcpy(spl_v, es.d_spl_v, es.n_spl_v * sizeof(float4), cudaMemcpyDeviceToHost));
  return RGG_OK;
}

int rgg_obb_work(rgg_roadmap_t r, uint64_t* sat_tests, uint64_t* segment_tests) {
  if (!r || !sat_tests || !segment_tests) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_OBB) return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  unsigned long long w[2] = {0, 0};
  RGG_CK(cudaDeviceSynchronize());
  RGG_CK(cudaMemcpy(w, r->d_obbwork, sizeof(w), cudaMemcpyDeviceToHost));
  RGG_CK(cudaMemset(r->d_obbwork, 0, sizeof(w)));
  *sat_tests = w[0];
  *segment_tests = w[1];
  return RGG_OK;
}

int rgg_set_launch_shape(rgg_roadmap_t r, uint32_t variant, uint32_t consumer_warps) {
  if (!r) return RGG_ERR_INVALID;
  const uint32_t cw = consumer_warps ? consumer_warps : kDefaultConsumerWarps;
  if (!shape_ok(variant, cw)) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  return apply_shape(r, (int)variant, cw);
}

// ---------------------------------------------------------------------------
// Non-lazy resolution of gray edges
// ---------------------------------------------------------------------------
int rgg_resolve_gray(rgg_roadmap_t r, uint32_t factor, uint8_t* labels_out, float* clearance_out,
                     int dst_is_device, rgg_resolve_stats* stats, void* stream) {
  if (!r || factor < 1 || factor > RGG_MAX_RESOLVE_FACTOR || dst_is_device < 0 ||
      dst_is_device > 1)
    return RGG_ERR_INVALID;
  if (!r->has_edges || !r->has_robot || !r->pending.empty()) return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EdgeState& es = r->es;
  const uint64_t N = es.N;
  if (N && !es.d_resolved) {
    cudaError_t e = dalloc(&es.d_resolved, N);
    if (e == cudaSuccess) e = dalloc(&es.d_clear, N);
    if (e != cudaSuccess) {
      cudaFree(es.d_resolved);
      es.d_resolved = nullptr;
      return cuda_status(e);
    }
    es.device_bytes += 5 * N;
  }
  RGG_CK(cudaMemsetAsync(r->d_work, 0, 4 * sizeof(unsigned long long), s));
  ResolveParams p{};
  p.L = r->L;
  p.Wm = r->Wm;
  p.F = factor;
  // FP32 kinematics and distances stay within ~5e-6 m; the margin covers that
  p.thr = std::max(r->margin, kRegularMinMargin);
  for (uint32_t i = 0; i < r->L; ++i) {
    p.a[i] = (float)r->dh_a[i];
    p.d[i] = (float)r->dh_d[i];
    p.ca[i] = (float)std::cos(r->dh_alpha[i]);
    p.sa[i] = (float)std::sin(r->dh_alpha[i]);
    p.radius[i] = (float)r->dh_radius[i];
  }
  p.qa = es.d_qa;
  p.qb = es.d_qb;
  p.soff = es.d_soff;
  p.labels = es.d_labels;
  p.touch = es.d_touch;
  p.table = r->d_table;
  p.out = es.d_resolved;
  p.clearance = es.d_clear;
  p.work = r->d_work;
  p.n_edges = N;
  RGG_CK(launch_resolve_gray(p, r->num_sms, s));
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (labels_out && N) RGG_CK(cudaMemcpyAsync(labels_out, es.d_resolved, N, kind, s));
  if (clearance_out && N)
    RGG_CK(cudaMemcpyAsync(clearance_out, es.d_clear, N * sizeof(float), kind, s));
  if (stats) {
    unsigned long long w[4] = {0, 0, 0, 0};
    RGG_CK(cudaMemcpyAsync(w, r->d_work, sizeof(w), cudaMemcpyDeviceToHost, s));
    RGG_CK(cudaStreamSynchronize(s));
    stats->gray_edges = w[0];
    stats->resolved_red = w[1];
    stats->resolved_green = w[2];
    stats->evaluations = w[3];
  }
  if (!dst_is_device && (labels_out || clearance_out)) return check_status_locked(r, s);
  return RGG_OK;
}

// ---------------------------------------------------------------------------
// Persistence: rgg_save / rgg_load
// ---------------------------------------------------------------------------
struct SaveHeader {
  char magic[8];
  uint32_t version, L, K, M, Wm;
  float margin;
  uint32_t flags;  // bit 0: regular inner records
  uint32_t pad;
  uint64_t N, S, n_inner, n_outer;
  uint64_t reserved[3];
};
static_assert(sizeof(SaveHeader) == 96, "save header size");

static const char kSaveMagic[8] = {'R', 'G', 'G', 'S', 'A', 'V', 'E', '1'};
static const size_t kStagingBytes = 64ull << 20;

// 64-bit checksum of a byte stream, eight bytes at a time (xor, multiply by
// an odd constant, fold the high bits down); the stream is fed in pieces.
struct StreamHash {
  uint64_t h = 0x6a09e667f3bcc909ull;
  uint64_t word = 0;
  unsigned fill = 0;
  void mix(uint64_t w) {
    h = (h ^ w) * 0x9e3779b97f4a7c15ull;
    h ^= h >> 29;
  }
  void update(const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    while (n && fill) {
      word |= (uint64_t)*p++ << (8 * fill);
      --n;
      if (++fill == 8) {
        mix(word);
        word = 0;
        fill = 0;
      }
    }
    for (; n >= 8; n -= 8, p += 8) {
      uint64_t w;
      std::memcpy(&w, p, 8);
      mix(w);
    }
    for (; n; --n) word |= (uint64_t)*p++ << (8 * fill++);
  }
  uint64_t digest() const {
    StreamHash t = *this;
    t.mix(t.word ^ ((uint64_t)t.fill << 56));
    return t.h;
  }
};

struct FileIO {
  FILE* f = nullptr;
  StreamHash hash;
  unsigned char* staging = nullptr;
  bool io_ok = true;
  ~FileIO() {
    if (f) fclose(f);
    if (staging) cudaFreeHost(staging);
  }
  bool put(const void* p, size_t n) {
    if (!io_ok) return false;
    hash.update(p, n);
    io_ok = n == 0 || fwrite(p, 1, n, f) == n;
    return io_ok;
  }
  bool get(void* p, size_t n) {
    if (!io_ok) return false;
    io_ok = n == 0 || fread(p, 1, n, f) == n;
    if (io_ok) hash.update(p, n);
    return io_ok;
  }
};

// Device bytes to the file through the page-locked staging buffer.
static int save_device(FileIO& io, const void* src, size_t bytes, cudaStream_t s) {
  const unsigned char* p = static_cast<const unsigned char*>(src);
  for (size_t off = 0; off < bytes; off += kStagingBytes) {
    const size_t n = std::min(kStagingBytes, bytes - off);
    RGG_CK(cudaMemcpyAsync(io.staging, p + off, n, cudaMemcpyDeviceToHost, s));
    RGG_CK(cudaStreamSynchronize(s));
    if (!io.put(io.staging, n)) return RGG_ERR_IO;
  }
  return RGG_OK;
}

// File bytes to device memory through the staging buffer.  A short read is
// a truncated file.
static int load_device(FileIO& io, void* dst, size_t bytes, cudaStream_t s) {
  unsigned char* p = static_cast<unsigned char*>(dst);
  for (size_t off = 0; off < bytes; off += kStagingBytes) {
    const size_t n = std::min(kStagingBytes, bytes - off);
    if (!io.get(io.staging, n)) return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
    RGG_CK(cudaMemcpyAsync(p + off, io.staging, n, cudaMemcpyHostToDevice, s));
    RGG_CK(cudaStreamSynchronize(s));
  }
  return RGG_OK;
}

int rgg_save(rgg_roadmap_t r, const char* path, void* stream) {
  if (!r || !path) return RGG_ERR_INVALID;
  if (!r->has_edges || !r->pending.empty() || r->geometry != RGG_GEOMETRY_SPHERES)
    return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RGG_CK(cudaStreamSynchronize(s));
  const EdgeState& es = r->es;
  FileIO io;
  RGG_CK(cudaMallocHost(reinterpret_cast<void**>(&io.staging), kStagingBytes));
  io.f = std::fopen(path, "wb");
  if (!io.f) return RGG_ERR_IO;
  SaveHeader h{};
  std::memcpy(h.magic, kSaveMagic, 8);
  h.version = 1;
  h.L = r->L;
  h.K = r->K;
  h.M = r->M;
  h.Wm = r->Wm;
  h.margin = r->margin;
  h.flags = es.regular ? 1u : 0u;
  h.N = es.N;
  h.S = es.S_tot;
  h.n_inner = es.n_inner;
  h.n_outer = es.n_outer;
  if (!io.put(&h, sizeof(h)) || !io.put(es.h_soff.data(), (es.N + 1) * sizeof(uint64_t)))
    return RGG_ERR_IO;
  int rc = RGG_OK;
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = save_device(io, es.d_inner + p * es.in_stride, es.n_inner * 4, s);
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = save_device(io, es.d_outer + p * es.out_stride, es.n_outer * 4, s);
  const size_t set_bytes = es.N * r->Wm * sizeof(uint32_t);
  if (rc == RGG_OK) rc = save_device(io, es.d_red, set_bytes, s);
  if (rc == RGG_OK) rc = save_device(io, es.d_touch, set_bytes, s);
  if (rc == RGG_OK) rc = save_device(io, es.d_counts, es.N * sizeof(uint32_t), s);
  if (rc == RGG_OK) rc = save_device(io, es.d_labels, es.N, s);
  if (rc == RGG_OK) rc = save_device(io, r->d_table, (size_t)r->M * 16 * sizeof(float), s);
  if (rc == RGG_OK && !io.put(r->present.data(), r->M)) rc = RGG_ERR_IO;
  if (rc != RGG_OK) return rc;
  const uint64_t digest = io.hash.digest();
  if (std::fwrite(&digest, sizeof(digest), 1, io.f) != 1) return RGG_ERR_IO;
  const int closed = std::fclose(io.f);
  io.f = nullptr;
  return closed == 0 ? RGG_OK : RGG_ERR_IO;
}

int rgg_load(rgg_roadmap_t r, const char* path, void* stream) {
  if (!r || !path) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FileIO io;
  io.f = std::fopen(path, "rb");
  if (!io.f) return RGG_ERR_IO;
  SaveHeader h{};
  if (!io.get(&h, sizeof(h))) return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  if (std::memcmp(h.magic, kSaveMagic, 8) != 0 || h.version != 1 || h.L != r->L || h.K != r->K ||
      h.M != r->M || h.Wm != r->Wm || h.N >= 0xffffffffull || h.S < 2 * h.N ||
      h.n_inner != (uint64_t)h.K * h.L * h.S || h.n_outer != (uint64_t)h.L * (h.S - h.N))
    return RGG_ERR_INVALID;
  std::vector<uint64_t> soff(h.N + 1);
  if (!io.get(soff.data(), soff.size() * sizeof(uint64_t)))
    return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  if (!valid_soff(soff.data(), h.N, r->L) || soff[h.N] != h.S) return RGG_ERR_INVALID;
  RGG_CK(cudaMallocHost(reinterpret_cast<void**>(&io.staging), kStagingBytes));
  EdgeState es;
  int rc = alloc_edges(r, &es, h.N, std::move(soff), s);
  if (rc != RGG_OK) return rc;
  float* d_table = nullptr;
  cudaError_t e = dalloc(&d_table, (size_t)r->M * 16);
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  std::vector<uint8_t> present(r->M);
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = load_device(io, es.d_inner + p * es.in_stride, es.n_inner * 4, s);
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = load_device(io, es.d_outer + p * es.out_stride, es.n_outer * 4, s);
  const size_t set_bytes = es.N * r->Wm * sizeof(uint32_t);
  if (rc == RGG_OK) rc = load_device(io, es.d_red, set_bytes, s);
  if (rc == RGG_OK) rc = load_device(io, es.d_touch, set_bytes, s);
  if (rc == RGG_OK) rc = load_device(io, es.d_counts, es.N * sizeof(uint32_t), s);
  if (rc == RGG_OK) rc = load_device(io, es.d_labels, es.N, s);
  if (rc == RGG_OK) rc = load_device(io, d_table, (size_t)r->M * 16 * sizeof(float), s);
  if (rc == RGG_OK && !io.get(present.data(), r->M))
    rc = ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  uint64_t stored = 0;
  if (rc == RGG_OK && std::fread(&stored, sizeof(stored), 1, io.f) != 1) rc = RGG_ERR_INVALID;
  if (rc == RGG_OK && stored != io.hash.digest()) rc = RGG_ERR_INVALID;
  if (rc != RGG_OK) {
    es.release();
    cudaFree(d_table);
    return rc;
  }
  // the file checks out: swap in the edges, the state and the boxes
  es.regular = (h.flags & 1u) != 0;
  e = cudaMemcpyAsync(r->d_table, d_table, (size_t)r->M * 16 * sizeof(float),
                      cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_table);
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  for (uint32_t b = 0; b < r->M; ++b) r->present[b] = present[b] ? 1 : 0;
  r->es.release();
  r->es = std::move(es);
  r->has_edges = true;
  r->has_robot = false;
  ++r->gen;
  clear_pending(r);
  std::fill(r->req_state.begin(), r->req_state.end(), 0);
  return RGG_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time the classify launch of these roadmaps at every supported
// launch shape, on their own records and boxes, and keep the fastest.
// ---------------------------------------------------------------------------
// One classify launch over the roadmaps' tiles with C[i] boxes each, OR-ing
// into the scratch accumulators acc[i] (labels and box sets are untouched).
static int tune_launch(rgg_roadmap_t* rs, uint32_t n, const std::vector<uint32_t*>& acc,
                const std::vector<uint32_t>& C, ClassifyParams<kMaxJobs>* cpp,
                cudaStream_t s) {
  ClassifyParams<1> cp1;
  uint32_t nj = 0;
  uint64_t tiles = 0;
  for (uint32_t i = 0; i < n; ++i) {
    rgg_roadmap* r = rs[i];
    if (r->es.N == 0 || C[i] == 0) continue;
    ClassifyJob j = make_job(r, C[i], tiles);
    j.edge_acc = acc[i];
    if (n == 1) cp1.job[0] = j; else cpp->job[nj] = j;
    ++nj;
    tiles += r->es.T;
  }
  if (nj == 0) return RGG_OK;
  rgg_roadmap* r0 = rs[0];
  ClassifyLaunch lc;
  lc.consumer_warps = r0->consumer_warps;
  lc.variant = r0->variant;
  lc.grid = std::max<uint32_t>(1, (uint32_t)std::min<uint64_t>((tiles + 1) / 2, launch_ctas(r0)));
  uint32_t* counter = reinterpret_cast<uint32_t*>(r0->d_status + 1);
  RGG_CK(cudaMemsetAsync(counter, 0, sizeof(uint32_t), s));
  if (n == 1) {
    cp1.njobs = 1;
    cp1.total_tiles = tiles;
    cp1.status = r0->d_status;
    cp1.work_counter = counter;
    RGG_CK(launch_classify_single(cp1, lc, s));
  } else {
    cpp->njobs = nj;
    cpp->total_tiles = tiles;
    cpp->status = r0->d_status;
    cpp->work_counter = counter;
    RGG_CK(launch_classify_batched(*cpp, lc, s));
  }
  return RGG_OK;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

int rgg_autotune(rgg_roadmap_t* rs, uint32_t n, uint32_t reps, rgg_tune_result* results,
                 uint32_t max_results, uint32_t* n_results, void* stream) {
  if (!rs || n == 0 || n > (uint32_t)kMaxJobs || (max_results && !results)) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < n; ++i) {
    if (!rs[i]) return RGG_ERR_INVALID;
    if (!rs[i]->has_edges || rs[i]->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;
    if (rs[i]->device != rs[0]->device) return RGG_ERR_INVALID;
    for (uint32_t j = 0; j < i; ++j)
      if (rs[j] == rs[i]) return RGG_ERR_INVALID;
  }
  if (n_results) *n_results = 0;
  reps = std::max<uint32_t>(1, std::min<uint32_t>(reps, 100));
  DeviceGuard g(rs[0]->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the first 32 present boxes of each roadmap, prepared from the box table
  // (table row = box id); a pending pass re-prepares its own boxes later
  std::vector<uint32_t> C(n, 0);
  std::unique_ptr<BoxPrepParams> bpp(new (std::nothrow) BoxPrepParams);
  std::unique_ptr<ClassifyParams<kMaxJobs>> cpp(new (std::nothrow) ClassifyParams<kMaxJobs>);
  if (!bpp || !cpp) return RGG_ERR_OOM;
  bpp->njobs = 0;
  bool any = false;
  for (uint32_t i = 0; i < n; ++i) {
    rgg_roadmap* r = rs[i];
    BoxPrepJob& pj = bpp->job[bpp->njobs++];
    pj.stage = r->d_table;
    pj.out = r->d_changed;
    pj.C = 0;
    for (uint32_t b = 0; b < r->M && pj.C < (uint32_t)kBoxesPerPass; ++b)
      if (r->present[b]) {
        pj.ids[pj.C] = b;
        pj.rows[pj.C] = (uint16_t)b;
        ++pj.C;
      }
    C[i] = pj.C;
    any = any || (pj.C > 0 && r->es.N > 0);
  }
  if (!any) return RGG_OK;  // nothing to time: the shape stays
  RGG_CK(launch_box_prep(*bpp, s));
  std::vector<uint32_t*> acc(n, nullptr);
  auto free_acc = [&]() {
    for (uint32_t* p : acc) cudaFree(p);
  };
  for (uint32_t i = 0; i < n; ++i) {
    cudaError_t e = dalloc(&acc[i], 2 * rs[i]->es.N);
    if (e != cudaSuccess) {
      free_acc();
      return cuda_status(e);
    }
  }
  EventPair ev;
  if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
    free_acc();
    return RGG_ERR_CUDA;
  }
  static const uint32_t kWarps[] = {16, 20, 24, 27};
  std::vector<rgg_tune_result> res;
  int rc = RGG_OK;
  for (int v = 0; v < kNumVariants && rc == RGG_OK; ++v)
    for (uint32_t cw : kWarps) {
      if (!shape_ok((uint32_t)v, cw)) continue;
      for (uint32_t i = 0; i < n && rc == RGG_OK; ++i) rc = apply_shape(rs[i], v, cw);
      if (rc != RGG_OK) break;
      rc = tune_launch(rs, n, acc, C, cpp.get(), s);  // warm-up
      if (rc == RGG_OK && cudaEventRecord(ev.a, s) != cudaSuccess) rc = RGG_ERR_CUDA;
      for (uint32_t k = 0; k < reps && rc == RGG_OK; ++k) rc = tune_launch(rs, n, acc, C, cpp.get(), s);
      if (rc == RGG_OK && cudaEventRecord(ev.b, s) != cudaSuccess) rc = RGG_ERR_CUDA;
      float ms = 0.f;
      if (rc == RGG_OK && (cudaEventSynchronize(ev.b) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess))
        rc = RGG_ERR_CUDA;
      if (rc != RGG_OK) break;
      rgg_tune_result t{};
      t.variant = (uint32_t)v;
      t.consumer_warps = cw;
      t.classify_ms = ms / (float)reps;
      res.push_back(t);
    }
  cudaStreamSynchronize(s);
  free_acc();
  if (rc == RGG_OK) rc = check_status_locked(rs[0], s);
  std::stable_sort(res.begin(), res.end(), [](const rgg_tune_result& a, const rgg_tune_result& b) {
    return a.classify_ms < b.classify_ms;
  });
  // keep the fastest shape (the previous one if the sweep failed part-way)
  if (!res.empty()) {
    for (uint32_t i = 0; i < n; ++i) {
      const int rc2 = apply_shape(rs[i], (int)res[0].variant, res[0].consumer_warps);
      if (rc == RGG_OK) rc = rc2;
    }
  }
  if (n_results) *n_results = (uint32_t)res.size();
  for (uint32_t i = 0; i < std::min<uint32_t>(max_results, (uint32_t)res.size()); ++i)
    results[i] = res[i];
  return rc;
}

// ---------------------------------------------------------------------------
// Step graphs: one update + classify of several roadmaps captured once and
// replayed with cudaGraphLaunch.
// ---------------------------------------------------------------------------
struct rgg_step_graph {
  int device = 0;
  std::vector<rgg_roadmap*> rs;
  std::vector<uint64_t> gens;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
};

int rgg_step_graph_create(rgg_roadmap_t* rs, uint32_t n, const uint32_t* n_ids,
                          const uint32_t* const* ids, const float* const* poses,
                          rgg_step_graph_t* out) {
  if (!out) return RGG_ERR_INVALID;
  *out = nullptr;
  if (!rs || n == 0 || !n_ids || !ids || !poses) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < n; ++i) {
    if (!rs[i]) return RGG_ERR_INVALID;
    if (!rs[i]->has_edges || !rs[i]->pending.empty() || rs[i]->geometry != RGG_GEOMETRY_SPHERES)
      return RGG_ERR_STATE;
    if (rs[i]->device != rs[0]->device || rs[i]->variant != rs[0]->variant) return RGG_ERR_INVALID;
    for (uint32_t j = 0; j < i; ++j)
      if (rs[j] == rs[i]) return RGG_ERR_INVALID;
    if (n_ids[i] && (!ids[i] || !poses[i])) return RGG_ERR_INVALID;
    uint32_t fresh = 0;
    if (n_ids[i]) {
      const int rc = check_moves(rs[i], n_ids[i], ids[i], poses[i], 1, &fresh);
      if (rc != RGG_OK) return rc;
    }
  }
  DeviceGuard g(rs[0]->device);
  if (!g.ok) return RGG_ERR_CUDA;
  std::unique_ptr<rgg_step_graph> G(new (std::nothrow) rgg_step_graph);
  if (!G) return RGG_ERR_OOM;
  G->device = rs[0]->device;
  std::vector<std::vector<uint8_t>> present(n);
  std::vector<uint8_t> timing(n);
  for (uint32_t i = 0; i < n; ++i) {
    present[i] = rs[i]->present;
    timing[i] = rs[i]->timing;
    rs[i]->timing = false;  // no event records inside the graph
  }
  cudaStream_t cs = nullptr;
  RGG_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int rc = RGG_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) rc = cuda_status(e);
  for (uint32_t i = 0; i < n && rc == RGG_OK; ++i)
    if (n_ids[i]) rc = stage_moves(rs[i], n_ids[i], ids[i], poses[i], 1, cs);
  for (uint32_t base = 0; base < n && rc == RGG_OK; base += kMaxJobs)
    rc = classify_group(rs + base, std::min<uint32_t>(kMaxJobs, n - base), cs);
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) {
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (rc == RGG_OK && e2 != cudaSuccess) rc = cuda_status(e2);
  }
  if (rc == RGG_OK) {
    e = cudaGraphInstantiate(&G->exec, graph, 0);
    if (e != cudaSuccess) rc = cuda_status(e);
    else cudaGraphGetNodes(graph, nullptr, &G->nodes);
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  for (uint32_t i = 0; i < n; ++i) {
    rs[i]->timing = timing[i] != 0;
    if (rc != RGG_OK) {
      // nothing ran: drop the entries the capture staged
      clear_pending(rs[i]);
      rs[i]->present = present[i];
    }
  }
  if (rc != RGG_OK) return rc;
  G->rs.assign(rs, rs + n);
  for (uint32_t i = 0; i < n; ++i) G->gens.push_back(rs[i]->gen);
  *out = G.release();
  return RGG_OK;
}

int rgg_step_graph_launch(rgg_step_graph_t g, void* stream) {
  if (!g) return RGG_ERR_INVALID;
  for (size_t i = 0; i < g->rs.size(); ++i)
    if (g->rs[i]->gen != g->gens[i] || !g->rs[i]->pending.empty()) return RGG_ERR_STATE;
  DeviceGuard dg(g->device);
  if (!dg.ok) return RGG_ERR_CUDA;
  RGG_CK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return RGG_OK;
}

int rgg_step_graph_nodes(rgg_step_graph_t g, uint64_t* nodes) {
  if (!g || !nodes) return RGG_ERR_INVALID;
  *nodes = g->nodes;
  return RGG_OK;
}

int rgg_step_graph_destroy(rgg_step_graph_t g) {
  if (!g) return RGG_OK;
  DeviceGuard dg(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return RGG_OK;
}

}  // extern "C"
