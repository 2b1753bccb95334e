// Host side of the C ABI declared in include/rgg.h: argument checks, device
// memory, tiling of the record stream, and kernel launches.  Every step of
// the classification runs in the kernels of rgg_kernels.cu.  The OBB
// geometry, persistence, the autotuner and step graphs, and the gray
// resolution have their own host files.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "rgg_host.h"

using namespace rgg;
using namespace rgg_host;

namespace rgg_host {

// Allocation-failure injection (a test hook, rgg_inject_alloc_failure): when
// the countdown reaches zero the allocation fails as if the device were out
// of memory.
static std::atomic<uint64_t> g_fail_countdown{0};

// Guard bytes: every allocation holds kGuardBytes of the byte kGuardByte
// after its requested size (rounded up to 16 B), and the live allocations are
// listed here with the offset of their guard and their device, so that
// rgg_check_guards can tell whether anything wrote past the end of a buffer.
constexpr size_t kGuardBytes = 64;
constexpr unsigned char kGuardByte = 0xA5;
struct Guarded {
  size_t offset;
  int device;
};
static std::mutex g_guard_mu;
static std::unordered_map<void*, Guarded> g_guards;

cudaError_t device_alloc(void** p, size_t bytes) {
  uint64_t c = g_fail_countdown.load();
  while (c != 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
      if (c == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  const size_t off = (bytes + 15) & ~(size_t)15;
  cudaError_t e = cudaMalloc(p, off + kGuardBytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaMemset(static_cast<unsigned char*>(*p) + off, kGuardByte, kGuardBytes);
  if (e != cudaSuccess) {
    cudaFree(*p);
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lk(g_guard_mu);
  g_guards[*p] = Guarded{off, dev};
  return cudaSuccess;
}

void device_free(void* p) {
  if (p == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(g_guard_mu);
    g_guards.erase(p);
  }
  cudaFree(p);
}

// Device bytes every roadmap holds whatever its edges: the box table, the
// staging rows, the pass's box records and the status words.
uint64_t fixed_device_bytes(const rgg_roadmap* r) {
  return (uint64_t)r->M * 64 + (uint64_t)r->stage_rows * 64 + kBoxAreaFloats * 4 + 16;
}

// Built sphere-geometry edges get link-end records unless the roadmap asked
// for sphere records or its margin is too small to cover the interpolated
// centres' error.
bool use_joints(const rgg_roadmap* r) {
  return r->geometry == RGG_GEOMETRY_SPHERES && r->record_format == 0 &&
         r->margin >= kRegularMinMargin;
}

// The default launch shape of the record format, unless the caller or the
// autotuner chose one.
void default_shape(rgg_roadmap* r, bool joints) {
  if (r->shape_set) return;
  r->variant = joints ? kDefaultVariantLinkEnds : kDefaultVariant;
  r->consumer_warps = joints ? kDefaultConsumerWarpsLinkEnds : kDefaultConsumerWarps;
}

ShapeRestore::ShapeRestore(rgg_roadmap* rm) : r(rm), variant(rm->variant), warps(rm->consumer_warps) {}
ShapeRestore::~ShapeRestore() {
  if (!keep) {
    r->variant = variant;
    r->consumer_warps = warps;
  }
}

// A roadmap's tiles can run in a launch of another variant when that
// variant's tiles are at least as long and its stages hold the tile's data.
bool tiles_fit(const rgg_roadmap* r, int variant) {
  const VariantShape v = variant_shape(variant);
  const Tiling& t = r->es.tiling;
  if (filter_active(r) && !filter_variant(variant)) return false;
  return t.S <= 31u * (uint32_t)v.rounds && (uint64_t)t.off_out + 16ull * t.out_cap <= (uint64_t)v.stage_bytes;
}

// The link radii R_i, rounded down to FP32, behind the pass's box records
// (link-end records take their inner radius from there).
int set_link_radii(rgg_roadmap* r, const double* radius, cudaStream_t s) {
  float lr[kLinkRadiiFloats] = {};
  for (uint32_t i = 0; i < r->L && i < (uint32_t)kLinkRadiiFloats; ++i) {
    float f = (float)radius[i];
    if ((double)f > radius[i]) f = std::nextafter(f, 0.0f);
    lr[i] = f;
  }
  RGG_CK(cudaMemcpyAsync(r->d_changed + kBoxesPerPass * kBoxRecFloats, lr, sizeof(lr),
                         cudaMemcpyHostToDevice, s));
  RGG_CK(cudaStreamSynchronize(s));  // lr lives on this stack frame
  return RGG_OK;
}

uint32_t launch_ctas(const rgg_roadmap* r) { return (uint32_t)r->num_sms * r->ctas_per_sm; }

// Tile descriptors and per-tile edge tables of a roadmap (see
// rgg_device.cuh): tile t covers global samples [t*S, min((t+1)*S, G)).
bool build_tiles(uint32_t L, uint64_t N, const std::vector<uint64_t>& soff, uint64_t G,
                 uint32_t S, std::vector<TileDesc>* tiles, std::vector<int4>* etab,
                 std::vector<uint32_t>* halo) {
  const uint64_t T = (G + S - 1) / S;
  tiles->resize(T);
  if (halo) halo->resize(T);
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
    // link-end records: the entries before the tile that belong to its first
    // edge, up to one link's run (they hold its first samples' near ends)
    if (halo) (*halo)[t] = (uint32_t)std::min<uint64_t>(n_f, rf);
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
  Tiling tiling = choose_tiling(r->L, r->K, es->G, 2 * launch_ctas(r), r->variant, es->joints,
                                es->max_n);
  if (tiling.S == 0) return RGG_ERR_INVALID;
  std::vector<TileDesc> h_tiles;
  std::vector<int4> h_etab;
  std::vector<uint32_t> h_halo;
  if (es->N && !build_tiles(r->L, es->N, es->h_soff, es->G, tiling.S, &h_tiles, &h_etab,
                            es->joints ? &h_halo : nullptr))
    return RGG_ERR_INVALID;
  TileDesc* d_tiles = nullptr;
  int4* d_etab = nullptr;
  uint32_t* d_halo = nullptr;
  cudaError_t e = dalloc(&d_tiles, h_tiles.size());
  if (e == cudaSuccess) e = dalloc(&d_etab, h_etab.size());
  if (e == cudaSuccess) e = dalloc(&d_halo, h_halo.size());
  if (e == cudaSuccess && !h_halo.empty())
    e = cudaMemcpyAsync(d_halo, h_halo.data(), h_halo.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !h_tiles.empty())
    e = cudaMemcpyAsync(d_tiles, h_tiles.data(), h_tiles.size() * sizeof(TileDesc),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !h_etab.empty())
    e = cudaMemcpyAsync(d_etab, h_etab.data(), h_etab.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s);
  // the host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    device_free(d_tiles);
    device_free(d_etab);
    device_free(d_halo);
    return cuda_status(e);
  }
  release_rounds(es);  // they describe the old tiles
  es->device_bytes -= es->T * sizeof(TileDesc) + es->n_etab * sizeof(int4) +
                      (es->d_tile_halo ? es->T * sizeof(uint32_t) : 0);
  device_free(es->d_tiles);
  device_free(es->d_etab);
  device_free(es->d_tile_halo);
  es->d_tiles = d_tiles;
  es->d_etab = d_etab;
  es->d_tile_halo = d_halo;
  es->T = h_tiles.size();
  es->n_etab = h_etab.size();
  es->tiling = tiling;
  es->device_bytes += es->T * sizeof(TileDesc) + es->n_etab * sizeof(int4) +
                      (d_halo ? es->T * sizeof(uint32_t) : 0);
  return RGG_OK;
}

// Bytes of the spatial filter's data for T tiles: per round slot a bounding
// sphere, an outer range and a candidate mask; per tile a sphere about its
// rounds and a list entry; the list's count.
uint64_t round_data_bytes(uint64_t T) {
  return T * kRoundSlots * (sizeof(float4) + 2 * sizeof(uint32_t)) + T * sizeof(float4) +
         (T + 1) * sizeof(uint32_t);
}

void release_rounds(EdgeState* es) {
  if (es->d_rsph) es->device_bytes -= round_data_bytes(es->T);
  device_free(es->d_rsph);
  device_free(es->d_rout);
  device_free(es->d_rcand);
  device_free(es->d_tlist);
  es->d_rsph = nullptr;
  es->d_rout = nullptr;
  es->d_rcand = nullptr;
  es->d_tlist = nullptr;
}

// The spatial filter runs with the default pipeline variant only (the one
// its kernel instance is compiled for).
bool filter_active(const rgg_roadmap* r) {
  return filter_wanted(r, &r->es) && r->es.d_rcand && filter_variant(r->variant);
}

// The spatial filter is on by default for link-end records, where the
// kernel is bound by its per-round work and the filter skips rounds and
// tiles no moved box can reach, and off for sphere records.
bool filter_wanted(const rgg_roadmap* r, const EdgeState* es) {
  return r->round_filter_mode == 1 || (r->round_filter_mode < 0 && es->joints);
}

// The spatial filter's per-round bounding spheres and outer ranges of the
// current tiles, from the resident outer records (stream-ordered after them);
// nothing while the filter is off.
int compute_rounds(rgg_roadmap* r, EdgeState* es, cudaStream_t s) {
  release_rounds(es);
  if (!filter_wanted(r, es) || r->geometry != RGG_GEOMETRY_SPHERES || es->T == 0) return RGG_OK;
  const uint64_t n = es->T * kRoundSlots;
  cudaError_t e = dalloc(&es->d_rsph, n + es->T);  // the round spheres, then the tile spheres
  if (e == cudaSuccess) e = dalloc(&es->d_rout, n);
  if (e == cudaSuccess) e = dalloc(&es->d_rcand, n);
  // the per-pass tile list and its count, zeroed so that no entry is ever
  // outside the tile table
  if (e == cudaSuccess) e = dalloc(&es->d_tlist, es->T + 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(es->d_tlist, 0, (es->T + 1) * sizeof(uint32_t), s);
  if (e != cudaSuccess) {
    device_free(es->d_rsph);
    device_free(es->d_rout);
    device_free(es->d_rcand);
    device_free(es->d_tlist);
    es->d_rsph = nullptr;
    es->d_rout = nullptr;
    es->d_rcand = nullptr;
    es->d_tlist = nullptr;
    return cuda_status(e);
  }
  es->device_bytes += round_data_bytes(es->T);
  RoundBoundsParams p;
  p.outer = es->d_outer;
  p.out_stride = es->out_stride;
  p.tiles = es->d_tiles;
  p.etab = es->d_etab;
  p.T = es->T;
  p.G = es->G;
  p.S = es->tiling.S;
  p.rsph = es->d_rsph;
  p.rout = es->d_rout;
  p.tsph = es->d_rsph + n;
  RGG_CK(launch_round_bounds(p, r->num_sms, s));
  return RGG_OK;
}

// Allocate the per-edge state and record planes for N edges with per-edge
// sample offsets h_soff (host), into `es` (not yet visible to the roadmap).
int alloc_edges(rgg_roadmap* r, EdgeState* es, uint64_t N, std::vector<uint64_t>&& soff,
                cudaStream_t s, bool joints) {
  const bool spheres = r->geometry == RGG_GEOMETRY_SPHERES;
  es->N = N;
  es->h_soff = std::move(soff);
  es->S_tot = es->h_soff[N];
  es->G = (uint64_t)r->L * es->S_tot;
  es->joints = spheres && joints;
  es->max_n = 0;
  for (uint64_t e = 0; e < N; ++e)
    es->max_n = std::max<uint64_t>(es->max_n, es->h_soff[e + 1] - es->h_soff[e]);
  // link-end records: one entry per (edge, link, configuration), 3 planes
  es->n_inner = spheres ? (es->joints ? es->G : (uint64_t)r->K * es->G) : 0;
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
    RGG_AL(es->d_inner, (es->joints ? 3 : 4) * es->in_stride);
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
    e = cudaMemsetAsync(es->d_inner, 0, (es->joints ? 3 : 4) * es->in_stride * sizeof(float), s);
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

// Drop the pending entries and make every present box pending again, its
// staged pose copied from the box table, so that the next classify tests
// every present box against every edge and replaces all of their bits.
int requeue_present(rgg_roadmap* r, cudaStream_t s) {
  clear_pending(r);
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

// Swap in freshly built edges: labels GREEN, box sets empty, open requests
// closed, and every present box pending so that the next classify tests it
// against the new edges.
int install_edges(rgg_roadmap* r, EdgeState&& es, cudaStream_t s) {
  const int rc = compute_rounds(r, &es, s);
  if (rc != RGG_OK) {
    es.release();
    return rc;
  }
  r->es.release();
  r->es = std::move(es);
  r->has_edges = true;
  ++r->gen;
  std::fill(r->req_state.begin(), r->req_state.end(), 0);
  return requeue_present(r, s);
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
  j.joints = es.joints ? 1u : 0u;
  j.tile_halo = es.d_tile_halo;
  j.inv_k = 1.0f / (float)r->K;
  j.inv_km1 = r->K > 1 ? 1.0f / (float)(r->K - 1) : 0.0f;
  if (filter_active(r)) {
    j.rsph = es.d_rsph;
    j.tsph = es.d_rsph + es.T * kRoundSlots;
    j.rout = es.d_rout;
    j.rcand = es.d_rcand;
    j.tlist = es.d_tlist;
    j.tcount = es.d_tlist + es.T;
  }
  j.streamed = r->d_streamed;
  j.status = r->d_status;
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
  m.status = r->d_status;
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
  // every warp of the launch must find an end marker among the first
  // `stages` slots past the last tile
  return (uint64_t)cw + 1 <=
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
    int rc = set_tiles(r, &r->es, nullptr);
    if (rc != RGG_OK) {  // the old tiles stay
      r->variant = old_v;
      r->consumer_warps = old_cw;
      return rc;
    }
    ++r->gen;  // captured step graphs hold the old tiles
    // the new tiles' round data; without them the roadmap runs unfiltered
    rc = compute_rounds(r, &r->es, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess && rc == RGG_OK) rc = RGG_ERR_CUDA;
    return rc;
  }
  return RGG_OK;
}


// Checks a move's ids and host poses; counts the entries it would append.
int check_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
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
int stage_moves(rgg_roadmap_t r, uint32_t n, const uint32_t* ids, const float* pose,
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

// One streaming pass per group of <= 32 pending entries; for several
// roadmaps, pass p of every roadmap that has one goes into the same
// persistent launch.  Without requests the entries (distinct boxes) are
// sorted so that each pass's ids ascend, for the merge kernel's word-grouped
// update; with requests they keep their order and merge one by one.
int classify_group(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s) {
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
      pj.tcount = filter_active(r) ? r->es.d_tlist + r->es.T : nullptr;
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
    // a roadmap on its default link-end shape whose last pass listed nearly
    // every tile runs variant 12 (the same tiles, 3 rounds per work item);
    // the count may be a pass old, which only affects speed
    const bool track = n == 1 && !r0->shape_set && r0->variant == kDefaultVariantLinkEnds &&
                       r0->d_listed && filter_active(r0) && r0->es.T >= kDensePassMinTiles;
    if (track &&
        (uint64_t)*reinterpret_cast<volatile uint32_t*>(r0->h_listed) * 1000 >=
            (uint64_t)kDensePassPermille * r0->es.T)
      lc.variant = kDenseVariantLinkEnds;
    for (uint32_t i = 0; i < n; ++i) rs[i]->last_variant = lc.variant;
    lc.grid = (uint32_t)std::min<uint64_t>((tiles + 1) / 2, launch_ctas(r0));
    lc.grid = std::max<uint32_t>(lc.grid, 1);
    cudaEvent_t* ev = timed ? next_events(timed) : nullptr;
    if (ev) RGG_CK(cudaEventRecord(ev[0], s));
    if (n == 1) {
      cp1.njobs = 1;
      cp1.total_tiles = tiles;
      cp1.status = r0->d_status;
      cp1.wait_ns = r0->wait_ns;
      cp1.work = r0->counting ? r0->d_count : nullptr;
      cp1.listed_out = track ? r0->d_listed : nullptr;
      RGG_CK(launch_classify_single(cp1, lc, s));
    } else {
      cpp->njobs = nj;
      cpp->total_tiles = tiles;
      cpp->status = r0->d_status;
      cpp->wait_ns = r0->wait_ns;
      RGG_CK(launch_classify_batched(*cpp, lc, s));
    }
    if (ev) RGG_CK(cudaEventRecord(ev[1], s));
    if (n == 1) {
      mp1.njobs = 1;
      mp1.total_edges = edges;
      mp1.status = r0->d_status;
      RGG_CK(launch_merge_single(mp1, s));
    } else {
      mpp->njobs = nj;
      mpp->total_edges = edges;
      mpp->status = r0->d_status;
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

// Reports a device error latched on the roadmap (a classify launch whose
// bounded wait ran out, or a pass skipped because of an earlier one) and
// recovers from it: the word is cleared, every present box is queued again
// (the box table holds the latest poses, so the next classify recomputes
// every bit the failed passes left out), and open request handles are
// marked lost (their snapshots may be partial).
int check_status_locked(rgg_roadmap_t r, cudaStream_t s) {
  int st = 0;
  RGG_CK(cudaMemcpyAsync(&st, r->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  RGG_CK(cudaStreamSynchronize(s));
  if (st != 0) {
    RGG_CK(cudaMemsetAsync(r->d_status, 0, sizeof(int), s));
    for (auto& q : r->req_state)
      if (q != 0) q = 3;
    if (r->has_edges) {
      const int rc = requeue_present(r, s);
      if (rc != RGG_OK) return rc;
    }
    RGG_CK(cudaStreamSynchronize(s));
    return RGG_ERR_TIMEOUT;
  }
  return RGG_OK;
}


}  // namespace rgg_host

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
      !std::isfinite(desc->margin_m) || desc->geometry > RGG_GEOMETRY_OBB ||
      desc->record_format > RGG_RECORDS_SPHERES)
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
  r->record_format = desc->record_format;
  r->present.assign(r->M, 0);
  r->run_idx.assign(r->M, -1);
  r->req_state.assign(RGG_MAX_REQUESTS, 0);
  r->stage_rows = r->M + RGG_PENDING_EXTRA;
  cudaError_t e = cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, r->device);
  if (e == cudaSuccess) e = dalloc(&r->d_table, (size_t)r->M * 16);
  if (e == cudaSuccess) e = dalloc(&r->d_stage, (size_t)r->stage_rows * 16);
  if (e == cudaSuccess) e = dalloc(&r->d_changed, (size_t)kBoxAreaFloats);
  if (e == cudaSuccess) e = cudaMemset(r->d_changed, 0, (size_t)kBoxAreaFloats * sizeof(float));
  if (e == cudaSuccess) e = dalloc(&r->d_status, 4);
  if (e == cudaSuccess) e = dalloc(&r->d_work, 6);
  if (e == cudaSuccess) e = dalloc(&r->d_count, 3);
  if (e == cudaSuccess) e = cudaMemset(r->d_count, 0, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = dalloc(&r->d_obbwork, 2);
  if (e == cudaSuccess) e = dalloc(&r->d_streamed, 1);
  if (e == cudaSuccess) e = cudaMemset(r->d_obbwork, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(r->d_streamed, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(r->d_table, 0, (size_t)r->M * 16 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(r->d_status, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    device_free(r->d_table);
    device_free(r->d_stage);
    device_free(r->d_changed);
    device_free(r->d_status);
    device_free(r->d_work);
    device_free(r->d_count);
    device_free(r->d_obbwork);
    device_free(r->d_streamed);
    delete r;
    return cuda_status(e);
  }
  // one mapped page-locked word for the listed-tile count (optional: without
  // it every pass runs the roadmap's own variant)
  if (cudaHostAlloc(reinterpret_cast<void**>(&r->h_listed), sizeof(uint32_t), cudaHostAllocMapped) !=
          cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&r->d_listed), r->h_listed, 0) != cudaSuccess) {
    cudaGetLastError();
    if (r->h_listed) cudaFreeHost(r->h_listed);
    r->h_listed = r->d_listed = nullptr;
  } else {
    *r->h_listed = 0;
  }
  *out = r;
  return RGG_OK;
}

int rgg_roadmap_destroy(rgg_roadmap_t r) {
  if (!r) return RGG_OK;
  DeviceGuard g(r->device);
  cudaDeviceSynchronize();
  r->es.release();
  device_free(r->d_table);
  device_free(r->d_stage);
  device_free(r->d_changed);
  device_free(r->d_status);
  device_free(r->d_work);
  device_free(r->d_count);
  device_free(r->d_obbwork);
  device_free(r->d_streamed);
  if (r->h_listed) cudaFreeHost(r->h_listed);
  for (auto& ev : r->events)
    for (cudaEvent_t x : ev) cudaEventDestroy(x);
  delete r;
  return RGG_OK;
}

int rgg_upload_edges(rgg_roadmap_t r, uint64_t num_edges, const uint64_t* sample_off,
                     const float* inner_xyzr, const float* outer_xyzr, int src_is_device,
                     void* stream) {
  TraceRange trace_("rgg_upload_edges");
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
  ShapeRestore shape(r);
  default_shape(r, false);
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
  rc = install_edges(r, std::move(es), s);
  if (rc == RGG_OK) {
    shape.keep = true;
    r->has_robot = false;
  }
  return rc;
}

int rgg_build_edges(rgg_roadmap_t r, const rgg_robot_desc* robot, uint64_t num_edges,
                    const double* q_from, const double* q_to, double step, void* stream) {
  TraceRange trace_("rgg_build_edges");
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
    device_free(d_qa);
    device_free(d_qb);
    device_free(d_counts);
    device_free(d_bad);
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
  const bool joints = use_joints(r);
  ShapeRestore shape(r);
  default_shape(r, joints);
  int rc = alloc_edges(r, &es, num_edges, std::move(soff), s, joints);
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
    bp.joints = joints ? 1u : 0u;
    e = launch_build_records(bp, r->num_sms, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  device_free(d_counts);
  device_free(d_bad);
  if (e != cudaSuccess) {
    device_free(d_qa);
    device_free(d_qb);
    es.release();
    return cuda_status(e);
  }
  // the endpoints stay for the gray resolution
  es.d_qa = d_qa;
  es.d_qb = d_qb;
  es.device_bytes += 2 * qn * sizeof(double);
  // sphere records: centres at (j + 1/2)/K, one radius per link
  es.regular = r->geometry == RGG_GEOMETRY_SPHERES && !joints;
  if (joints) {
    rc = set_link_radii(r, robot->radius, s);
    if (rc != RGG_OK) {
      es.release();
      return rc;
    }
  }
  rc = install_edges(r, std::move(es), s);
  if (rc == RGG_OK) {
    shape.keep = true;
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

int rgg_update_obstacles(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                         const float* pose, int src_is_device, void* stream) {
  TraceRange trace_("rgg_update_obstacles");
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
  TraceRange trace_("rgg_update_request");
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

int rgg_classify(rgg_roadmap_t r, void* stream) {
  TraceRange trace_("rgg_classify");
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges) return RGG_ERR_STATE;
  if (r->pending.empty()) return RGG_OK;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  if (r->geometry == RGG_GEOMETRY_OBB) return classify_group_obb(&r, 1, static_cast<cudaStream_t>(stream));
  return classify_group(&r, 1, static_cast<cudaStream_t>(stream));
}

int rgg_classify_many(rgg_roadmap_t* rs, uint32_t n, void* stream) {
  TraceRange trace_("rgg_classify_many");
  if (!rs && n) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < n; ++i) {
    if (!rs[i]) return RGG_ERR_INVALID;
    if (!rs[i]->has_edges) return RGG_ERR_STATE;
    // one launch runs every roadmap's tiles at the first roadmap's shape
    if (rs[i]->device != rs[0]->device || rs[i]->geometry != rs[0]->geometry ||
        (rs[i]->geometry == RGG_GEOMETRY_SPHERES && rs[i]->es.N && !tiles_fit(rs[i], rs[0]->variant)))
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

int rgg_fetch_labels(rgg_roadmap_t r, uint8_t* out, uint64_t first, uint64_t count,
                     int dst_is_device, void* stream) {
  TraceRange trace_("rgg_fetch_labels");
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
  TraceRange trace_("rgg_fetch_request_labels");
  if (!r || handle >= RGG_MAX_REQUESTS || (!out && count) || dst_is_device < 0 ||
      dst_is_device > 2)
    return RGG_ERR_INVALID;
  if (r->has_edges && r->req_state[handle] == 3) return RGG_ERR_TIMEOUT;
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
  if (r->req_state[handle] != 2 && r->req_state[handle] != 3) return RGG_ERR_STATE;
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
  if (inner_xyzr && es.joints) {
    // link-end records: the inner spheres they stand for, centres
    // interpolated in FP64 from the stored FP32 ends and rounded, radii R_i
    const uint32_t L = r->L, K = r->K;
    const uint64_t g0 = (uint64_t)L * s0, ng = (uint64_t)L * (s1 - s0);
    std::vector<float> J(3 * ng);
    float lr[kLinkRadiiFloats];
    for (int p = 0; p < 3; ++p)
      RGG_CK(cudaMemcpy(J.data() + p * ng, es.d_inner + p * es.in_stride + g0, ng * 4,
                        cudaMemcpyDeviceToHost));
    RGG_CK(cudaMemcpy(lr, r->d_changed + kBoxesPerPass * kBoxRecFloats, sizeof(lr),
                      cudaMemcpyDeviceToHost));
    for (uint64_t e = first; e < first + count; ++e) {
      const uint64_t n = es.h_soff[e + 1] - es.h_soff[e];
      const uint64_t ge = (uint64_t)L * es.h_soff[e] - g0;
      for (uint32_t i = 0; i < L; ++i)
        for (uint64_t k = 0; k < n; ++k) {
          const uint64_t g = ge + i * n + k;
          for (uint32_t j = 0; j < K; ++j) {
            const double f = ((double)j + 0.5) / (double)K;
            const uint64_t out = (uint64_t)K * g + j;
            for (int c = 0; c < 3; ++c) {
              const double b = J[c * ng + g], a = i > 0 ? J[c * ng + g - n] : 0.0;
              inner_xyzr[c * ni + out] = (float)(a + f * (b - a));
            }
            inner_xyzr[3 * ni + out] = lr[i];
          }
        }
    }
  }
  for (int p = 0; p < 4; ++p) {
    if (inner_xyzr && !es.joints)
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
  out->num_inner = es.joints ? (uint64_t)r->K * es.G : es.n_inner;
  out->num_outer = es.n_outer;
  out->record_bytes = es.joints ? 12 * es.n_inner + 16 * es.n_outer : 16 * (es.n_inner + es.n_outer);
  out->record_format = es.joints ? RGG_RECORDS_LINK_ENDS : RGG_RECORDS_SPHERES;
  out->device_bytes = es.device_bytes + fixed_device_bytes(r);
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
  out->round_filter = filter_active(r) ? 1u : 0u;
  out->variant = (uint32_t)r->variant;
  out->last_variant = (uint32_t)(r->last_variant >= 0 ? r->last_variant : r->variant);
  if (r->geometry == RGG_GEOMETRY_OBB) {
    // boxes, spline vertices and spline offsets
    out->num_inner = es.n_spl_v;
    out->num_outer = es.n_obb;
    out->record_bytes = 64 * es.n_obb + 16 * es.n_spl_v + 8 * (es.n_spl + 1);
  }
  out->grid_ctas = (uint32_t)std::min<uint64_t>(es.T, launch_ctas(r));
  return RGG_OK;
}

int rgg_set_round_filter(rgg_roadmap_t r, int enable) {
  if (!r) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;
  const int mode = enable ? 1 : 0;
  const bool was = filter_wanted(r, &r->es);
  const int old_mode = r->round_filter_mode;
  r->round_filter_mode = mode;
  if (filter_wanted(r, &r->es) == was) return RGG_OK;
  DeviceGuard g(r->device);
  if (!g.ok) {
    r->round_filter_mode = old_mode;
    return RGG_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {  // no launch may still read the round data
    cudaGetLastError();
    r->round_filter_mode = old_mode;
    return RGG_ERR_CUDA;
  }
  ++r->gen;                                    // captured step graphs hold the old jobs
  // the round data exist while the filter is on (computed from the records)
  int rc = mode ? compute_rounds(r, &r->es, nullptr) : (release_rounds(&r->es), RGG_OK);
  if (cudaDeviceSynchronize() != cudaSuccess && rc == RGG_OK) rc = RGG_ERR_CUDA;
  if (rc != RGG_OK) {
    release_rounds(&r->es);
    r->round_filter_mode = 0;
  }
  return rc;
}

int rgg_streamed_bytes(rgg_roadmap_t r, uint64_t* record_bytes) {
  if (!r || !record_bytes) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  unsigned long long v = 0;
  RGG_CK(cudaDeviceSynchronize());
  RGG_CK(cudaMemcpy(&v, r->d_streamed, sizeof(v), cudaMemcpyDeviceToHost));
  RGG_CK(cudaMemset(r->d_streamed, 0, sizeof(v)));
  *record_bytes = v;
  return RGG_OK;
}

int rgg_check_status(rgg_roadmap_t r, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  return check_status_locked(r, static_cast<cudaStream_t>(stream));
}

int rgg_set_work_counting(rgg_roadmap_t r, int enable) {
  if (!r) return RGG_ERR_INVALID;
  r->counting = enable != 0;
  return RGG_OK;
}

int rgg_work_counts(rgg_roadmap_t r, uint64_t* rounds, uint64_t* outer_tests,
                    uint64_t* inner_pairs) {
  if (!r) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  unsigned long long v[3] = {0, 0, 0};
  RGG_CK(cudaDeviceSynchronize());
  RGG_CK(cudaMemcpy(v, r->d_count, sizeof(v), cudaMemcpyDeviceToHost));
  RGG_CK(cudaMemset(r->d_count, 0, sizeof(v)));
  if (rounds) *rounds = v[0];
  if (outer_tests) *outer_tests = v[1];
  if (inner_pairs) *inner_pairs = v[2];
  return RGG_OK;
}

int rgg_set_wait_limit(rgg_roadmap_t r, uint64_t limit_ns) {
  if (!r || limit_ns == 0) return RGG_ERR_INVALID;
  r->wait_ns = limit_ns;
  return RGG_OK;
}

int rgg_inject_alloc_failure(uint64_t nth) {
  g_fail_countdown.store(nth);
  return RGG_OK;
}

int rgg_check_guards(uint64_t* n_checked, uint64_t* n_bad) {
  std::lock_guard<std::mutex> lk(g_guard_mu);
  uint64_t checked = 0, bad = 0;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  int status = RGG_OK;
  std::vector<int> synced;
  unsigned char got[kGuardBytes];
  for (const auto& kv : g_guards) {
    const int dev = kv.second.device;
    if (cudaSetDevice(dev) != cudaSuccess) {
      status = RGG_ERR_CUDA;
      break;
    }
    if (std::find(synced.begin(), synced.end(), dev) == synced.end()) {
      if (cudaDeviceSynchronize() != cudaSuccess) {
        status = RGG_ERR_CUDA;
        break;
      }
      synced.push_back(dev);
    }
    // read only what the runtime still knows as device memory: a buffer
    // released without device_free would be an address nothing backs (it is
    // counted as changed, since its guard cannot be read)
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, kv.first) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      ++checked;
      ++bad;
      continue;
    }
    if (cudaMemcpy(got, static_cast<const unsigned char*>(kv.first) + kv.second.offset, kGuardBytes,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      status = RGG_ERR_CUDA;
      break;
    }
    ++checked;
    for (size_t i = 0; i < kGuardBytes; ++i)
      if (got[i] != kGuardByte) {
        ++bad;
        break;
      }
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (status != RGG_OK) cudaGetLastError();
  if (n_checked) *n_checked = checked;
  if (n_bad) *n_bad = bad;
  if (status == RGG_OK && bad) status = RGG_ERR_STATE;
  return status;
}

int rgg_estimate_bytes(const rgg_roadmap_desc* desc, uint64_t num_edges, const double* q_from,
                       const double* q_to, double step, uint64_t* bytes) {
  if (!desc || !bytes || desc->num_links < 1 || desc->num_links > RGG_MAX_LINKS ||
      desc->inner_per_link < 1 || desc->inner_per_link > RGG_MAX_INNER ||
      desc->max_obstacles < 1 || desc->max_obstacles > RGG_MAX_OBSTACLES ||
      !(step > 0.0) || !std::isfinite(step) || (num_edges && (!q_from || !q_to)) ||
      num_edges >= 0xffffffffull)
    return RGG_ERR_INVALID;
  if (desc->geometry != RGG_GEOMETRY_SPHERES || desc->record_format > RGG_RECORDS_SPHERES)
    return desc->geometry != RGG_GEOMETRY_SPHERES ? RGG_ERR_STATE : RGG_ERR_INVALID;
  const uint32_t L = desc->num_links, K = desc->inner_per_link, M = desc->max_obstacles;
  const bool joints = desc->record_format == RGG_RECORDS_LINK_ENDS &&
                      desc->margin_m >= kRegularMinMargin;
  const uint32_t Wm = (M + 31) / 32;
  // rgg_build_edges' configuration counts, on the host
  std::vector<uint64_t> soff(num_edges + 1, 0);
  for (uint64_t e = 0; e < num_edges; ++e) {
    double m = 0.0;
    for (uint32_t j = 0; j < L; ++j) {
      const double a = q_from[e * L + j], b = q_to[e * L + j];
      if (!std::isfinite(a) || !std::isfinite(b)) return RGG_ERR_INVALID;
      m = std::max(m, std::fabs(b - a));
    }
    const double c = std::ceil(m / step);
    if (!(c < 2147483647.0)) return RGG_ERR_INVALID;
    soff[e + 1] = soff[e] + std::max<uint64_t>(2, (uint64_t)c + 1);
  }
  const uint64_t N = num_edges, S = soff[N], G = (uint64_t)L * S;
  if (N && !valid_soff(soff.data(), N, L)) return RGG_ERR_INVALID;
  // the tiles of the default launch shape (their size depends on the SM
  // count only for roadmaps too small to give every CTA two tiles)
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, desc->device) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  uint64_t tile_bytes = 0;
  uint32_t max_n = 0;
  for (uint64_t e = 0; e < N; ++e) max_n = std::max<uint64_t>(max_n, soff[e + 1] - soff[e]);
  if (N) {
    const Tiling t = choose_tiling(L, K, G, 2 * (uint32_t)sms,
                                   joints ? kDefaultVariantLinkEnds : kDefaultVariant, joints, max_n);
    if (t.S == 0) return RGG_ERR_INVALID;
    std::vector<TileDesc> tiles;
    std::vector<int4> etab;
    if (!build_tiles(L, N, soff, G, t.S, &tiles, &etab)) return RGG_ERR_INVALID;
    // link-end records also keep the spatial filter's round data (on by
    // default for them)
    tile_bytes = tiles.size() * (sizeof(TileDesc) + (joints ? sizeof(uint32_t) : 0)) +
                 etab.size() * sizeof(int4) + (joints ? round_data_bytes(tiles.size()) : 0);
  }
  const uint64_t n_in = joints ? G : (uint64_t)K * G, n_out = (uint64_t)L * (S - N);
  const uint64_t in_stride = ((n_in + 4 + 63) / 64) * 64, out_stride = ((n_out + 4 + 63) / 64) * 64;
  uint64_t b = (N + 1) * 8 + (joints ? 12 : 16) * in_stride + 16 * out_stride;  // offsets, records
  b += N * (2ull * Wm * 4 + 4 + 1 + 8);                         // box sets, counts, labels, pass bits
  b += tile_bytes;
  b += 2 * N * L * sizeof(double);                              // endpoints (gray resolution)
  b += (uint64_t)M * 64 + (uint64_t)(M + RGG_PENDING_EXTRA) * 64 + kBoxAreaFloats * 4 + 16;
  *bytes = b;
  return RGG_OK;
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

int rgg_set_launch_shape(rgg_roadmap_t r, uint32_t variant, uint32_t consumer_warps) {
  if (!r) return RGG_ERR_INVALID;
  const uint32_t cw = consumer_warps ? consumer_warps
                                     : (r->es.joints ? kDefaultConsumerWarpsLinkEnds
                                                     : kDefaultConsumerWarps);
  if (!shape_ok(variant, cw)) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  const int rc = apply_shape(r, (int)variant, cw);
  if (rc == RGG_OK) r->shape_set = true;
  return rc;
}

}  // extern "C"
