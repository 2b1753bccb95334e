// Host side of the C ABI declared in include/rgg.h: argument checks, device
// memory, tiling of the record stream, and kernel launches.  Every step of
// the classification runs in the kernels of rgg_kernels.cu.
#include <algorithm>
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

// Streaming tile geometry of one roadmap (see the classify kernel): each
// stage buffer holds a header, the tile's edge table, the pass's box
// records, 4 inner planes and 4 outer planes.
struct Tiling {
  uint32_t S = 0, max_edges = 0;
  uint32_t off_edges = 0, off_boxes = 0, off_in = 0, off_out = 0, in_cap = 0, out_cap = 0;
};

uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }
uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

bool tiling_for(uint32_t L, uint32_t K, uint32_t S, Tiling* t) {
  t->S = S;
  t->max_edges = S / (2 * L) + 3;
  t->off_edges = kStageHdrBytes;
  t->off_boxes = align16(t->off_edges + 16 * t->max_edges);
  t->off_in = align16(t->off_boxes + kBoxesPerPass * kBoxRecFloats * 4);
  t->in_cap = round4(K * S + 8);
  t->off_out = t->off_in + 16 * t->in_cap;
  t->out_cap = round4(S + 1 + 8);
  return (uint64_t)t->off_out + 16ull * t->out_cap <= (uint64_t)kStageBytes;
}

// Largest tile that fits a stage, reduced for small roadmaps so that every
// CTA of the launch gets a few tiles.
Tiling choose_tiling(uint32_t L, uint32_t K, uint64_t G, uint32_t ctas) {
  uint32_t smax = kStageBytes / (16 * (K + 1));
  Tiling t;
  while (smax > 1 && !tiling_for(L, K, smax, &t)) --smax;
  uint64_t want = (G + 4ull * ctas - 1) / (4ull * ctas);
  uint32_t s = (uint32_t)std::min<uint64_t>(smax, std::max<uint64_t>(want, 128));
  s = std::max<uint32_t>(1, std::min(s, smax));
  tiling_for(L, K, s, &t);
  return t;
}

struct EdgeState {
  uint64_t N = 0, S_tot = 0, G = 0, n_inner = 0, n_outer = 0;
  uint64_t in_stride = 0, out_stride = 0;
  std::vector<uint64_t> h_soff;
  uint64_t* d_soff = nullptr;
  float* d_inner = nullptr;
  float* d_outer = nullptr;
  uint32_t* d_tile_edge = nullptr;
  uint64_t T = 0;
  Tiling tiling;
  uint32_t* d_red = nullptr;
  uint32_t* d_touch = nullptr;
  uint8_t* d_labels = nullptr;
  uint32_t* d_edge_acc = nullptr;
  uint32_t* d_edge_done = nullptr;
  uint64_t device_bytes = 0;

  void release() {
    cudaFree(d_soff);
    cudaFree(d_inner);
    cudaFree(d_outer);
    cudaFree(d_tile_edge);
    cudaFree(d_red);
    cudaFree(d_touch);
    cudaFree(d_labels);
    cudaFree(d_edge_acc);
    cudaFree(d_edge_done);
    *this = EdgeState();
  }
};

}  // namespace

struct rgg_roadmap {
  int device = 0;
  uint32_t L = 0, K = 0, M = 0, Wm = 0;
  float margin = 2e-5f;
  int num_sms = 0;
  uint32_t ctas_per_sm = 1, consumer_warps = 16;
  bool has_edges = false;
  EdgeState es;
  float* d_table = nullptr;    // [M][16] box poses
  float* d_changed = nullptr;  // [32][24] derived records of the current pass
  int* d_status = nullptr;
  std::vector<uint8_t> present, is_pending;
  std::vector<uint32_t> pending;
  // kernel timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t events_used = 0;
};

namespace {

uint32_t launch_ctas(const rgg_roadmap* r) { return (uint32_t)r->num_sms * r->ctas_per_sm; }

// Allocate the per-edge state and record planes for N edges with per-edge
// sample offsets h_soff (host), into `es` (not yet visible to the roadmap).
int alloc_edges(rgg_roadmap* r, EdgeState* es, uint64_t N, std::vector<uint64_t>&& soff,
                cudaStream_t s) {
  es->N = N;
  es->h_soff = std::move(soff);
  es->S_tot = es->h_soff[N];
  es->G = (uint64_t)r->L * es->S_tot;
  es->n_inner = (uint64_t)r->K * es->G;
  es->n_outer = (uint64_t)r->L * (es->S_tot - N);
  // plane stride: count + 4 floats of tail slack for 16-byte rounding of the
  // bulk copies, rounded to 64 floats (256 B) to keep planes aligned
  es->in_stride = ((es->n_inner + 4 + 63) / 64) * 64;
  es->out_stride = ((es->n_outer + 4 + 63) / 64) * 64;
  es->tiling = choose_tiling(r->L, r->K, es->G, launch_ctas(r));
  es->T = (es->G + es->tiling.S - 1) / es->tiling.S;
  cudaError_t e = cudaSuccess;
#define RGG_AL(ptr, cnt)                 \
  if (e == cudaSuccess) {                \
    e = dalloc(&(ptr), (cnt));           \
    es->device_bytes += (cnt) * sizeof(*(ptr)); \
  }
  RGG_AL(es->d_soff, N + 1);
  RGG_AL(es->d_inner, 4 * es->in_stride);
  RGG_AL(es->d_outer, 4 * es->out_stride);
  RGG_AL(es->d_tile_edge, es->T + 1);
  RGG_AL(es->d_red, N * r->Wm);
  RGG_AL(es->d_touch, N * r->Wm);
  RGG_AL(es->d_labels, N);
  RGG_AL(es->d_edge_acc, 2 * N);
  RGG_AL(es->d_edge_done, N);
#undef RGG_AL
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(es->d_soff, es->h_soff.data(), (N + 1) * sizeof(uint64_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && N) {
    e = cudaMemsetAsync(es->d_red, 0, N * r->Wm * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_touch, 0, N * r->Wm * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_labels, RGG_GREEN, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_edge_acc, 0, 2 * N * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_edge_done, 0, N * 4, s);
  }
  if (e == cudaSuccess && N) {
    // zero the padded tails so that the rounded bulk copies read defined data
    e = cudaMemsetAsync(es->d_inner, 0, 4 * es->in_stride * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(es->d_outer, 0, 4 * es->out_stride * sizeof(float), s);
  }
  if (e == cudaSuccess && N)
    e = launch_tile_edge(es->d_soff, N, r->L, es->tiling.S, es->T, es->d_tile_edge, s);
  if (e != cudaSuccess) {
    es->release();
    return cuda_status(e);
  }
  return RGG_OK;
}

// Swap in freshly built edges: labels GREEN, box sets empty, every present
// box pending so that the next classify tests it against the new edges.
void install_edges(rgg_roadmap* r, EdgeState&& es) {
  r->es.release();
  r->es = std::move(es);
  r->has_edges = true;
  r->pending.clear();
  std::fill(r->is_pending.begin(), r->is_pending.end(), 0);
  for (uint32_t b = 0; b < r->M; ++b)
    if (r->present[b]) {
      r->pending.push_back(b);
      r->is_pending[b] = 1;
    }
}

bool valid_soff(const uint64_t* soff, uint64_t N) {
  if (!soff || soff[0] != 0) return false;
  for (uint64_t e = 0; e < N; ++e) {
    if (soff[e + 1] < soff[e] + 2) return false;
    if (soff[e + 1] - soff[e] > 0x7fffffffull) return false;
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

cudaEvent_t* next_event_pair(rgg_roadmap* r) {
  if (r->events_used == r->events.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return nullptr;
    }
    r->events.emplace_back(a, b);
  }
  return &r->events[r->events_used++].first;
}

ClassifyJob make_job(rgg_roadmap* r, uint32_t C, uint64_t tile_base) {
  ClassifyJob j{};
  const EdgeState& es = r->es;
  j.inner = es.d_inner;
  j.outer = es.d_outer;
  j.in_stride = es.in_stride;
  j.out_stride = es.out_stride;
  j.soff = es.d_soff;
  j.tile_edge = es.d_tile_edge;
  j.boxes = r->d_changed;
  j.red = es.d_red;
  j.touch = es.d_touch;
  j.labels = es.d_labels;
  j.edge_acc = es.d_edge_acc;
  j.edge_done = es.d_edge_done;
  j.num_edges = es.N;
  j.G = es.G;
  j.tile_base = tile_base;
  j.num_tiles = es.T;
  j.L = r->L;
  j.K = r->K;
  j.S = es.tiling.S;
  j.C = C;
  j.Wm = r->Wm;
  j.off_edges = es.tiling.off_edges;
  j.off_boxes = es.tiling.off_boxes;
  j.off_in = es.tiling.off_in;
  j.off_out = es.tiling.off_out;
  j.in_cap = es.tiling.in_cap;
  j.out_cap = es.tiling.out_cap;
  j.max_edges = es.tiling.max_edges;
  j.margin = r->margin;
  return j;
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
    default: return "unknown status";
  }
}

int rgg_roadmap_create(const rgg_roadmap_desc* desc, rgg_roadmap_t* out) {
  if (!desc || !out) return RGG_ERR_INVALID;
  *out = nullptr;
  if (desc->num_links < 1 || desc->num_links > RGG_MAX_LINKS || desc->inner_per_link < 1 ||
      desc->inner_per_link > RGG_MAX_INNER || desc->max_obstacles < 1 ||
      desc->max_obstacles > RGG_MAX_OBSTACLES || !(desc->margin_m >= 0.0f) ||
      !std::isfinite(desc->margin_m))
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
  r->present.assign(r->M, 0);
  r->is_pending.assign(r->M, 0);
  cudaError_t e = cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, r->device);
  if (e == cudaSuccess) e = dalloc(&r->d_table, (size_t)r->M * 16);
  if (e == cudaSuccess) e = dalloc(&r->d_changed, (size_t)kBoxesPerPass * kBoxRecFloats);
  if (e == cudaSuccess) e = dalloc(&r->d_status, 1);
  if (e == cudaSuccess) e = cudaMemset(r->d_table, 0, (size_t)r->M * 16 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(r->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(r->d_table);
    cudaFree(r->d_changed);
    cudaFree(r->d_status);
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
  cudaFree(r->d_changed);
  cudaFree(r->d_status);
  for (auto& p : r->events) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  delete r;
  return RGG_OK;
}

int rgg_upload_edges(rgg_roadmap_t r, uint64_t num_edges, const uint64_t* sample_off,
                     const float* inner_xyzr, const float* outer_xyzr, int src_is_device,
                     void* stream) {
  if (!r || !sample_off) return RGG_ERR_INVALID;
  if (!valid_soff(sample_off, num_edges)) return RGG_ERR_INVALID;
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
  install_edges(r, std::move(es));
  return RGG_OK;
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  install_edges(r, std::move(es));
  return RGG_OK;
}

int rgg_update_obstacles(rgg_roadmap_t r, uint32_t n_changed, const uint32_t* ids,
                         const float* pose, int src_is_device, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  if (n_changed == 0) return RGG_OK;
  if (!ids || !pose) return RGG_ERR_INVALID;
  std::vector<uint8_t> seen(r->M, 0);
  for (uint32_t i = 0; i < n_changed; ++i) {
    if (ids[i] >= r->M || seen[ids[i]]) return RGG_ERR_INVALID;
    seen[ids[i]] = 1;
    if (!src_is_device && !valid_pose(pose + 15 * (size_t)i)) return RGG_ERR_INVALID;
  }
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (uint32_t base = 0; base < n_changed; base += kMaxUpdateBoxes) {
    BoxUpdateParams p;
    p.n = std::min(kMaxUpdateBoxes, n_changed - base);
    p.table = r->d_table;
    p.dev_pose = src_is_device ? pose + 15 * (size_t)base : nullptr;
    for (uint32_t i = 0; i < p.n; ++i) {
      p.ids[i] = ids[base + i];
      if (!src_is_device) std::memcpy(p.pose[i], pose + 15 * (size_t)(base + i), 15 * sizeof(float));
    }
    RGG_CK(launch_box_update(p, s));
  }
  for (uint32_t i = 0; i < n_changed; ++i) {
    const uint32_t b = ids[i];
    r->present[b] = 1;
    if (!r->is_pending[b]) {
      r->is_pending[b] = 1;
      r->pending.push_back(b);
    }
  }
  return RGG_OK;
}

// One streaming pass per group of <= 32 boxes; for several roadmaps, pass p
// of every roadmap that has one goes into the same persistent launch.
static int classify_group(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s) {
  uint32_t max_passes = 0;
  for (uint32_t i = 0; i < n; ++i)
    max_passes = std::max<uint32_t>(max_passes, (uint32_t)((rs[i]->pending.size() + kBoxesPerPass - 1) /
                                                            kBoxesPerPass));
  std::unique_ptr<BoxPrepParams> bpp(new (std::nothrow) BoxPrepParams);
  std::unique_ptr<ClassifyParams<kMaxJobs>> cpp;
  if (n > 1) cpp.reset(new (std::nothrow) ClassifyParams<kMaxJobs>);
  if (!bpp || (n > 1 && !cpp)) return RGG_ERR_OOM;
  for (uint32_t pass = 0; pass < max_passes; ++pass) {
    BoxPrepParams& bp = *bpp;
    bp.njobs = 0;
    ClassifyParams<1> cp1;
    uint32_t nj = 0;
    uint64_t tiles = 0;
    uint32_t tw_cap = 0, acc_cap = 0;
    rgg_roadmap* timed = nullptr;
    for (uint32_t i = 0; i < n; ++i) {
      rgg_roadmap* r = rs[i];
      const size_t lo = (size_t)pass * kBoxesPerPass;
      if (lo >= r->pending.size()) continue;
      const uint32_t C = (uint32_t)std::min<size_t>(kBoxesPerPass, r->pending.size() - lo);
      BoxPrepJob& pj = bp.job[bp.njobs++];
      pj.table = r->d_table;
      pj.out = r->d_changed;
      pj.C = C;
      for (uint32_t b = 0; b < C; ++b) pj.ids[b] = r->pending[lo + b];
      if (r->es.N == 0) continue;
      ClassifyJob job = make_job(r, C, tiles);
      if (n == 1) cp1.job[0] = job; else cpp->job[nj] = job;
      ++nj;
      tiles += r->es.T;
      tw_cap = std::max(tw_cap, r->es.tiling.S + 2);
      acc_cap = std::max(acc_cap, r->es.tiling.max_edges);
      if (r->timing && !timed) timed = r;
    }
    RGG_CK(launch_box_prep(bp, s));
    if (nj == 0) continue;
    rgg_roadmap* r0 = rs[0];
    ClassifyLaunch lc;
    lc.consumer_warps = r0->consumer_warps;
    lc.grid = (uint32_t)std::min<uint64_t>(tiles, launch_ctas(r0));
    lc.tw_cap = tw_cap;
    lc.acc_cap = acc_cap;
    cudaEvent_t* ev = timed ? next_event_pair(timed) : nullptr;
    if (ev) RGG_CK(cudaEventRecord(ev[0], s));
    if (n == 1) {
      cp1.njobs = 1;
      cp1.total_tiles = tiles;
      cp1.status = r0->d_status;
      RGG_CK(launch_classify_single(cp1, lc, s));
    } else {
      cpp->njobs = nj;
      cpp->total_tiles = tiles;
      cpp->status = r0->d_status;
      RGG_CK(launch_classify_batched(*cpp, lc, s));
    }
    if (ev) RGG_CK(cudaEventRecord(ev[1], s));
  }
  for (uint32_t i = 0; i < n; ++i) {
    for (uint32_t b : rs[i]->pending) rs[i]->is_pending[b] = 0;
    rs[i]->pending.clear();
  }
  return RGG_OK;
}

int rgg_classify(rgg_roadmap_t r, void* stream) {
  if (!r) return RGG_ERR_INVALID;
  if (!r->has_edges) return RGG_ERR_STATE;
  if (r->pending.empty()) return RGG_OK;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  return classify_group(&r, 1, static_cast<cudaStream_t>(stream));
}

int rgg_classify_many(rgg_roadmap_t* rs, uint32_t n, void* stream) {
  if (!rs && n) return RGG_ERR_INVALID;
  for (uint32_t i = 0; i < n; ++i) {
    if (!rs[i]) return RGG_ERR_INVALID;
    if (!rs[i]->has_edges) return RGG_ERR_STATE;
    if (rs[i]->device != rs[0]->device) return RGG_ERR_INVALID;
    for (uint32_t j = 0; j < i; ++j)
      if (rs[j] == rs[i]) return RGG_ERR_INVALID;
  }
  if (n == 0) return RGG_OK;
  DeviceGuard g(rs[0]->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
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
  if (!r || (!out && count)) return RGG_ERR_INVALID;
  if (!r->has_edges && count) return RGG_ERR_STATE;
  if (first > r->es.N || count > r->es.N - first) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (count)
    RGG_CK(cudaMemcpyAsync(out, r->es.d_labels + first, count,
                           dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!dst_is_device) return check_status_locked(r, s);
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
  if (!r->has_edges) return RGG_ERR_STATE;
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
  out->device_bytes = es.device_bytes + (uint64_t)r->M * 64 + kBoxesPerPass * kBoxRecFloats * 4 + 4;
  out->num_links = r->L;
  out->inner_per_link = r->K;
  out->max_obstacles = r->M;
  out->mask_words = r->Wm;
  out->tile_samples = es.tiling.S;
  out->num_tiles = es.T;
  out->pending_boxes = (uint32_t)r->pending.size();
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

int rgg_kernel_time(rgg_roadmap_t r, double* ms, uint64_t* launches) {
  if (!r || !ms || !launches) return RGG_ERR_INVALID;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  double total = 0.0;
  for (size_t i = 0; i < r->events_used; ++i) {
    RGG_CK(cudaEventSynchronize(r->events[i].second));
    float t = 0.f;
    RGG_CK(cudaEventElapsedTime(&t, r->events[i].first, r->events[i].second));
    total += t;
  }
  *ms = total;
  *launches = r->events_used;
  r->events_used = 0;
  return RGG_OK;
}

int rgg_set_launch_shape(rgg_roadmap_t r, uint32_t ctas_per_sm, uint32_t consumer_warps) {
  if (!r) return RGG_ERR_INVALID;
  const uint32_t cps = ctas_per_sm ? ctas_per_sm : 1;
  const uint32_t cw = consumer_warps ? consumer_warps : 16;
  if (cw < 1 || cw > 31 || cps < 1 || cps > 2) return RGG_ERR_INVALID;
  if (cps * classify_smem_bytes(kStageBytes / 16 + 2, kStageBytes / 16) > 232448) return RGG_ERR_INVALID;
  r->ctas_per_sm = cps;
  r->consumer_warps = cw;
  return RGG_OK;
}

}  // extern "C"
