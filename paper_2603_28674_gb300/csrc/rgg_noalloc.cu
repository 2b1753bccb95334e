// rgg_classify_noalloc: one classification pass for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- a real-time control loop that must not block on the driver's
// allocator, a host that owns every device byte through its own memory
// manager, or a plugin that is handed device buffers and may only launch
// work on them.  Such a caller keeps the records and the per-edge state in
// its own buffers; this entry point only launches kernels on them.
//
// The scratch the pass needs (tile descriptors, per-tile edge tables, the
// per-edge cross-tile accumulators and the moved boxes' derived records)
// lives in one file-scope __device__ array below.  Every device that loads
// this library holds that array (about 3.7 MB) until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "rgg.h"
#include "rgg_kernels.h"

using namespace rgg;

namespace {

// Scratch capacity.
constexpr uint64_t kNaMaxEdges = RGG_NOALLOC_MAX_EDGES;
constexpr uint64_t kNaMaxTiles = RGG_NOALLOC_MAX_TILES;
constexpr uint64_t kNaEtabEntries = kNaMaxEdges + kNaMaxTiles;  // tile t's entries start at e_first + t
constexpr size_t kNaTilesOff = 0;
constexpr size_t kNaEtabOff = kNaTilesOff + kNaMaxTiles * sizeof(TileDesc);
constexpr size_t kNaAccOff = kNaEtabOff + kNaEtabEntries * sizeof(int4);
constexpr size_t kNaBoxOff = kNaAccOff + 2 * kNaMaxEdges * sizeof(uint32_t);
// the box area the classify kernel copies: box records and link radii
constexpr size_t kNaStatusOff = kNaBoxOff + ((kBoxAreaFloats * sizeof(float) + 255) & ~(size_t)255);
constexpr size_t kNaBytes = kNaStatusOff + 256;
constexpr int kNaMaxDevices = 64;

static_assert(kNaEtabOff % 256 == 0 && kNaAccOff % 256 == 0 && kNaBoxOff % 256 == 0 &&
                  kNaStatusOff % 256 == 0,
              "scratch regions stay 256-byte aligned");

}  // namespace

// The scratch array.  In host code its name is only a host-side stand-in:
// kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

namespace {

std::mutex g_na_mutex;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this; make that call before
// any stream capture).
cudaError_t scratch_ptr(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// Tile geometry for this pass (the same stage layout as the library's
// streaming tiles), on the default pipeline shape.
struct NaTiling {
  uint32_t S, off_in, off_out, in_cap, out_cap;
};

bool na_tiling(uint32_t L, uint32_t K, NaTiling* t) {
  const VariantShape v = variant_shape(kDefaultVariant);
  for (uint32_t S = 31 * v.rounds; S >= 1; --S) {
    const uint32_t max_edges = S / (2 * L) + 3;
    const uint32_t off_in = (kStageEtabOff + 16 * max_edges + 15u) & ~15u;
    const uint32_t in_cap = (K * S + 8 + 3u) & ~3u;
    const uint32_t off_out = off_in + 16 * in_cap;
    const uint32_t out_cap = (S + 1 + 8 + 3u) & ~3u;
    if (max_edges <= (uint32_t)kMaxTileEdges &&
        (uint64_t)off_out + 16ull * out_cap <= (uint64_t)v.stage_bytes) {
      *t = NaTiling{S, off_in, off_out, in_cap, out_cap};
      return true;
    }
  }
  return false;
}

bool na_valid_pose(const float* p) {
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

struct NaPrepParams {
  uint32_t C;
  uint32_t ids[kBoxesPerPass];
  float pose[kBoxesPerPass][15];
  float* out;
};

}  // namespace

// Tile descriptors and edge tables from the caller's device sample offsets.
// An edge or tile that breaks the layout rules (n_e < 2, offsets not
// ascending, soff[N] != num_samples, too many edges in a tile) gets a
// degenerate tile whose every access stays inside its stage, so bad input
// gives wrong labels but never an out-of-bounds access.
__global__ void noalloc_tiles_kernel(const uint64_t* __restrict__ soff, uint64_t N,
                                     uint64_t num_samples, uint32_t L, uint32_t S, uint64_t T,
                                     TileDesc* __restrict__ tiles, int4* __restrict__ etab) {
  const uint64_t max_edges = S / (2 * L) + 3;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const uint64_t G = (uint64_t)L * num_samples;
  const uint64_t g0 = t * S, g1 = min(g0 + S, G);
  bool ok = soff[0] == 0 && soff[N] == num_samples;
  // largest e < N with L*soff[e] <= g (bounded search whatever soff holds)
  auto edge_of = [&](uint64_t g) {
    uint64_t lo = 0, hi = N - 1;
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) >> 1;
      if ((uint64_t)L * soff[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  const uint64_t ef = edge_of(g0), el = edge_of(g1 - 1);
  ok = ok && el >= ef && el - ef + 1 <= max_edges;
  for (uint64_t e = ef; ok && e <= el; ++e) {
    const uint64_t a = soff[e], b = soff[e + 1];
    ok = b >= a + 2 && (b - a) * L <= 0x7fffffffull && (uint64_t)L * a <= g1 - 1 &&
         (uint64_t)L * b > g0;
  }
  if (ok) {
    const uint64_t so_f = soff[ef], n_f = soff[ef + 1] - so_f;
    const uint64_t so_l = soff[el], n_l = soff[el + 1] - so_l;
    const uint64_t rf = g0 - L * so_f, i_f = rf / n_f, k_f = rf - i_f * n_f;
    const uint64_t o0 = L * (so_f - ef) + i_f * (n_f - 1) + (k_f > 0 ? k_f - 1 : 0);
    const uint64_t rl = g1 - 1 - L * so_l, i_l = rl / n_l, k_l = rl - i_l * n_l;
    const uint64_t o1 = L * (so_l - el) + i_l * (n_l - 1) + min(k_l, n_l - 2) + 1;
    ok = o1 > o0 && o1 - o0 <= (uint64_t)S + 1;
    if (ok) {
      const uint64_t n_edges = el - ef + 1;
      tiles[t].packed = o0 | ((o1 - o0) << 40) | (n_edges << 56);
      tiles[t].etab = (uint32_t)(ef + t);
      tiles[t].e_first = (uint32_t)ef;
      for (uint64_t e = ef; e <= el; ++e) {
        const uint64_t n = soff[e + 1] - soff[e];
        etab[ef + t + (e - ef)] =
            make_int4((int)((int64_t)(L * soff[e]) - (int64_t)g0), (int)n,
                      (int)((int64_t)(L * (soff[e] - e)) - (int64_t)o0),
                      __float_as_int(__fdiv_rn(1.0f, (float)n)));
      }
      return;
    }
  }
  // degenerate tile: one edge entry with runs of 2 samples, one outer sphere
  tiles[t].packed = 0ull | (1ull << 40) | (1ull << 56);
  tiles[t].etab = (uint32_t)(ef + t);
  tiles[t].e_first = (uint32_t)ef;
  etab[ef + t] = make_int4(0, 2, 0, __float_as_int(0.5f));
}

// Derived records of the pass's boxes from poses given by value (same
// arithmetic as the library's box preparation).
__global__ void noalloc_box_prep_kernel(const __grid_constant__ NaPrepParams p) {
  const uint32_t b = threadIdx.x;
  if (b >= p.C) return;
  const float* row = p.pose[b];
  const double c[3] = {row[0], row[1], row[2]};
  double R[9];
  for (int m = 0; m < 9; ++m) R[m] = row[3 + m];
  const double h[3] = {row[12], row[13], row[14]};
  float* out = p.out + kBoxRecFloats * (size_t)b;
  out[0] = row[0];
  out[1] = row[1];
  out[2] = row[2];
  out[3] = __double2float_ru(sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]) * (1.0 + 1e-6));
  for (int k = 0; k < 3; ++k) {
    const double ax = R[k], ay = R[3 + k], az = R[6 + k];
    out[4 + 4 * k + 0] = (float)ax;
    out[4 + 4 * k + 1] = (float)ay;
    out[4 + 4 * k + 2] = (float)az;
    out[4 + 4 * k + 3] = (float)((double)(float)ax * c[0] + (double)(float)ay * c[1] +
                                 (double)(float)az * c[2]);
  }
  out[16] = row[12];
  out[17] = row[13];
  out[18] = row[14];
  out[19] = __uint_as_float(p.ids[b]);
  for (int m = 20; m < 24; ++m) out[m] = 0.0f;
}

extern "C" int rgg_classify_noalloc(const rgg_noalloc_args* a, void* stream) {
  if (!a) return RGG_ERR_INVALID;
  const uint32_t L = a->num_links, K = a->inner_per_link, C = a->num_boxes, Wm = a->mask_words;
  const uint64_t N = a->num_edges;
  if (L < 1 || L > RGG_MAX_LINKS || K < 1 || K > RGG_MAX_INNER || C > kBoxesPerPass ||
      Wm < 1 || Wm > (RGG_MAX_OBSTACLES + 31) / 32 || !(a->margin_m >= 0.0f) ||
      !std::isfinite(a->margin_m))
    return RGG_ERR_INVALID;
  NaTiling tl;
  if (!na_tiling(L, K, &tl)) return RGG_ERR_INVALID;
  const uint64_t G = (uint64_t)L * a->num_samples;
  const uint64_t T = (G + tl.S - 1) / tl.S;
  if (N > kNaMaxEdges || T > kNaMaxTiles) return RGG_ERR_CAPACITY;
  if (N == 0 || C == 0) return RGG_OK;
  if (a->num_samples < 2 * N || !a->sample_off || !a->inner_xyzr || !a->outer_xyzr ||
      !a->box_ids || !a->box_poses || !a->hit || !a->touch || !a->counts || !a->labels)
    return RGG_ERR_INVALID;
  // planes: 16-byte aligned, strides a multiple of 4 floats with 4 floats of tail room
  const uint64_t n_in = (uint64_t)K * G, n_out = (uint64_t)L * (a->num_samples - N);
  if ((reinterpret_cast<uintptr_t>(a->inner_xyzr) & 15) ||
      (reinterpret_cast<uintptr_t>(a->outer_xyzr) & 15) || (a->inner_stride & 3) ||
      (a->outer_stride & 3) || a->inner_stride < n_in + 4 || a->outer_stride < n_out + 4)
    return RGG_ERR_INVALID;
  // boxes: ids below 32*Wm, no repeats, valid poses; sorted ascending for the merge
  NaPrepParams pp;
  pp.C = C;
  uint32_t order[kBoxesPerPass];
  for (uint32_t i = 0; i < C; ++i) {
    if (a->box_ids[i] >= 32 * Wm || !na_valid_pose(a->box_poses + 15 * (size_t)i))
      return RGG_ERR_INVALID;
    order[i] = i;
  }
  std::sort(order, order + C, [&](uint32_t x, uint32_t y) { return a->box_ids[x] < a->box_ids[y]; });
  for (uint32_t i = 0; i < C; ++i) {
    if (i && a->box_ids[order[i]] == a->box_ids[order[i - 1]]) return RGG_ERR_INVALID;
    pp.ids[i] = a->box_ids[order[i]];
    std::memcpy(pp.pose[i], a->box_poses + 15 * (size_t)order[i], 15 * sizeof(float));
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return RGG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RGG_ERR_CUDA;
  unsigned char* base = nullptr;
  if (scratch_ptr(dev, &base) != cudaSuccess) return RGG_ERR_CUDA;
  TileDesc* tiles = reinterpret_cast<TileDesc*>(base + kNaTilesOff);
  int4* etab = reinterpret_cast<int4*>(base + kNaEtabOff);
  uint32_t* acc = reinterpret_cast<uint32_t*>(base + kNaAccOff);
  float* boxes = reinterpret_cast<float*>(base + kNaBoxOff);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  int* st = reinterpret_cast<int*>(base + kNaStatusOff);
  // the accumulators and the status word must start at zero; the array keeps
  // the last call's contents
  if (cudaMemsetAsync(acc, 0, 2 * N * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess)
    return RGG_ERR_CUDA;
  noalloc_tiles_kernel<<<(unsigned)((T + 127) / 128), 128, 0, s>>>(a->sample_off, N, a->num_samples,
                                                                   L, tl.S, T, tiles, etab);
  pp.out = boxes;
  noalloc_box_prep_kernel<<<1, kBoxesPerPass, 0, s>>>(pp);
  if (cudaGetLastError() != cudaSuccess) return RGG_ERR_CUDA;

  ClassifyParams<1> cp;
  ClassifyJob& j = cp.job[0];
  j = ClassifyJob{};
  j.inner = a->inner_xyzr;
  j.outer = a->outer_xyzr;
  j.in_stride = a->inner_stride;
  j.out_stride = a->outer_stride;
  j.tiles = tiles;
  j.etab = etab;
  j.boxes = boxes;
  j.edge_acc = acc;
  j.G = G;
  j.tile_base = 0;
  j.num_tiles = T;
  j.L = L;
  j.K = K;
  j.S = tl.S;
  j.C = C;
  j.off_in = tl.off_in;
  j.off_out = tl.off_out;
  j.in_cap = tl.in_cap;
  j.out_cap = tl.out_cap;
  j.margin = a->margin_m;
  // the same rule as rgg_classify: interpolated inner centres only for
  // regular records and a margin that covers their error
  j.regular = (a->regular_records && a->margin_m >= 1e-5f) ? 1u : 0u;
  j.inv_k = 1.0f / (float)K;
  j.inv_km1 = K > 1 ? 1.0f / (float)(K - 1) : 0.0f;
  cp.njobs = 1;
  cp.total_tiles = T;
  cp.status = st;
  cp.wait_ns = a->wait_limit_ns ? a->wait_limit_ns : 4000000000ull;
  ClassifyLaunch lc;
  lc.consumer_warps = kDefaultConsumerWarps;
  lc.variant = kDefaultVariant;
  lc.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((T + 1) / 2, (uint64_t)sms));
  if (launch_classify_single(cp, lc, s) != cudaSuccess) return RGG_ERR_CUDA;

  MergeParams<1> mp;
  MergeJob& m = mp.job[0];
  m = MergeJob{};
  m.red = a->hit;
  m.touch = a->touch;
  m.counts = a->counts;
  m.labels = a->labels;
  m.edge_acc = acc;
  m.num_edges = N;
  m.edge_base = 0;
  m.Wm = Wm;
  m.C = C;
  for (uint32_t i = 0; i < C; ++i) m.ids[i] = pp.ids[i];
  mp.njobs = 1;
  mp.total_edges = N;
  // a launch whose bounded wait ran out leaves the caller's state untouched
  mp.status = st;
  if (launch_merge_single(mp, s) != cudaSuccess) return RGG_ERR_CUDA;
  if (a->status &&
      cudaMemcpyAsync(a->status, st, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RGG_ERR_CUDA;
  return RGG_OK;
}
