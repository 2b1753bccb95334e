// Host-visible launch interface of the RGG kernels (internal to librgg.so).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rgg_device.cuh"

namespace rgg {

// Compiled shapes of the streaming pipeline: (id, stages in the shared-memory
// ring, bytes per stage, rounds of 31 samples per tile, rounds per work item).
// Each stage holds one tile: header, accumulators, edge table, inner and
// outer record planes; beside it, the tile's round candidates and 3 KB for
// the tile's job's box records.
// Variants 7..9 keep big tiles but hold more of them in flight: link-end
// records need 12 B per sample instead of 16*K, so a 23..31-round tile fits
// a 27..38 KB stage.  Variants 10 and 11 trade tile size for ring depth
// (8 x 20-round and 10 x 16-round tiles): a sparse pass, whose tiles carry
// few live rounds, is bound by how many tiles each CTA has in flight.  Every
// shape also fits the batched launch, whose stages each keep a box area.
#define RGG_VARIANTS(X)             \
  X(0, 14, 10 * 1024, 3, 1)        \
  X(1, 7, 28 * 1024, 9, 1)         \
  X(2, 6, 33 * 1024, 10, 1)        \
  X(3, 5, 40 * 1024, 13, 1)        \
  X(4, 4, 51 * 1024, 17, 1)        \
  X(5, 3, 69 * 1024, 23, 1)        \
  X(6, 4, 51 * 1024, 16, 2)        \
  X(7, 7, 27 * 1024, 23, 2)        \
  X(8, 6, 32 * 1024, 27, 1)        \
  X(9, 5, 38 * 1024, 31, 1)        \
  X(10, 8, 23 * 1024, 20, 2)       \
  X(11, 10, 18 * 1024, 16, 2)      \
  X(12, 8, 23 * 1024, 20, 3)
constexpr int kNumVariants = 13;
// Default shapes: sphere records take variant 5 with 24 consumer warps;
// link-end records (a third of the bytes per tile) variant 10, whose deeper
// ring keeps more tiles in flight, with 27: of the shapes timed on the large
// dense, large mixed-label and 7-DOF roadmaps it was the one faster than
// variant 7 on all three (variant 11 is faster still on the sparse two and
// slower on the dense one).
constexpr int kDefaultVariant = 5;
constexpr uint32_t kDefaultConsumerWarps = 24;
constexpr int kDefaultVariantLinkEnds = 10;
constexpr uint32_t kDefaultConsumerWarpsLinkEnds = 27;
// Variant 12 is variant 10 (the same stages and tiles) with 3 rounds per work
// item: faster when nearly every tile has rounds to test (each item's later
// rounds see its earlier rounds' hits, and a tile has fewer items), slower
// when tiles carry few live rounds (fewer warps share a tile).  A roadmap on
// the default shape with at least kDensePassMinTiles tiles runs it for a pass
// when its previous pass listed at least kDensePassPermille / 1000 of its
// tiles.  The count reaches the host through one store of the classify
// kernel into mapped host memory, which measured about 2 us longer per launch
// on a 46k-tile roadmap and nothing measurable on longer launches: smaller
// roadmaps keep variant 10 and skip the store.
constexpr int kDenseVariantLinkEnds = 12;
constexpr uint32_t kDensePassPermille = 950;
constexpr uint64_t kDensePassMinTiles = 262144;
// The spatial filter's kernel instance exists for the default variants and
// the other deep-ring link-end shapes.
constexpr bool filter_variant(int v) { return v == kDefaultVariant || v == 7 || v >= 10; }
constexpr int kMaxClassifyThreads = 896;  // up to 28 worker warps
struct VariantShape {
  int stages, stage_bytes, rounds, rounds_per_item;
};
inline VariantShape variant_shape(int v) {
  switch (v) {
#define RGG_VARIANT(id, ns, sb, rd, rpi) \
  case id: return VariantShape{ns, sb, rd, rpi};
    RGG_VARIANTS(RGG_VARIANT)
#undef RGG_VARIANT
    default: return VariantShape{0, 0, 0, 0};
  }
}
constexpr int kMaxBuildLinks = 32;
constexpr uint32_t kMaxUpdateBoxes = 256;  // poses carried by value per update launch

struct BuildParams {
  uint32_t L, K;
  double a[kMaxBuildLinks], alpha[kMaxBuildLinks], d[kMaxBuildLinks], radius[kMaxBuildLinks];
  const double* qa;
  const double* qb;
  const uint64_t* soff;
  float* inner;
  float* outer;
  uint64_t in_stride, out_stride;
  uint64_t n_edges;
  uint32_t joints;   // 1: write link-end records (3 planes) instead of inner spheres
};

// Writes boxes' poses into the box table and into the staging rows of their
// pending entries; with from_table set, copies table rows into staging rows.
struct BoxUpdateParams {
  uint32_t n;
  uint32_t ids[kMaxUpdateBoxes];
  uint32_t rows[kMaxUpdateBoxes];   // staging row of each id's pending entry
  float pose[kMaxUpdateBoxes][15];
  const float* dev_pose;  // if non-null, poses are read from device memory
  float* table;           // [M][16]
  float* stage;           // [rows][16]
  uint32_t from_table;
};

struct BoxPrepJob {
  const float* stage;     // staging rows of the pending entries
  float* out;             // [C][24]
  // the roadmap's count of spatially filtered tiles, zeroed here before the
  // pass's filter kernel appends to its list (null: no list)
  uint32_t* tcount = nullptr;
  uint32_t C;
  uint32_t ids[kBoxesPerPass];
  uint16_t rows[kBoxesPerPass];  // staging row of pass position p
};

struct BoxPrepParams {
  BoxPrepJob job[kMaxJobs];
  uint32_t njobs;
};

struct ClassifyLaunch {
  uint32_t grid;
  uint32_t consumer_warps;
  int variant;
};

// Non-lazy resolution of gray edges (Algorithm 1 with lazy = false): each
// gray edge's link capsules are checked at (n_e - 1) * F + 1 configurations
// against the boxes of its touch set.
struct ResolveParams {
  uint32_t L, Wm, F;
  float thr;                        // decision margin, metres
  float a[kMaxBuildLinks], d[kMaxBuildLinks], ca[kMaxBuildLinks], sa[kMaxBuildLinks];
  float radius[kMaxBuildLinks];
  const double* qa;                 // [N][L] edge endpoints
  const double* qb;
  const uint64_t* soff;             // [N+1]
  const uint8_t* labels;            // [N] lazy labels
  const uint32_t* touch;            // [N][Wm] touch sets
  const float* table;               // [M][16] box poses
  uint8_t* out;                     // [N] resolved labels
  float* clearance;                 // [N] minimum clearance found (NaN: not gray)
  unsigned long long* work;         // [6]: gray edges, red, green, segment-box evaluations,
                                    // gray edges listed, gray edges taken
  uint32_t* gray;                   // [N] the gray edges, in no particular order
  uint64_t n_edges;
};

// ---------------------------------------------------------------------------
// The paper's primitives (Sec. 4.2, 4.3): per (edge, body) OBBs and shortcut
// splines, a uniform grid over the OBBs, and the per-pass queries.
// ---------------------------------------------------------------------------
// OBB record: 4 float4 = (centre, 0), (u1, h1), (u2, h2), (u3, h3).
// Grid-cell boxes per query work item, chosen per pass between these bounds
// from the pass's total work (obb_pairs_kernel).
constexpr uint32_t kObbChunkMin = 256, kObbChunkMax = 4096;
struct ObbBuildParams {
  uint32_t L, K;
  double a[kMaxBuildLinks], alpha[kMaxBuildLinks], d[kMaxBuildLinks], radius[kMaxBuildLinks];
  const double* qa;
  const double* qb;
  const uint64_t* soff;
  uint64_t n_edges;
  double* scratch;            // per warp: max_n * (L + 1) * 3 doubles of joint positions
  uint64_t scratch_per_warp;  // doubles
  float4* obb;                // [N * L][4] (pass 0 only)
  uint32_t* spl_count;        // [N * L * K] kept vertices per spline (pass 0)
  const uint64_t* spl_off;    // [N * L * K + 1] (pass 1)
  float4* spl_v;              // vertices (pass 1)
  int pass;                   // 0: boxes and counts; 1: vertices
};

struct GridSpec {
  float ox, oy, oz, cell;     // origin and cell side
  uint32_t gx, gy, gz;        // cells per axis
};

struct ObbGridParams {
  const float4* obb;
  uint64_t n_obb;
  GridSpec g;
  uint32_t* cell_count;       // pass 0: incidences per cell (atomic)
  const uint32_t* cell_off;   // pass 1: offsets
  uint32_t* cell_cursor;      // pass 1: fill cursors (atomic)
  float4* cell_items;         // pass 1: per item (AABB low corner, OBB index bits), (high corner, 0)
  int pass;
};

struct ObbQueryParams {
  uint32_t L, K, C;
  float margin;
  GridSpec g;
  const float4* obb;
  const uint64_t* spl_off;
  const float4* spl_v;
  const uint32_t* cell_off;
  const float4* cell_items;   // 2 float4 per item, see ObbGridParams
  const float* boxes;         // [C][24] derived records of the pass's boxes
  uint32_t* edge_acc;         // [N][2]
  uint2* pairs;               // (box position | chunk << 5, cell) work list
  uint32_t* counters;         // [0] pairs listed, [1] pairs taken, [2] this pass's chunk size
  uint32_t target_items;      // work items the chunk size aims at
  uint32_t pair_cap;
  uint32_t filter;            // 0: every non-empty cell for every box (no spatial filter)
  unsigned long long* work;   // [2] SAT tests, spline-segment tests (may be null)
};

// Per-round bounding spheres and outer ranges of one roadmap's tiles (see
// rgg_device.cuh), computed from its resident outer records.
struct RoundBoundsParams {
  const float* outer;
  uint64_t out_stride;
  const TileDesc* tiles;
  const int4* etab;
  uint64_t T, G;
  uint32_t S;
  float4* rsph;               // [T][kRoundSlots]
  uint32_t* rout;             // [T][kRoundSlots]
  float4* tsph;               // [T] a sphere about each tile's round spheres
};

size_t classify_smem_bytes(int variant, uint32_t consumer_warps);

cudaError_t launch_count_samples(const double* qa, const double* qb, uint64_t n_edges, uint32_t L,
                                 double step, uint64_t* counts, int* bad, cudaStream_t s);
cudaError_t launch_build_records(const BuildParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_box_update(const BoxUpdateParams& p, cudaStream_t s);
cudaError_t launch_box_prep(const BoxPrepParams& p, cudaStream_t s);
cudaError_t launch_classify_single(const ClassifyParams<1>& p, const ClassifyLaunch& lc,
                                   cudaStream_t s);
cudaError_t launch_classify_batched(const ClassifyParams<kMaxJobs>& p, const ClassifyLaunch& lc,
                                    cudaStream_t s);
cudaError_t launch_round_bounds(const RoundBoundsParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_merge_single(const MergeParams<1>& p, cudaStream_t s);
cudaError_t launch_merge_batched(const MergeParams<kMaxJobs>& p, cudaStream_t s);
cudaError_t launch_resolve_gray(const ResolveParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_obb_build(const ObbBuildParams& p, uint32_t warps, cudaStream_t s);
cudaError_t launch_obb_bounds(const float4* obb, uint64_t n_obb, float* partial, uint32_t blocks,
                              cudaStream_t s);
cudaError_t launch_obb_grid(const ObbGridParams& p, cudaStream_t s);
cudaError_t launch_obb_query(const ObbQueryParams& p, int num_sms, cudaStream_t s);

}  // namespace rgg
