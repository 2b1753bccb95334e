// Device-side structures and PTX helpers shared by the RGG kernels.
//
// Record layout on the device (one roadmap), in one of two formats:
//   sphere records (uploaded edges, or built ones on request)
//     inner spheres  4 FP32 planes (x, y, z, r), plane p at inner + p*in_stride;
//                    sphere (edge e, link i, sample k, sphere j) at
//                    K*(L*soff[e] + i*n_e + k) + j   (Sec. 4.3's E^- tensor,
//                    unpadded: edge, body, configuration, sphere)
//   link-end records (built edges, the default)
//     link ends      3 FP32 planes (x, y, z); entry L*soff[e] + i*n_e + k holds
//                    the far end o_{i+1} of link i at configuration k.  The
//                    near end of link i is entry - n_e (the far end of link
//                    i-1), or the base (the world origin) for link 0.  The K
//                    inner spheres of (e, i, k) sit at fractions (j + 1/2)/K of
//                    the segment between the two ends, radius R_i (a per-
//                    roadmap table), so only 12 B per (edge, link,
//                    configuration) are stored instead of 16*K.
//   outer spheres  4 FP32 planes; sphere (e, i, interval k) at
//                  L*(soff[e] - e) + i*(n_e - 1) + k
// A "global sample" g indexes the concatenation over edges and links of the
// configurations: edge e owns g in [L*soff[e], L*soff[e+1]), link i of it the
// n_e consecutive values starting at L*soff[e] + i*n_e.  Sample g's inner
// spheres are K consecutive records starting at K*g.
//
// Streaming tiles: tile t covers the global samples [t*S, min((t+1)*S, G)),
// every interval adjacent to one of them (one halo interval before the first
// sample when the tile starts inside a link's run), and a table with one
// entry per edge that has samples in the tile.  With link-end records the
// tile also copies the h_t entries before its first sample that belong to
// its first edge (h_t = min(n_e, offset of the tile in that edge), at most
// one link's run), which hold the near ends of its first samples.
//
// Rounds: round r of a tile is its samples [31r, 31r+31) and the intervals
// that follow its local samples 31r-1 .. 31r+30 (those a consumer warp tests
// in one step).  Spatial filter (Sec. 4.3, "spatially filtered many-to-many
// checking"; on by default for link-end records): while it is on, every
// round has a bounding sphere of those intervals' outer spheres and their
// range of outer records, and every tile a sphere holding its rounds'
// spheres (recomputed whenever the tiles change); before each pass a small
// kernel tests the spheres against the pass's moved boxes and lists the
// tiles some box can reach, and the classify kernel copies only those tiles'
// rounds that some box can reach.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rgg {

constexpr int kMaxJobs = 128;          // roadmaps per batched launch
constexpr int kBoxesPerPass = 32;      // moved boxes per streaming pass (one mask word)
constexpr int kBoxRecFloats = 24;      // derived box record, 6 x float4 = 96 B
constexpr int kStageHdrBytes = 32;
constexpr int kRoundSlots = 32;        // round entries per tile (rounds per tile <= 32)
constexpr int kAccMax = 96;            // per-stage accumulator entries (edges per tile)
constexpr int kStageAccOff = kStageHdrBytes;                 // hit[kAccMax], touch[kAccMax]
constexpr int kStageEtabOff = kStageAccOff + 8 * kAccMax;    // edge table
constexpr int kMaxTileEdges = kAccMax;
constexpr int kBoxSlots = 2;           // jobs whose box records a CTA stages in shared memory
// The pass's box area: 32 derived box records, then the link radii R_i of the
// roadmap (link-end records take their inner radius from there).
constexpr int kLinkRadiiFloats = 32;
constexpr int kBoxAreaFloats = kBoxesPerPass * kBoxRecFloats + kLinkRadiiFloats;

// Derived record of one moved box, built by the box-prep kernel:
//   r0 = (centre.xyz, bounding radius |h| rounded up)
//   r1..r3 = (box axis k in world coordinates, axis_k . centre)
//   r4 = (half-extents, box id as raw bits), r5 = padding
// so that the box-frame coordinate k of a point x is dot(axis_k, x) - u_k.

// Per-tile descriptor (16 B), built on the host when edges are set.
struct TileDesc {
  uint64_t packed;   // bits 0..39 o0 (first outer sphere), 40..55 n_out, 56..63 n_edges
  uint32_t etab;     // index of the tile's first edge-table entry
  uint32_t e_first;  // global index of the tile's first edge
};
// Edge-table entry (int4): {estart, n, ostart, bits of (float)1/n}
//   estart  local sample index of the edge's first sample (may be < 0)
//   n       configurations of the edge
//   ostart  local interval index of the edge's first interval (may be < 0)

// One roadmap's part of a classify launch.
struct ClassifyJob {
  const float* inner;               // inner-sphere planes, or link-end planes (joints)
  const float* outer;
  uint64_t in_stride, out_stride;   // floats between planes
  const TileDesc* tiles;            // [T]
  const int4* etab;                 // edge tables of all tiles
  const float* boxes;               // box area: [32][24] derived records, then link radii
  uint32_t* edge_acc;               // [N][2] (hit, touch) bits of this pass, kept zero between passes
  uint64_t G;                       // L * soff[N] global samples
  uint64_t tile_base;               // first queue index of this job's tiles
  uint64_t num_tiles;
  uint32_t L, K, S, C;              // links, inner/link, samples per tile, boxes
  uint32_t off_in, off_out;         // byte offsets of the first inner / outer plane in a stage
  uint32_t in_cap, out_cap;         // floats per plane slot in a stage
  float margin;
  // 1: every sample's K inner spheres share one radius and sit at equal steps
  // along a segment (the records rgg_build_edges writes), so the kernel may
  // interpolate their centres from the first and the last
  uint32_t regular;
  // 1: link-end records (see above); the inner spheres are interpolated from
  // the two ends of their link, always (the margin covers it)
  uint32_t joints;
  const uint32_t* tile_halo;        // [T] link-end entries copied before a tile's first sample
  float inv_k, inv_km1;             // 1/K and 1/(K-1) (0 when K = 1)
  // spatial filter (null: every round of every tile is copied)
  const float4* rsph;               // [T][kRoundSlots] bounding sphere (radius < 0: empty)
  const float4* tsph = nullptr;     // [T] a sphere holding the tile's round spheres (radius < 0: none)
  const uint32_t* rout;             // [T][kRoundSlots] outer records lo | hi << 16, tile-local
  uint32_t* rcand;                  // [T][kRoundSlots] moved boxes that may reach the round
  // the pass's tiles that some moved box may reach: local tile indices in no
  // particular order, appended by the filter kernel, and their count (zeroed
  // by the box-prep kernel at the start of each pass).  With a list the
  // classify kernel's ring slots take only these tiles.  Null: every tile.
  uint32_t* tlist = nullptr;        // [T]
  uint32_t* tcount = nullptr;
  unsigned long long* streamed;     // record bytes copied (may be null)
  const int* status = nullptr;      // the roadmap's own status word (may be null)
};

template <int MAXJ>
struct ClassifyParams {
  ClassifyJob job[MAXJ];
  uint32_t njobs;
  uint64_t total_tiles;
  int* status;                      // device status word of the launch (0 = ok)
  unsigned long long* work = nullptr;  // [3] work counters (counting launches only)
  uint64_t wait_ns = 4000000000ull; // limit of every bounded wait, ns of wall time
  // a mapped page-locked host word that receives the launch's listed tiles
  // (filtered single-roadmap launches; the host picks the next pass's shape)
  uint32_t* listed_out = nullptr;
};

// Per-stage header, written by the warp that fills the stage.
struct StageHdr {
  int32_t job;
  int32_t n_samp;      // configurations in the tile
  int32_t n_out;       // intervals in the tile (including the halo)
  int32_t n_edges;     // local edges
  int32_t in_shift;    // first inner float inside the aligned copy
  int32_t out_shift;
  uint32_t e_first;
  int32_t end;         // 1: no more tiles for the warp that takes this slot
};
static_assert(sizeof(StageHdr) == kStageHdrBytes, "stage header size");

// Merge of one roadmap's pass results into its per-edge box sets.
struct MergeJob {
  uint32_t* red;          // [N][Wm]
  uint32_t* touch;        // [N][Wm]
  uint32_t* counts;       // [N] red count | touch count << 16
  uint8_t* labels;        // [N]
  uint32_t* edge_acc;     // [N][2]
  uint64_t num_edges;
  uint64_t edge_base;     // first global thread index of this job
  uint32_t Wm, C;
  uint32_t ids[kBoxesPerPass];  // box id of pass position p
  // ordered == 0: ids ascend and are distinct (word-grouped update);
  // ordered == 1: positions apply in order (a box may repeat), and after each
  // position p in snap_mask the labels so far go to hist[snap_slot[p]][e]
  uint32_t ordered;
  uint32_t snap_mask;
  uint8_t* hist;
  uint8_t snap_slot[kBoxesPerPass];
  int* status = nullptr;  // the roadmap's status word: a failed launch's code is copied here
};

template <int MAXJ>
struct MergeParams {
  MergeJob job[MAXJ];
  uint32_t njobs;
  uint64_t total_edges;
  // status word of the classify launch whose bits are merged (may be null):
  // when it is set, the launch did not finish its tiles, so the per-edge
  // sets and labels are left as they were and only the accumulators are
  // cleared
  const int* status = nullptr;
};

enum StatusCode : int {
  kStatusOk = 0,
  kStatusTimeoutFull = 1,
  kStatusTimeoutEmpty = 2,
  kStatusTimeoutBoxes = 3,
  // the launch found an error already latched (by an earlier launch) and
  // did no work: its pass still has to be run again
  kStatusSkipped = 4,
};

// ---------------------------------------------------------------------------
// PTX helpers (mbarrier + bulk async copy, sm_90+ / sm_100+ forms)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Non-blocking test of phase `parity` (acquire, CTA scope): true once the
// phase has completed, and the data its transactions delivered is visible.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: non-blocking tests of the phase until it completes or
// `limit_ns` of wall time have passed (then false).  On the classify kernel
// this measured faster than the blocking try_wait with a suspend hint, and
// faster than sleeping 10-400 ns between tests.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_test_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Bulk copy global -> shared (this CTA), completion counted on `bar` in bytes.
// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace rgg
