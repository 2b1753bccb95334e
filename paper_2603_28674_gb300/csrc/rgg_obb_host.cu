// Host side of the OBB / shortcut-spline geometry (Sec. 4.2, 4.3): building
// the boxes, splines and grid, the per-pass queries, and the calls that only
// this geometry has.
#include "rgg_host.h"

using namespace rgg;
using namespace rgg_host;

namespace rgg_host {

// OBB geometry (Sec. 4.2, 4.3): per (edge, body) boxes and shortcut splines
// built on the GPU in FP64 (spline vertices counted, then written at their
// offsets), then the uniform grid over the boxes: cells of about the boxes'
// mean largest AABB side, at most 32 per axis, each listing the boxes whose
// AABB meets it.
int build_obb(rgg_roadmap* r, EdgeState* es, const rgg_robot_desc* robot, const double* d_qa,
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
    device_free(scratch);
    device_free(d_count);
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
  device_free(scratch);
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
    device_free(d_part);
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
    device_free(d_cc);
    return done(cuda_status(e));
  }
  std::vector<uint32_t> coff(es->n_cells + 1, 0);
  uint64_t items = 0;
  for (uint32_t c = 0; c < es->n_cells; ++c) {
    items += cc[c];
    if (items > 0xffffffffull) {
      device_free(d_cc);
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
  device_free(d_cc);
  // every moved box may list every chunk of every cell, at the smallest chunk
  es->pair_cap = (uint32_t)std::min<uint64_t>(
      0xffffffffull, (uint64_t)kBoxesPerPass * (es->n_cells + items / kObbChunkMin + 1));
  RGG_OB(es->d_pairs, es->pair_cap);
  RGG_OB(es->d_qcnt, 3);
#undef RGG_OB
  if (e != cudaSuccess) return done(cuda_status(e));
  return done(RGG_OK);
}

// OBB geometry: each roadmap's passes in turn.  Per pass: the moved boxes'
// records, the (box, cell) work list and the box / spline tests (Sec. 4.3
// queries with the spatial filter), then the same merge as the sphere path.
int classify_group_obb(rgg_roadmap_t* rs, uint32_t n, cudaStream_t s) {
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
      RGG_CK(cudaMemsetAsync(es.d_qcnt, 0, 3 * sizeof(uint32_t), s));
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

}  // namespace rgg_host

extern "C" {

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

}  // extern "C"
