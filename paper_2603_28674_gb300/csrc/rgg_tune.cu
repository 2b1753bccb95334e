// Host side of the autotuner (rgg_autotune) and of captured step graphs
// (rgg_step_graph_*).
#include "rgg_host.h"

using namespace rgg;
using namespace rgg_host;

extern "C" {

// ---------------------------------------------------------------------------
// Autotuner: time the classify launch of these roadmaps at every supported
// launch shape, on their own records and boxes, and keep the fastest.
// ---------------------------------------------------------------------------
// One pass over the roadmaps' tiles with C[i] boxes each, OR-ing into the
// scratch accumulators acc[i] (labels and box sets are untouched): the box
// prep (which also starts the spatial filter's tile lists afresh), then the
// classify launch.
static int tune_launch(rgg_roadmap_t* rs, uint32_t n, const std::vector<uint32_t*>& acc,
                const std::vector<uint32_t>& C, const BoxPrepParams& bp,
                ClassifyParams<kMaxJobs>* cpp, cudaStream_t s) {
  RGG_CK(launch_box_prep(bp, s));
  ClassifyParams<1> cp1;
  uint32_t nj = 0;
  uint64_t tiles = 0;
  for (uint32_t i = 0; i < n; ++i) {
    rgg_roadmap* r = rs[i];
    if (r->es.N == 0 || C[i] == 0) continue;
    ClassifyJob j = make_job(r, C[i], tiles);
    j.edge_acc = acc[i];
    j.streamed = nullptr;
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
  if (n == 1) {
    cp1.njobs = 1;
    cp1.total_tiles = tiles;
    cp1.status = r0->d_status;
    cp1.wait_ns = r0->wait_ns;
    RGG_CK(launch_classify_single(cp1, lc, s));
  } else {
    cpp->njobs = nj;
    cpp->total_tiles = tiles;
    cpp->status = r0->d_status;
    cpp->wait_ns = r0->wait_ns;
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
  TraceRange trace_("rgg_autotune");
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
    pj.tcount = nullptr;
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
  std::vector<uint32_t*> acc(n, nullptr);
  auto free_acc = [&]() {
    for (uint32_t* p : acc) device_free(p);
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
      // the filter's list count of each shape's launches (filter_active
      // depends on the shape)
      for (uint32_t i = 0; i < n; ++i)
        bpp->job[i].tcount = filter_active(rs[i]) ? rs[i]->es.d_tlist + rs[i]->es.T : nullptr;
      rc = tune_launch(rs, n, acc, C, *bpp, cpp.get(), s);  // warm-up
      // each repetition between its own events; the median is kept, so that
      // one odd reading cannot pick the shape
      std::vector<float> times;
      for (uint32_t k = 0; k < reps && rc == RGG_OK; ++k) {
        if (cudaEventRecord(ev.a, s) != cudaSuccess) rc = RGG_ERR_CUDA;
        if (rc == RGG_OK) rc = tune_launch(rs, n, acc, C, *bpp, cpp.get(), s);
        float ms = 0.f;
        if (rc == RGG_OK && (cudaEventRecord(ev.b, s) != cudaSuccess ||
                             cudaEventSynchronize(ev.b) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess))
          rc = RGG_ERR_CUDA;
        times.push_back(ms);
      }
      if (rc != RGG_OK) break;
      std::sort(times.begin(), times.end());
      rgg_tune_result t{};
      t.variant = (uint32_t)v;
      t.consumer_warps = cw;
      t.classify_ms = times[times.size() / 2];
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
      if (rc2 == RGG_OK) rs[i]->shape_set = true;
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
  TraceRange trace_("rgg_step_graph_launch");
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
