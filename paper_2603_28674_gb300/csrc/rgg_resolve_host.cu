// Host side of the non-lazy resolution of gray edges (rgg_resolve_gray).
#include "rgg_host.h"

using namespace rgg;
using namespace rgg_host;

extern "C" {

// ---------------------------------------------------------------------------
// Non-lazy resolution of gray edges
// ---------------------------------------------------------------------------
int rgg_resolve_gray(rgg_roadmap_t r, uint32_t factor, uint8_t* labels_out, float* clearance_out,
                     int dst_is_device, rgg_resolve_stats* stats, void* stream) {
  TraceRange trace_("rgg_resolve_gray");
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
    if (e == cudaSuccess) e = dalloc(&es.d_gray, N);
    if (e != cudaSuccess) {
      device_free(es.d_resolved);
      device_free(es.d_clear);
      device_free(es.d_gray);
      es.d_resolved = nullptr;
      es.d_clear = nullptr;
      es.d_gray = nullptr;
      return cuda_status(e);
    }
    es.device_bytes += 9 * N;
  }
  RGG_CK(cudaMemsetAsync(r->d_work, 0, 6 * sizeof(unsigned long long), s));
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
  p.gray = es.d_gray;
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

}  // extern "C"
