// CUDA kernels of the RGG edge-classification pass (sm_103a).
//
//   count_samples_kernel   a0: configurations per edge (Sec. 3.2)
//   build_records_kernel   a0: FP64 kinematics -> FP32 inner/outer spheres
//                          (Sec. 4.2 inner spheres; swept outer spheres)
//   tile_edge_kernel       streaming tiles -> first edge of each tile
//   box_update_kernel      a1: write moved boxes' poses in place (Sec. 4.3,
//                          "Online updates")
//   box_prep_kernel        a1: derived per-pass box records
//   classify_kernel        a2..a6: persistent streaming classification
//                          (Sec. 4.1 labelling rule, Algorithm 1 merge)
#include <cstdio>

#include "rgg_device.cuh"
#include "rgg_kernels.h"

namespace rgg {

// ===========================================================================
// a0: configurations per edge
// ===========================================================================
// n_e = max(2, ceil(max_j |qb_j - qa_j| / step) + 1), in FP64 (Sec. 3.2's
// ||e||/eps with the max-norm as the edge length, both endpoints kept).
__global__ void count_samples_kernel(const double* __restrict__ qa, const double* __restrict__ qb,
                                     uint64_t n_edges, uint32_t L, double step,
                                     uint64_t* __restrict__ counts, int* __restrict__ bad) {
  uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e >= n_edges) return;
  double m = 0.0;
  bool finite = true;
  for (uint32_t j = 0; j < L; ++j) {
    double a = qa[e * L + j], b = qb[e * L + j];
    finite = finite && isfinite(a) && isfinite(b);
    m = fmax(m, fabs(b - a));
  }
  double c = ceil(m / step);
  // more than 2^31 configurations on one edge is rejected
  if (!finite || !(c < 2147483647.0)) {
    atomicExch(bad, 1);
    counts[e] = 2;
    return;
  }
  uint64_t n = (uint64_t)c + 1;
  counts[e] = n < 2 ? 2 : n;
}

// ===========================================================================
// a0: sphere records
// ===========================================================================
// One warp per edge; lane k handles configurations k, k+32, ...  Kinematics
// walks the DH chain frame by frame (R, o), emitting each link's spheres as
// soon as both of its end frames are known.
__global__ void __launch_bounds__(256) build_records_kernel(const __grid_constant__ BuildParams p) {
  __shared__ double s_ca[32], s_sa[32], s_len[32];
  if (threadIdx.x < p.L) {
    double s, c;
    sincos(p.alpha[threadIdx.x], &s, &c);
    s_ca[threadIdx.x] = c;
    s_sa[threadIdx.x] = s;
    s_len[threadIdx.x] = sqrt(p.a[threadIdx.x] * p.a[threadIdx.x] + p.d[threadIdx.x] * p.d[threadIdx.x]);
  }
  __syncthreads();
  const uint32_t L = p.L, K = p.K;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  float* ix = p.inner;
  float* iy = p.inner + p.in_stride;
  float* iz = p.inner + 2 * p.in_stride;
  float* ir = p.inner + 3 * p.in_stride;
  float* ox = p.outer;
  float* oy = p.outer + p.out_stride;
  float* oz = p.outer + 2 * p.out_stride;
  float* orr = p.outer + 3 * p.out_stride;

  for (uint64_t e = warp; e < p.n_edges; e += nwarps) {
    const uint64_t so = p.soff[e];
    const uint64_t n = p.soff[e + 1] - so;
    const double inv = 1.0 / (double)(n - 1);
    const double* qa = p.qa + e * L;
    const double* qb = p.qb + e * L;
    const uint64_t in_base = (uint64_t)K * ((uint64_t)L * so);
    const uint64_t out_base = (uint64_t)L * (so - e);
    for (uint64_t k = lane; k < n; k += 32) {
      // ---- inner spheres at q_k = qa + (k/(n-1)) (qb - qa)
      {
        const double t = (double)k * inv;
        double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        double o[3] = {0, 0, 0};
        for (uint32_t i = 0; i < L; ++i) {
          const double q = qa[i] + t * (qb[i] - qa[i]);
          double st, ct;
          sincos(q, &st, &ct);
          const double ca = s_ca[i], sa = s_sa[i];
          const double v0 = p.a[i] * ct, v1 = p.a[i] * st, v2 = p.d[i];
          double on[3];
          for (int r = 0; r < 3; ++r) on[r] = o[r] + R[3 * r] * v0 + R[3 * r + 1] * v1 + R[3 * r + 2] * v2;
          const float rad = __double2float_rd(p.radius[i]);
          const uint64_t base = in_base + (uint64_t)K * ((uint64_t)i * n + k);
          for (uint32_t j = 0; j < K; ++j) {
            const double f = ((double)j + 0.5) / (double)K;
            ix[base + j] = (float)(o[0] + f * (on[0] - o[0]));
            iy[base + j] = (float)(o[1] + f * (on[1] - o[1]));
            iz[base + j] = (float)(o[2] + f * (on[2] - o[2]));
            ir[base + j] = rad;
          }
          // R <- R * Rz(q) Rx(alpha)
          const double A[9] = {ct, -st * ca, st * sa, st, ct * ca, -ct * sa, 0.0, sa, ca};
          double Rn[9];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
              Rn[3 * r + c] = R[3 * r] * A[c] + R[3 * r + 1] * A[3 + c] + R[3 * r + 2] * A[6 + c];
          for (int m = 0; m < 9; ++m) R[m] = Rn[m];
          for (int r = 0; r < 3; ++r) o[r] = on[r];
        }
      }
      // ---- outer sphere of each link over [q_k, q_{k+1}], at its middle
      if (k + 1 < n) {
        const double t = ((double)k + 0.5) * inv;
        double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        double o[3] = {0, 0, 0};
        double prefix_dq = 0.0;  // sum_{j<=m} |dq_j|
        double sweep = 0.0;      // sum_{m<=i} l_m * prefix_dq(m) = sum_{j<=i} |dq_j| rho_{j,i}
        for (uint32_t i = 0; i < L; ++i) {
          const double dqi = (qb[i] - qa[i]) * inv;
          const double q = qa[i] + t * (qb[i] - qa[i]);
          double st, ct;
          sincos(q, &st, &ct);
          const double ca = s_ca[i], sa = s_sa[i];
          const double v0 = p.a[i] * ct, v1 = p.a[i] * st, v2 = p.d[i];
          double on[3];
          for (int r = 0; r < 3; ++r) on[r] = o[r] + R[3 * r] * v0 + R[3 * r + 1] * v1 + R[3 * r + 2] * v2;
          prefix_dq += fabs(dqi);
          sweep += s_len[i] * prefix_dq;
          const double rad = 0.5 * s_len[i] + p.radius[i] + 0.5 * sweep;
          const uint64_t idx = out_base + (uint64_t)i * (n - 1) + k;
          ox[idx] = (float)(0.5 * (o[0] + on[0]));
          oy[idx] = (float)(0.5 * (o[1] + on[1]));
          oz[idx] = (float)(0.5 * (o[2] + on[2]));
          orr[idx] = __double2float_ru(rad);
          const double A[9] = {ct, -st * ca, st * sa, st, ct * ca, -ct * sa, 0.0, sa, ca};
          double Rn[9];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
              Rn[3 * r + c] = R[3 * r] * A[c] + R[3 * r + 1] * A[3 + c] + R[3 * r + 2] * A[6 + c];
          for (int m = 0; m < 9; ++m) R[m] = Rn[m];
          for (int r = 0; r < 3; ++r) o[r] = on[r];
        }
      }
    }
  }
}

// ===========================================================================
// streaming tiles: edge holding the first sample of each tile
// ===========================================================================
__global__ void tile_edge_kernel(const uint64_t* __restrict__ soff, uint64_t n_edges, uint32_t L,
                                 uint32_t S, uint64_t n_tiles, uint32_t* __restrict__ out) {
  uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  const uint64_t G = (uint64_t)L * soff[n_edges];
  const uint64_t g = t * (uint64_t)S;
  if (g >= G) {
    out[t] = (uint32_t)n_edges;
    return;
  }
  // largest e < N with L*soff[e] <= g
  uint64_t lo = 0, hi = n_edges - 1;
  while (lo < hi) {
    uint64_t mid = (lo + hi + 1) >> 1;
    if ((uint64_t)L * soff[mid] <= g) lo = mid; else hi = mid - 1;
  }
  out[t] = (uint32_t)lo;
}

// ===========================================================================
// a1: obstacle update and per-pass box records
// ===========================================================================
__global__ void box_update_kernel(const __grid_constant__ BoxUpdateParams p) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const float* src = p.dev_pose ? p.dev_pose + 15 * (size_t)i : p.pose[i];
  float* dst = p.table + 16 * (size_t)p.ids[i];
  for (int c = 0; c < 15; ++c) dst[c] = src[c];
  dst[15] = 0.0f;
}

// Derived records (see rgg_device.cuh) from the box table, in FP64 then
// rounded: axis_k = column k of R, u_k = axis_k . centre, bounding radius
// |h| rounded up.
__global__ void box_prep_kernel(const __grid_constant__ BoxPrepParams p) {
  const BoxPrepJob& J = p.job[blockIdx.x];
  const uint32_t b = threadIdx.x;
  if (b >= J.C) return;
  const uint32_t id = J.ids[b];
  const float* row = J.table + 16 * (size_t)id;
  const double c[3] = {row[0], row[1], row[2]};
  double R[9];
  for (int m = 0; m < 9; ++m) R[m] = row[3 + m];
  const double h[3] = {row[12], row[13], row[14]};
  float* out = J.out + kBoxRecFloats * (size_t)b;
  out[0] = row[0];
  out[1] = row[1];
  out[2] = row[2];
  out[3] = __double2float_ru(sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]) * (1.0 + 1e-6));
  for (int k = 0; k < 3; ++k) {
    const double ax = R[k], ay = R[3 + k], az = R[6 + k];
    out[4 + 4 * k + 0] = (float)ax;
    out[4 + 4 * k + 1] = (float)ay;
    out[4 + 4 * k + 2] = (float)az;
    // use the FP32-rounded axis so that dot(axis_f, x) - u matches the kernel
    out[4 + 4 * k + 3] = (float)((double)(float)ax * c[0] + (double)(float)ay * c[1] +
                                 (double)(float)az * c[2]);
  }
  out[16] = row[12];
  out[17] = row[13];
  out[18] = row[14];
  out[19] = __uint_as_float(id);
  for (int m = 20; m < 24; ++m) out[m] = 0.0f;
}

// ===========================================================================
// a2..a6: persistent streaming classification
// ===========================================================================
__device__ __forceinline__ float box_dist2(float x, float y, float z, const float4* __restrict__ B) {
  const float4 a0 = B[1], a1 = B[2], a2 = B[3], h = B[4];
  const float p0 = fmaf(a0.x, x, fmaf(a0.y, y, fmaf(a0.z, z, -a0.w)));
  const float p1 = fmaf(a1.x, x, fmaf(a1.y, y, fmaf(a1.z, z, -a1.w)));
  const float p2 = fmaf(a2.x, x, fmaf(a2.y, y, fmaf(a2.z, z, -a2.w)));
  const float e0 = fmaxf(fabsf(p0) - h.x, 0.0f);
  const float e1 = fmaxf(fabsf(p1) - h.y, 0.0f);
  const float e2 = fmaxf(fabsf(p2) - h.z, 0.0f);
  return fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
}

// largest j in [0, n) with tab[4*j + field] <= v (tab[field] <= v holds)
__device__ __forceinline__ int search_le(const int* tab, int field, int n, int v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[4 * mid + field] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Algorithm 1 merge for one edge, by one warp: replace the bits of this
// pass's boxes in the edge's hit / touch sets, then label from the sets.
__device__ __forceinline__ void merge_edge(const ClassifyJob& J, uint64_t e, uint32_t hit,
                                           uint32_t tch, const float4* __restrict__ bx, int lane) {
  bool any_r = false, any_t = false;
  for (uint32_t w = lane; w < J.Wm; w += 32) {
    uint32_t* pr = J.red + e * J.Wm + w;
    uint32_t* pt = J.touch + e * J.Wm + w;
    const uint32_t rw = *pr, tw = *pt;
    uint32_t rn = rw, tn = tw;
    for (uint32_t b = 0; b < J.C; ++b) {
      const uint32_t id = __float_as_uint(bx[6 * b + 4].w);
      if ((id >> 5) == w) {
        const uint32_t bit = 1u << (id & 31);
        rn = ((hit >> b) & 1u) ? (rn | bit) : (rn & ~bit);
        tn = ((tch >> b) & 1u) ? (tn | bit) : (tn & ~bit);
      }
    }
    if (rn != rw) *pr = rn;
    if (tn != tw) *pt = tn;
    any_r |= rn != 0;
    any_t |= tn != 0;
  }
  any_r = __any_sync(0xffffffffu, any_r);
  any_t = __any_sync(0xffffffffu, any_t);
  if (lane == 0) J.labels[e] = any_r ? 2 : (any_t ? 1 : 0);
}

template <int MAXJ>
__device__ __forceinline__ int find_job(const ClassifyParams<MAXJ>& P, uint64_t t) {
  int lo = 0, hi = (int)P.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.job[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr uint32_t kWaitLimit = 1u << 25;

template <int MAXJ, int NSTAGE, int STAGE_BYTES>
__global__ void __launch_bounds__(1024, 1) classify_kernel(const __grid_constant__ ClassifyParams<MAXJ> P,
                                                           uint32_t tw_cap, uint32_t acc_cap) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
  uint64_t* empty = full + NSTAGE;
  volatile int* s_abort = reinterpret_cast<volatile int*>(empty + NSTAGE);
  uint32_t* tw = reinterpret_cast<uint32_t*>(empty + NSTAGE + 2);
  uint32_t* acc_hit = tw + tw_cap;
  uint32_t* acc_touch = acc_hit + acc_cap;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ncw = (blockDim.x >> 5) - 1;
  const int nct = ncw * 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    *s_abort = 0;
    fence_mbar_init();
  }
  for (uint32_t i = threadIdx.x; i < acc_cap; i += blockDim.x) {
    acc_hit[i] = 0;
    acc_touch[i] = 0;
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t it = 0;
    for (uint64_t t = blockIdx.x; t < P.total_tiles; t += gridDim.x, ++it) {
      const int stage = it % NSTAGE;
      const uint32_t round = it / NSTAGE;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_bounded(&empty[stage], (round & 1) ^ 1, kWaitLimit);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicCAS(P.status, 0, (int)kStatusTimeoutEmpty);
          *s_abort = 1;
        }
        break;
      }
      if (*s_abort) break;
      const int jb = find_job(P, t);
      const ClassifyJob& J = P.job[jb];
      const uint64_t lt = t - J.tile_base;
      const uint64_t L = J.L, K = J.K;
      const uint64_t g0 = lt * J.S;
      const uint64_t g1 = min(g0 + J.S, J.G);
      const uint64_t ef = J.tile_edge[lt];
      uint64_t el = J.tile_edge[lt + 1];
      if (el >= J.num_edges || L * J.soff[el] >= g1) el = el - 1;  // edge of sample g1-1
      const uint64_t so_f = J.soff[ef], n_f = J.soff[ef + 1] - so_f;
      const uint64_t so_l = J.soff[el], n_l = J.soff[el + 1] - so_l;
      // first interval: the one before the first sample (halo) if the tile starts
      // inside a link's run of configurations, else the run's first interval
      const uint64_t rf = g0 - L * so_f, i_f = rf / n_f, k_f = rf - i_f * n_f;
      const uint64_t o0 = L * (so_f - ef) + i_f * (n_f - 1) + (k_f > 0 ? k_f - 1 : 0);
      // last interval: the one after the last sample, or the one before it if
      // the last sample ends its run
      const uint64_t rl = g1 - 1 - L * so_l, i_l = rl / n_l, k_l = rl - i_l * n_l;
      const uint64_t o1 = L * (so_l - el) + i_l * (n_l - 1) + min(k_l, n_l - 2) + 1;
      const int n_edges = (int)(el - ef + 1);
      unsigned char* sb = stages + (size_t)stage * STAGE_BYTES;
      int4* etab = reinterpret_cast<int4*>(sb + J.off_edges);
      const bool fits = n_edges <= (int)J.max_edges && (o1 - o0) <= (uint64_t)tw_cap &&
                        n_edges <= (int)acc_cap;
      if (fits) {
        for (int x = lane; x < n_edges; x += 32) {
          const uint64_t e = ef + x;
          const uint64_t so = J.soff[e], sn = J.soff[e + 1];
          const int64_t estart = (int64_t)(L * so) - (int64_t)g0;
          const int64_t ostart = (int64_t)(L * (so - e)) - (int64_t)o0;
          const uint64_t lo = max(g0, L * so), hi = min(g1, L * sn);
          etab[x] = make_int4((int)estart, (int)(sn - so), (int)ostart, (int)(hi - lo));
        }
      }
      const uint64_t a0 = (K * g0) & ~3ull, a1 = (K * g1 + 3) & ~3ull;
      const uint64_t b0 = o0 & ~3ull, b1 = (o1 + 3) & ~3ull;
      if (lane == 0) {
        StageHdr* h = reinterpret_cast<StageHdr*>(sb);
        h->job = jb;
        h->n_samp = (int)(g1 - g0);
        h->n_out = (int)(o1 - o0);
        h->n_edges = n_edges;
        h->in_shift = (int)(K * g0 - a0);
        h->out_shift = (int)(o0 - b0);
        h->valid = fits ? 1 : 0;
        h->e_first = ef;
        h->g0 = g0;
      }
      __syncwarp();
      if (lane == 0) {
        const uint32_t in_bytes = fits ? (uint32_t)((a1 - a0) * 4) : 0;
        const uint32_t out_bytes = fits ? (uint32_t)((b1 - b0) * 4) : 0;
        const uint32_t box_bytes = fits ? J.C * (uint32_t)(kBoxRecFloats * 4) : 0;
        mbar_arrive_expect_tx(&full[stage], 4 * in_bytes + 4 * out_bytes + box_bytes);
        if (fits) {
          for (int pl = 0; pl < 4; ++pl) {
            bulk_g2s(sb + J.off_in + (size_t)pl * J.in_cap * 4, J.inner + pl * J.in_stride + a0,
                     in_bytes, &full[stage]);
            bulk_g2s(sb + J.off_out + (size_t)pl * J.out_cap * 4, J.outer + pl * J.out_stride + b0,
                     out_bytes, &full[stage]);
          }
          if (box_bytes) bulk_g2s(sb + J.off_boxes, J.boxes, box_bytes, &full[stage]);
        }
      }
    }
    // On abort, wait (bounded) for copies this CTA may still have in flight.
    if (*s_abort && lane == 0) {
      const uint32_t first = it > (uint32_t)NSTAGE ? it - NSTAGE : 0;
      for (uint32_t k = first; k < it; ++k)
        mbar_wait_bounded(&full[k % NSTAGE], (k / NSTAGE) & 1, 1u << 16);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int cw = warp - 1;
  const int ctid = threadIdx.x - 32;
  uint32_t it = 0;
  for (uint64_t t = blockIdx.x; t < P.total_tiles; t += gridDim.x, ++it) {
    const int stage = it % NSTAGE;
    const uint32_t round = it / NSTAGE;
    // One thread takes the bounded wait and the abort decision, so that all
    // consumer threads leave the loop together (the named barriers below
    // need every consumer thread).
    if (ctid == 0) {
      int stop = *s_abort;
      if (!stop && !mbar_wait_bounded(&full[stage], round & 1, kWaitLimit)) {
        atomicCAS(P.status, 0, (int)kStatusTimeoutFull);
        *s_abort = 1;
        stop = 1;
      }
      s_abort[1] = stop;
    }
    named_bar_sync(1, nct);
    if (s_abort[1]) break;
    // the phase is complete: this returns at once and orders the stage's
    // bulk-copied data before this thread's reads
    mbar_wait_bounded(&full[stage], round & 1, kWaitLimit);
    unsigned char* sb = stages + (size_t)stage * STAGE_BYTES;
    const StageHdr* hdr = reinterpret_cast<const StageHdr*>(sb);
    const ClassifyJob& J = P.job[hdr->job];
    if (!hdr->valid) {
      if (ctid == 0) atomicCAS(P.status, 0, (int)kStatusBadTile);
      named_bar_sync(1, nct);
      if (ctid == 0) mbar_arrive(&empty[stage]);
      continue;
    }
    const int n_samp = hdr->n_samp, n_out = hdr->n_out, n_edges = hdr->n_edges;
    const int K = (int)J.K;
    const int L = (int)J.L;
    const int C = (int)J.C;
    const float margin = J.margin;
    const float* ix = reinterpret_cast<const float*>(sb + J.off_in) + hdr->in_shift;
    const float* iy = ix + J.in_cap;
    const float* iz = iy + J.in_cap;
    const float* ir = iz + J.in_cap;
    const float* ox = reinterpret_cast<const float*>(sb + J.off_out) + hdr->out_shift;
    const float* oy = ox + J.out_cap;
    const float* oz = oy + J.out_cap;
    const float* orad = oz + J.out_cap;
    const float4* bx = reinterpret_cast<const float4*>(sb + J.off_boxes);
    const int* etab = reinterpret_cast<const int*>(sb + J.off_edges);

    // ---- a3: outer spheres vs moved boxes, warp-culled
    for (int base = cw * 32; base < n_out; base += nct) {
      const int o = base + lane;
      const bool act = o < n_out;
      float x = 0.f, y = 0.f, z = 0.f, r = 0.f;
      if (act) {
        x = ox[o];
        y = oy[o];
        z = oz[o];
        r = orad[o];
      }
      const int nact = min(32, n_out - base);
      const int mid = nact >> 1;
      const float mx = __shfl_sync(0xffffffffu, x, mid);
      const float my = __shfl_sync(0xffffffffu, y, mid);
      const float mz = __shfl_sync(0xffffffffu, z, mid);
      const float dx = x - mx, dy = y - my, dz = z - mz;
      const float reach = act ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + r : 0.0f;
      const float rw = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(reach)));
      bool cb = false;
      if (lane < C) {
        const float4 b0 = bx[6 * lane];
        const float ex = b0.x - mx, ey = b0.y - my, ez = b0.z - mz;
        const float thr = (rw + b0.w + margin) * (1.0f + 1e-6f) + 1e-5f;
        cb = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= thr * thr;
      }
      uint32_t cand = __ballot_sync(0xffffffffu, cb);
      const float rt = r + margin;
      const float rt2 = rt * rt;
      uint32_t bits = 0;
      while (cand) {
        const int b = __ffs(cand) - 1;
        cand &= cand - 1;
        if (box_dist2(x, y, z, bx + 6 * b) <= rt2) bits |= 1u << b;
      }
      if (act) {
        tw[o] = bits;
        if (bits) {
          const int j = search_le(etab, 2, n_edges, o);
          atomicOr(&acc_touch[j], bits);
        }
      }
    }
    named_bar_sync(1, nct);

    // ---- a4: inner spheres, only against boxes their outer spheres touched
    for (int q = ctid; q < n_samp; q += nct) {
      const int j = search_le(etab, 0, n_edges, q);
      const int estart = etab[4 * j], n = etab[4 * j + 1], ostart = etab[4 * j + 2];
      const int rr = q - estart;
      const int li = rr / n;
      const int k = rr - li * n;
      const int ib = ostart + li * (n - 1);
      uint32_t need = (k < n - 1 ? tw[ib + k] : 0u) | (k > 0 ? tw[ib + k - 1] : 0u);
      need &= ~*reinterpret_cast<volatile uint32_t*>(&acc_hit[j]);
      uint32_t hits = 0;
      while (need) {
        const int b = __ffs(need) - 1;
        need &= need - 1;
        const float4* B = bx + 6 * b;
        for (int s = K * q, se = K * q + K; s < se; ++s) {
          const float rin = ir[s] - margin;
          if (rin > 0.0f && box_dist2(ix[s], iy[s], iz[s], B) <= rin * rin) {
            hits |= 1u << b;
            break;
          }
        }
      }
      if (hits) atomicOr(&acc_hit[j], hits);
    }
    named_bar_sync(1, nct);

    // ---- a5/a6: per-edge reduction and merge
    for (int jl = cw; jl < n_edges; jl += ncw) {
      const int estart = etab[4 * jl], n = etab[4 * jl + 1], cnt = etab[4 * jl + 3];
      const uint64_t e = hdr->e_first + jl;
      uint32_t h = acc_hit[jl], tc = acc_touch[jl];
      const bool complete = estart >= 0 && estart + L * n <= n_samp;
      bool do_merge = true;
      if (!complete) {
        int last = 0;
        if (lane == 0) {
          if (h) atomicOr(&J.edge_acc[2 * e], h);
          if (tc) atomicOr(&J.edge_acc[2 * e + 1], tc);
          __threadfence();
          const uint32_t old = atomicAdd(&J.edge_done[e], (uint32_t)cnt);
          last = (old + (uint32_t)cnt == (uint32_t)(L * n));
          if (last) {
            __threadfence();
            h = atomicExch(&J.edge_acc[2 * e], 0u);
            tc = atomicExch(&J.edge_acc[2 * e + 1], 0u);
            J.edge_done[e] = 0;
          }
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        h = __shfl_sync(0xffffffffu, h, 0);
        tc = __shfl_sync(0xffffffffu, tc, 0);
        do_merge = last != 0;
      }
      if (do_merge) merge_edge(J, e, h, tc, bx, lane);
      if (lane == 0) {
        acc_hit[jl] = 0;
        acc_touch[jl] = 0;
      }
    }
    named_bar_sync(1, nct);
    if (ctid == 0) mbar_arrive(&empty[stage]);
  }
}

// ===========================================================================
// host-side launchers
// ===========================================================================
cudaError_t launch_count_samples(const double* qa, const double* qb, uint64_t n_edges, uint32_t L,
                                 double step, uint64_t* counts, int* bad, cudaStream_t s) {
  if (n_edges == 0) return cudaSuccess;
  const uint32_t blk = 256;
  const uint64_t grid = (n_edges + blk - 1) / blk;
  count_samples_kernel<<<(unsigned)grid, blk, 0, s>>>(qa, qb, n_edges, L, step, counts, bad);
  return cudaGetLastError();
}

cudaError_t launch_build_records(const BuildParams& p, int num_sms, cudaStream_t s) {
  if (p.n_edges == 0) return cudaSuccess;
  const uint32_t blk = 256;
  uint64_t want = (p.n_edges * 32 + blk - 1) / blk;
  uint64_t cap = (uint64_t)num_sms * 16;
  build_records_kernel<<<(unsigned)(want < cap ? want : cap), blk, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tile_edge(const uint64_t* soff, uint64_t n_edges, uint32_t L, uint32_t S,
                             uint64_t n_tiles, uint32_t* out, cudaStream_t s) {
  const uint32_t blk = 256;
  const uint64_t grid = (n_tiles + 1 + blk - 1) / blk;
  tile_edge_kernel<<<(unsigned)grid, blk, 0, s>>>(soff, n_edges, L, S, n_tiles, out);
  return cudaGetLastError();
}

cudaError_t launch_box_update(const BoxUpdateParams& p, cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;
  box_update_kernel<<<(p.n + 127) / 128, 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_box_prep(const BoxPrepParams& p, cudaStream_t s) {
  if (p.njobs == 0) return cudaSuccess;
  box_prep_kernel<<<p.njobs, kBoxesPerPass, 0, s>>>(p);
  return cudaGetLastError();
}

template <int MAXJ>
static cudaError_t launch_classify_t(const ClassifyParams<MAXJ>& p, const ClassifyLaunch& lc,
                                     cudaStream_t s) {
  auto kern = classify_kernel<MAXJ, kNumStages, kStageBytes>;
  const size_t smem = classify_smem_bytes(lc.tw_cap, lc.acc_cap);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<lc.grid, 32 * (1 + lc.consumer_warps), smem, s>>>(p, lc.tw_cap, lc.acc_cap);
  return cudaGetLastError();
}

size_t classify_smem_bytes(uint32_t tw_cap, uint32_t acc_cap) {
  return (size_t)kNumStages * kStageBytes + 2 * kNumStages * sizeof(uint64_t) + 16 +
         4 * (size_t)tw_cap + 8 * (size_t)acc_cap;
}

cudaError_t launch_classify_single(const ClassifyParams<1>& p, const ClassifyLaunch& lc,
                                   cudaStream_t s) {
  return launch_classify_t<1>(p, lc, s);
}

cudaError_t launch_classify_batched(const ClassifyParams<kMaxJobs>& p, const ClassifyLaunch& lc,
                                    cudaStream_t s) {
  return launch_classify_t<kMaxJobs>(p, lc, s);
}

}  // namespace rgg
