// CUDA kernels of the RGG edge-classification pass (sm_103a).
//
//   count_samples_kernel   a0: configurations per edge (Sec. 3.2)
//   build_records_kernel   a0: FP64 kinematics -> FP32 inner/outer spheres
//                          (Sec. 4.2 inner spheres; swept outer spheres)
//   box_update_kernel      a1: write moved boxes' poses in place (Sec. 4.3,
//                          "Online updates")
//   box_prep_kernel        a1: derived per-pass box records
//   round_bounds_kernel    per-round bounding spheres of the outer records
//                          (when tiles are set)
//   round_filter_kernel    spatial filter of a pass: rounds the moved boxes
//                          may reach (Sec. 4.3, spatially filtered checking)
//   classify_kernel        a2..a5: persistent streaming classification
//                          (Sec. 4.1 labelling rule)
//   merge_kernel           a6: per-edge box sets and labels (Algorithm 1)
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
  float* ir = p.joints ? nullptr : p.inner + 3 * p.in_stride;
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
          if (p.joints) {
            // link-end records: the far end of link i at q_k
            const uint64_t g = (uint64_t)L * so + (uint64_t)i * n + k;
            ix[g] = (float)on[0];
            iy[g] = (float)on[1];
            iz[g] = (float)on[2];
          } else {
            const float rad = __double2float_rd(p.radius[i]);
            const uint64_t base = in_base + (uint64_t)K * ((uint64_t)i * n + k);
            for (uint32_t j = 0; j < K; ++j) {
              const double f = ((double)j + 0.5) / (double)K;
              ix[base + j] = (float)(o[0] + f * (on[0] - o[0]));
              iy[base + j] = (float)(o[1] + f * (on[1] - o[1]));
              iz[base + j] = (float)(o[2] + f * (on[2] - o[2]));
              ir[base + j] = rad;
            }
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
// a1: obstacle update and per-pass box records
// ===========================================================================
__global__ void box_update_kernel(const __grid_constant__ BoxUpdateParams p) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  float* srow = p.stage + 16 * (size_t)p.rows[i];
  if (p.from_table) {
    const float* src = p.table + 16 * (size_t)p.ids[i];
    for (int c = 0; c < 16; ++c) srow[c] = src[c];
    return;
  }
  const float* src = p.dev_pose ? p.dev_pose + 15 * (size_t)i : p.pose[i];
  float* dst = p.table + 16 * (size_t)p.ids[i];
  for (int c = 0; c < 15; ++c) {
    dst[c] = src[c];
    srow[c] = src[c];
  }
  dst[15] = 0.0f;
  srow[15] = 0.0f;
}

// Derived records (see rgg_device.cuh) from the box table, in FP64 then
// rounded: axis_k = column k of R, u_k = axis_k . centre, bounding radius
// |h| rounded up.
__global__ void box_prep_kernel(const __grid_constant__ BoxPrepParams p) {
  const BoxPrepJob& J = p.job[blockIdx.x];
  const uint32_t b = threadIdx.x;
  if (b == 0 && J.tcount) *J.tcount = 0u;
  if (b >= J.C) return;
  const uint32_t id = J.ids[b];
  const float* row = J.stage + 16 * (size_t)J.rows[b];
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
// a2..a5: persistent streaming classification
// ===========================================================================
// One CTA per SM, every warp a worker.  A CTA's shared memory holds an
// NSTAGE-deep ring of stages; each stage holds one tile: its edge table and
// its record planes, brought in by TMA bulk copies that complete on the
// stage's `full` mbarriers.  Warps take work items (RPI rounds of 31
// configurations of a tile) from a shared counter, with no CTA-wide barrier:
// a round tests its outer spheres against the pass's moved boxes (a3) and
// the inner spheres against the boxes their enclosing outer spheres touched
// (a4), into per-stage accumulators.  The warp that finishes a tile's last
// item ORs the tile's per-edge hit / touch bits into the global per-edge
// accumulators (a5) and refills the stage with the CTA's next tile.  The
// merge kernel then updates the per-edge box sets and labels (a6).  The
// FILTER instance serves the spatial filter: its ring takes only the tiles
// the filter kernel listed, and it copies and tests only the rounds some
// moved box may reach, against those boxes.
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

// a4 for regular records: does one of the K inner spheres of a sample (first
// centre at s0 of the tile-local planes, common radius r - margin = rr > 0)
// lie within rr of box B?  The centres are c_0 + j (c_{K-1} - c_0) / (K-1),
// so in the box frame only c_0 and c_{K-1} are transformed and the rest are
// interpolated.  A sample whose centres' box-frame bounding box is farther
// than rr from the box is rejected first.
__device__ __forceinline__ bool inner_hit_regular(const float* __restrict__ ix,
                                                  const float* __restrict__ iy,
                                                  const float* __restrict__ iz, int s0, int K,
                                                  float inv_km1, float rr,
                                                  const float4* __restrict__ B) {
  const float4 a0 = B[1], a1 = B[2], a2 = B[3], h = B[4];
  const int s1 = s0 + K - 1;
  const float x0 = ix[s0], y0 = iy[s0], z0 = iz[s0];
  const float x1 = ix[s1], y1 = iy[s1], z1 = iz[s1];
  const float p0 = fmaf(a0.x, x0, fmaf(a0.y, y0, fmaf(a0.z, z0, -a0.w)));
  const float p1 = fmaf(a1.x, x0, fmaf(a1.y, y0, fmaf(a1.z, z0, -a1.w)));
  const float p2 = fmaf(a2.x, x0, fmaf(a2.y, y0, fmaf(a2.z, z0, -a2.w)));
  const float q0 = fmaf(a0.x, x1, fmaf(a0.y, y1, fmaf(a0.z, z1, -a0.w)));
  const float q1 = fmaf(a1.x, x1, fmaf(a1.y, y1, fmaf(a1.z, z1, -a1.w)));
  const float q2 = fmaf(a2.x, x1, fmaf(a2.y, y1, fmaf(a2.z, z1, -a2.w)));
  const float rr2 = rr * rr;
  const float g0 = fmaxf(fmaxf(fminf(p0, q0) - h.x, -h.x - fmaxf(p0, q0)), 0.0f);
  const float g1 = fmaxf(fmaxf(fminf(p1, q1) - h.y, -h.y - fmaxf(p1, q1)), 0.0f);
  const float g2 = fmaxf(fmaxf(fminf(p2, q2) - h.z, -h.z - fmaxf(p2, q2)), 0.0f);
  if (fmaf(g0, g0, fmaf(g1, g1, g2 * g2)) > rr2) return false;
  const float d0 = (q0 - p0) * inv_km1, d1 = (q1 - p1) * inv_km1, d2 = (q2 - p2) * inv_km1;
  for (int j = 0; j < K; ++j) {
    const float t = (float)j;
    const float e0 = fmaxf(fabsf(fmaf(t, d0, p0)) - h.x, 0.0f);
    const float e1 = fmaxf(fabsf(fmaf(t, d1, p1)) - h.y, 0.0f);
    const float e2 = fmaxf(fabsf(fmaf(t, d2, p2)) - h.z, 0.0f);
    if (fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) <= rr2) return true;
  }
  return false;
}

// a4 for link-end records: does one of the K inner spheres of a link at one
// configuration (centres at fractions (j + 1/2)/K of the segment from its near
// end a to its far end b, common radius R_i - margin = rr > 0) lie within rr
// of box B?  Both ends are transformed into the box frame once and the
// centres interpolated there; a link whose spheres' box-frame bounding box
// is farther than rr from the box is rejected first.
__device__ __forceinline__ bool inner_hit_joints(float ax, float ay, float az, float bx, float by,
                                                 float bz, int K, float inv_k, float rr,
                                                 const float4* __restrict__ B) {
  const float4 a0 = B[1], a1 = B[2], a2 = B[3], h = B[4];
  const float p0 = fmaf(a0.x, ax, fmaf(a0.y, ay, fmaf(a0.z, az, -a0.w)));
  const float p1 = fmaf(a1.x, ax, fmaf(a1.y, ay, fmaf(a1.z, az, -a1.w)));
  const float p2 = fmaf(a2.x, ax, fmaf(a2.y, ay, fmaf(a2.z, az, -a2.w)));
  const float q0 = fmaf(a0.x, bx, fmaf(a0.y, by, fmaf(a0.z, bz, -a0.w)));
  const float q1 = fmaf(a1.x, bx, fmaf(a1.y, by, fmaf(a1.z, bz, -a1.w)));
  const float q2 = fmaf(a2.x, bx, fmaf(a2.y, by, fmaf(a2.z, bz, -a2.w)));
  // step between consecutive centres, and the first and the last centre
  const float d0 = (q0 - p0) * inv_k, d1 = (q1 - p1) * inv_k, d2 = (q2 - p2) * inv_k;
  const float tl = (float)K - 0.5f;
  const float f0 = fmaf(0.5f, d0, p0), f1 = fmaf(0.5f, d1, p1), f2 = fmaf(0.5f, d2, p2);
  const float l0 = fmaf(tl, d0, p0), l1 = fmaf(tl, d1, p1), l2 = fmaf(tl, d2, p2);
  const float rr2 = rr * rr;
  const float g0 = fmaxf(fmaxf(fminf(f0, l0) - h.x, -h.x - fmaxf(f0, l0)), 0.0f);
  const float g1 = fmaxf(fmaxf(fminf(f1, l1) - h.y, -h.y - fmaxf(f1, l1)), 0.0f);
  const float g2 = fmaxf(fmaxf(fminf(f2, l2) - h.z, -h.z - fmaxf(f2, l2)), 0.0f);
  if (fmaf(g0, g0, fmaf(g1, g1, g2 * g2)) > rr2) return false;
  for (int j = 0; j < K; ++j) {
    const float t = (float)j + 0.5f;
    const float e0 = fmaxf(fabsf(fmaf(t, d0, p0)) - h.x, 0.0f);
    const float e1 = fmaxf(fabsf(fmaf(t, d1, p1)) - h.y, 0.0f);
    const float e2 = fmaxf(fabsf(fmaf(t, d2, p2)) - h.z, 0.0f);
    if (fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) <= rr2) return true;
  }
  return false;
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

// Where local sample q of a tile sits: its edge-table entry j, the edge's
// configuration count n, its link li and position k in that link's run, and
// the local index o of the interval that follows it (branch-free).  `valid`: q is one
// of the tile's samples [0, q_end); `has_next`: an interval follows it.
struct SampleAt {
  int j, n, k, o, li;
  bool valid, has_next;
};
__device__ __forceinline__ SampleAt locate_sample(const int* etab, int n_edges, int q, int q_end) {
  SampleAt a;
  a.j = search_le(etab, 0, n_edges, max(q, 0));
  const int4 ej = *reinterpret_cast<const int4*>(etab + 4 * a.j);
  a.n = ej.y;
  const int rr = q - ej.x;
  int li = __float2int_rz(((float)rr + 0.5f) * __int_as_float(ej.w));
  int k = rr - li * a.n;
  const int adj = k < 0 ? -1 : (k >= a.n ? 1 : 0);  // exact rr / n
  li += adj;
  k -= adj * a.n;
  a.k = k;
  a.li = li;
  a.valid = q < q_end && rr >= 0;
  a.has_next = a.valid && k < a.n - 1;
  a.o = a.has_next ? ej.z + li * (a.n - 1) + k : 0;
  return a;
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

// ---------------------------------------------------------------------------
// Spatial filter (Sec. 4.3): per-round bounding spheres, and the per-pass test
// ---------------------------------------------------------------------------
// Radius of the sphere about (cx, cy, cz) that holds every active lane's
// sphere, from the FP32 records in FP32.  Each step is one correctly rounded
// operation (the differences, then sums of non-negative terms and a square
// root), so the computed radius is within 8 * 2^-24 of the exact one,
// relatively; enlarged by 2e-6 relative and rounded up it is an upper bound.
__device__ __forceinline__ float cover_radius(float x, float y, float z, float r, bool on,
                                              float cx, float cy, float cz) {
  const float dx = x - cx, dy = y - cy, dz = z - cz;
  const float v = on ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + r : 0.0f;
  const float m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
  return __fmul_ru(m, 1.000002f);
}

// One warp per tile.  Round r's outer spheres are those of the intervals the
// classify kernel's consumer tests in that round (the same lane mapping).
// The centre starts at the midpoint of the first and the last sphere centre
// and takes 24 steps of the Badoiu-Clarkson iteration (a step of 1/(i+1)
// towards the sphere that reaches farthest), which approaches the centre of
// the smallest enclosing sphere; the smaller of the two radii is kept.
__global__ void __launch_bounds__(256) round_bounds_kernel(const __grid_constant__ RoundBoundsParams p) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < p.T; t += nw) {
    const TileDesc d = p.tiles[t];
    const uint64_t o0 = d.packed & ((1ull << 40) - 1);
    const int n_edges = (int)(d.packed >> 56);
    const int* etab = reinterpret_cast<const int*>(p.etab + d.etab);
    const uint64_t g0 = t * p.S;
    const int n_samp = (int)(min(g0 + p.S, p.G) - g0);
    float4 mine = make_float4(0.0f, 0.0f, 0.0f, -1.0f);  // lane r: round r's sphere
    for (int rnd = 0; rnd < kRoundSlots; ++rnd) {
      const int base = 31 * rnd;
      float4 sph = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
      uint32_t range = 0;
      if (base < n_samp) {
        const SampleAt a = locate_sample(etab, n_edges, base - 1 + lane, min(base + 31, n_samp));
        float x = 0.0f, y = 0.0f, z = 0.0f, r = 0.0f;
        if (a.has_next) {
          const float* o = p.outer + o0 + a.o;
          x = o[0];
          y = o[p.out_stride];
          z = o[2 * p.out_stride];
          r = o[3 * p.out_stride];
        }
        const uint32_t act = __ballot_sync(0xffffffffu, a.has_next);
        if (act) {
          const int lo_l = __ffs(act) - 1, hi_l = 31 - __clz(act);
          const float mx = 0.5f * (__shfl_sync(0xffffffffu, x, lo_l) + __shfl_sync(0xffffffffu, x, hi_l));
          const float my = 0.5f * (__shfl_sync(0xffffffffu, y, lo_l) + __shfl_sync(0xffffffffu, y, hi_l));
          const float mz = 0.5f * (__shfl_sync(0xffffffffu, z, lo_l) + __shfl_sync(0xffffffffu, z, hi_l));
          float cx = mx, cy = my, cz = mz;
          for (int it = 1; it <= 24; ++it) {
            const float dx = x - cx, dy = y - cy, dz = z - cz;
            const float f = a.has_next ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + r : 0.0f;
            const float fm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(f)));
            const int w0 = __ffs(__ballot_sync(0xffffffffu, a.has_next && f == fm)) - 1;
            const int w = w0 < 0 ? lo_l : w0;
            const float step = 1.0f / (float)(it + 1);
            cx = fmaf(__shfl_sync(0xffffffffu, x, w) - cx, step, cx);
            cy = fmaf(__shfl_sync(0xffffffffu, y, w) - cy, step, cy);
            cz = fmaf(__shfl_sync(0xffffffffu, z, w) - cz, step, cz);
          }
          const float r_mid = cover_radius(x, y, z, r, a.has_next, mx, my, mz);
          const float r_bc = cover_radius(x, y, z, r, a.has_next, cx, cy, cz);
          sph = r_bc < r_mid ? make_float4(cx, cy, cz, r_bc) : make_float4(mx, my, mz, r_mid);
          const uint32_t lo = (uint32_t)__shfl_sync(0xffffffffu, a.o, lo_l);
          const uint32_t hi = (uint32_t)__shfl_sync(0xffffffffu, a.o, hi_l) + 1u;
          range = lo | (hi << 16);
        }
      }
      if (lane == 0) {
        p.rsph[t * kRoundSlots + rnd] = sph;
        p.rout[t * kRoundSlots + rnd] = range;
      }
      if (lane == rnd) mine = sph;
    }
    // the tile's sphere: about the midpoint of its first and last live round
    // centres, holding every round sphere (the radius bound as in
    // cover_radius; the round radii are upper bounds already)
    const bool on = mine.w >= 0.0f;
    const uint32_t live = __ballot_sync(0xffffffffu, on);
    float4 ts = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    if (live) {
      const int lo = __ffs(live) - 1, hi = 31 - __clz(live);
      const float cx = 0.5f * (__shfl_sync(0xffffffffu, mine.x, lo) + __shfl_sync(0xffffffffu, mine.x, hi));
      const float cy = 0.5f * (__shfl_sync(0xffffffffu, mine.y, lo) + __shfl_sync(0xffffffffu, mine.y, hi));
      const float cz = 0.5f * (__shfl_sync(0xffffffffu, mine.z, lo) + __shfl_sync(0xffffffffu, mine.z, hi));
      ts = make_float4(cx, cy, cz, cover_radius(mine.x, mine.y, mine.z, mine.w, on, cx, cy, cz));
    }
    if (lane == 0) p.tsph[t] = ts;
  }
}

// Tiles per warp of the filter kernel (at most 32: lane i holds tile i's
// sphere and list flag).  Fewer tiles per warp give more, shorter blocks, so
// the launch's last wave of blocks is a smaller part of it.
constexpr int kFilterTilesPerWarp = 16;
static_assert(kFilterTilesPerWarp >= 1 && kFilterTilesPerWarp <= 32, "filter tiles per warp");

// Before a pass: per (tile, round), the moved boxes whose exact distance
// from the round's bounding sphere centre is within its radius plus the
// margin.  Any outer sphere of the round lies inside the bounding sphere, so
// a box that touches one of them (distance <= r + margin) passes this test;
// the slack covers FP32 rounding in both tests.  One warp per
// kFilterTilesPerWarp consecutive tiles, taken one after the other, one lane
// per round.  The warp stages its
// roadmap's box records in shared memory (again when the roadmap changes).
// A sphere about the tile's round spheres is tested against all boxes first;
// only the boxes it may reach are tested per round, and there a box whose
// bounding sphere is out of reach skips the exact distance.
// The tiles with a round to test are appended to their roadmap's tile list,
// one atomic per roadmap and warp; the list's order is arbitrary.
template <int MAXJ>
__global__ void __launch_bounds__(256) round_filter_kernel(const __grid_constant__ ClassifyParams<MAXJ> P) {
  __shared__ float4 s_bx[8][kBoxesPerPass * 6];
  const int lane = threadIdx.x & 31;
  const uint64_t t0 =
      (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (uint64_t)kFilterTilesPerWarp;
  if (t0 >= P.total_tiles) return;  // whole warps: t0 is the same on every lane
  float4* bx = s_bx[threadIdx.x >> 5];
  const int nt = (int)min((uint64_t)kFilterTilesPerWarp, P.total_tiles - t0);
  int staged = -1;
  bool listed = false;  // lane i: tile t0 + i goes on its roadmap's list
  // lane i: the sphere about tile t0 + i's rounds (radius < 0: none)
  float4 tile_s = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
  if (lane < nt) {
    const ClassifyJob& Jl = P.job[MAXJ == 1 ? 0 : find_job(P, t0 + (uint64_t)lane)];
    if (Jl.rcand) tile_s = Jl.tsph[t0 + (uint64_t)lane - Jl.tile_base];
  }
  for (int i = 0; i < nt; ++i) {
    const uint64_t t = t0 + (uint64_t)i;
    const int jb = MAXJ == 1 ? 0 : find_job(P, t);
    const ClassifyJob& J = P.job[jb];
    if (J.rcand == nullptr) continue;
    const int C = (int)J.C;
    if (jb != staged) {
      __syncwarp();
      if (lane < C)
        for (int c = 0; c < 6; ++c) bx[6 * lane + c] = reinterpret_cast<const float4*>(J.boxes)[6 * lane + c];
      __syncwarp();
      staged = jb;
    }
    // first the tile: its sphere against every box at once (lane b: box
    // b).  A tile no box may reach is done: its rounds are not loaded and
    // its candidate row is not written (the classify kernel reads the rows
    // of listed tiles only)
    const float ts_x = __shfl_sync(0xffffffffu, tile_s.x, i);
    const float ts_y = __shfl_sync(0xffffffffu, tile_s.y, i);
    const float ts_z = __shfl_sync(0xffffffffu, tile_s.z, i);
    const float ts_r = __shfl_sync(0xffffffffu, tile_s.w, i);
    if (ts_r < 0.0f) continue;
    bool cb = false;
    if (lane < C) {
      const float4 b0 = bx[6 * lane];
      const float ex = b0.x - ts_x, ey = b0.y - ts_y, ez = b0.z - ts_z;
      const float thr = (ts_r + b0.w + J.margin) * (1.0f + 1e-5f) + 1e-5f;
      cb = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= thr * thr;
    }
    const uint32_t tile_cand = __ballot_sync(0xffffffffu, cb);
    if (tile_cand == 0u) continue;
    // then the rounds, against the boxes the tile's sphere may reach
    const uint64_t slot = (t - J.tile_base) * kRoundSlots + lane;
    const float4 sph = lane < kRoundSlots - 1 ? J.rsph[slot] : make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    const bool on = sph.w >= 0.0f;
    uint32_t m = 0;
    if (on) {
      const float thr = (sph.w + J.margin) * (1.0f + 1e-6f) + 1e-5f;
      const float thr2 = thr * thr;
      for (uint32_t mm = tile_cand; mm; mm &= mm - 1) {
        const int b = __ffs(mm) - 1;
        const float4 b0 = bx[6 * b];
        const float ex = sph.x - b0.x, ey = sph.y - b0.y, ez = sph.z - b0.z;
        const float reach = thr + b0.w;  // the box lies in the sphere of radius |h|
        if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > reach * reach * (1.0f + 1e-6f)) continue;
        if (box_dist2(sph.x, sph.y, sph.z, bx + 6 * b) <= thr2) m |= 1u << b;
      }
    }
    // the last slot (never a round: tiles have at most 31 rounds) holds the
    // tile's rounds that some box may reach
    const uint32_t need = __ballot_sync(0xffffffffu, m != 0u);
    J.rcand[slot] = lane == kRoundSlots - 1 ? need : m;
    if (lane == i && need != 0u && J.tlist != nullptr) listed = true;
  }
  // the listed tiles, grouped by roadmap: one atomic per group
  const int jl = (listed && MAXJ != 1) ? find_job(P, t0 + (uint64_t)lane) : 0;
  const uint32_t peers = __match_any_sync(0xffffffffu, listed ? jl : -1);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (listed && lane == leader) base = atomicAdd(P.job[jl].tcount, (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (listed) {
    // bounded by the list's size whatever the count holds
    const ClassifyJob& J = P.job[jl];
    const uint32_t at = base + __popc(peers & ((1u << lane) - 1u));
    if (at < J.num_tiles) J.tlist[at] = (uint32_t)(t0 + (uint64_t)lane - J.tile_base);
  }
}

// Bound of the final wait for the CTA's own bulk copies before it exits
// (copies always land; the bound only keeps the wait finite).
constexpr uint64_t kDrainLimit = 500000000ull;

__device__ __forceinline__ void write_stage_hdr(unsigned char* sb, int job, uint64_t g0, uint64_t g1,
                                                uint32_t n_out, uint32_t n_edges, int in_shift,
                                                int out_shift, uint32_t e_first) {
  StageHdr* h = reinterpret_cast<StageHdr*>(sb);
  h->job = job;
  h->n_samp = (int)(g1 - g0);
  h->n_out = (int)n_out;
  h->n_edges = (int)n_edges;
  h->in_shift = in_shift;
  h->out_shift = out_shift;
  h->e_first = e_first;
  h->end = 0;
}

constexpr int kPairQueue = 64;   // (sample, box) pairs a warp compacts per round

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Full barriers per stage.  Slot m of a CTA completes on barrier m % (B*NSTAGE)
// with phase parity (m / (B*NSTAGE)) & 1.  Slots are refilled out of order (a
// stage is refilled as soon as its own tile is done), so a worker may reach
// slot m while the stage's earlier slots are still unfilled; the parity test
// is unambiguous as long as the barrier's previous use, slot m - B*NSTAGE, is
// filled.  If it were not, the B slots of that stage from m - B*NSTAGE on
// would all be unfilled with every item taken, i.e. B*IPT waiting workers,
// plus one on the slot before them and the one at slot m: so B*IPT + 1 >= the
// launch's warps keeps every wait exact.
constexpr int kMaxWorkers = kMaxClassifyThreads / 32;
__host__ __device__ constexpr int full_barriers_per_stage(int ipt) { return ipt >= kMaxWorkers - 1 ? 1 : (kMaxWorkers - 2) / ipt + 1; }

// What a slot's fill needs to know of its tile: the job, the local tile, its
// descriptor and halo count, and with the spatial filter the tile's round
// mask and (per lane) the outer range of round `lane`.  Loading it takes a
// chain of dependent global loads (the list entry, then the tile's own
// rows), so each fill also loads the metadata of the stage's next slot and
// leaves it in shared memory for the warp that will fill that slot.
struct SlotMeta {
  int jb;
  uint32_t lt;
  TileDesc d;
  uint32_t halo, need, ro;
  int end;
};
constexpr int kMetaWords = 48;  // per stage: 16 header words, then ro of the 32 lanes

template <int MAXJ, bool FILTER>
__device__ __forceinline__ SlotMeta slot_meta(const ClassifyParams<MAXJ>& P, uint32_t slot,
                                              const uint32_t* s_pref, int lane) {
  SlotMeta m{};
  const uint64_t t = blockIdx.x + (uint64_t)slot * gridDim.x;
  const uint32_t nj = MAXJ == 1 ? 1u : min(P.njobs, (uint32_t)MAXJ);
  if (t >= s_pref[nj]) {
    m.end = 1;
    return m;
  }
  // the job whose range of the launch's tiles holds t (the last with
  // s_pref[jb] <= t; jobs without tiles have empty ranges)
  int jb = 0;
  if (MAXJ != 1) {
    int hi = (int)nj - 1;
    while (jb < hi) {
      const int mid = (jb + hi + 1) >> 1;
      if (s_pref[mid] <= t) jb = mid; else hi = mid - 1;
    }
  }
  const ClassifyJob& J = P.job[jb];
  const uint64_t u = t - s_pref[jb];
  // a listed job's slots take its listed tiles (entries are below num_tiles;
  // the bound only keeps a stale entry inside the tile table)
  const uint64_t lt = (FILTER && J.tlist) ? min((uint64_t)J.tlist[u], J.num_tiles - 1) : u;
  m.jb = jb;
  m.lt = (uint32_t)lt;
  m.d = J.tiles[lt];
  m.halo = J.joints ? J.tile_halo[lt] : 0u;
  m.need = ~0u;
  if constexpr (FILTER) {
    if (J.rcand) {
      m.need = J.rcand[lt * kRoundSlots + kRoundSlots - 1];
      m.ro = J.rout[lt * kRoundSlots + lane];
    }
  }
  return m;
}

template <int NSTAGE>
__device__ __forceinline__ void store_meta(uint32_t* s_meta, uint32_t* s_meta_slot, int stage,
                                           uint32_t slot, const SlotMeta& m, int lane) {
  uint32_t* w = s_meta + stage * kMetaWords;
  if (lane == 0) {
    w[0] = (uint32_t)m.jb;
    w[1] = m.lt;
    w[2] = (uint32_t)m.d.packed;
    w[3] = (uint32_t)(m.d.packed >> 32);
    w[4] = m.d.etab;
    w[5] = m.d.e_first;
    w[6] = m.halo;
    w[7] = m.need;
    w[8] = (uint32_t)m.end;
  }
  w[16 + lane] = m.ro;
  __syncwarp();
  if (lane == 0) {
    __threadfence_block();
    *reinterpret_cast<volatile uint32_t*>(&s_meta_slot[stage]) = slot;
  }
}

// The metadata the stage's previous fill left for `slot` (false if it did
// not arrive within the wait limit).
__device__ __forceinline__ bool take_meta(const uint32_t* s_meta, const uint32_t* s_meta_slot,
                                          int stage, uint32_t slot, uint64_t limit_ns,
                                          SlotMeta& m, int lane) {
  int ok = 1;
  if (lane == 0) {
    const volatile uint32_t* f = &s_meta_slot[stage];
    if (*f != slot) {
      const uint64_t t0 = global_ns();
      while (*f != slot)
        if (global_ns() - t0 > limit_ns) {
          ok = 0;
          break;
        }
    }
    __threadfence_block();
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return false;
  const volatile uint32_t* w = s_meta + stage * kMetaWords;
  m.jb = (int)w[0];
  m.lt = w[1];
  m.d.packed = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
  m.d.etab = w[4];
  m.d.e_first = w[5];
  m.halo = w[6];
  m.need = w[7];
  m.end = (int)w[8];
  m.ro = w[16 + lane];
  return true;
}

// Fill ring slot `slot` of this CTA (stage slot % NSTAGE) with its tile,
// blockIdx.x + slot * gridDim.x of the launch's tiles (metadata `m`), or with
// an end marker once past the last tile.  The slot's tile is fixed by its
// number, so every worker sees the tiles in slot order and every end marker
// after the last tile.  Called by one whole warp: lanes derive the copies,
// lane 0 writes the header and arms the stage's barrier, and the lanes issue
// the bulk copies together.
template <int MAXJ, int NSTAGE, int STAGE_BYTES, int NBAR, bool FILTER>
__device__ __forceinline__ void fill_slot(const ClassifyParams<MAXJ>& P, uint32_t slot,
                                          const SlotMeta& m, unsigned char* stages,
                                          uint64_t* full_bars, int* s_sjob, uint32_t* s_last,
                                          uint32_t* s_cand, float4* s_boxes, int lane) {
  const int stage = (int)(slot % NSTAGE);
  uint64_t* bar = &full_bars[slot % NBAR];
  unsigned char* sb = stages + (size_t)stage * STAGE_BYTES;
  if (m.end) {
    if (lane == 0) {
      reinterpret_cast<StageHdr*>(sb)->end = 1;
      s_last[stage] = slot;
      mbar_arrive(bar);
    }
    __syncwarp();
    return;
  }
  const int jb = m.jb;
  const ClassifyJob& J = P.job[jb];
  const uint64_t lt = m.lt;
  const TileDesc d = m.d;
  const uint32_t halo = m.halo;
  const uint32_t need = m.need, ro = m.ro;
  const uint64_t K = J.K;
  const uint64_t g0 = lt * J.S;
  const uint64_t g1 = min(g0 + J.S, J.G);
  // inner window: the tile's K spheres per sample, or its link ends and the
  // h_t ends before it that hold its first samples' near ends
  const bool jt = J.joints != 0;
  const uint64_t w0 = jt ? g0 - halo : K * g0;
  const uint64_t a0 = w0 & ~3ull, a1 = ((jt ? g1 : K * g1) + 3) & ~3ull;
  const int in_shift = (int)((jt ? g0 : K * g0) - a0);
  const uint32_t n_in = jt ? 3u : 4u;
  const uint64_t o0 = d.packed & ((1ull << 40) - 1);
  const uint32_t n_out = (uint32_t)((d.packed >> 40) & 0xffff);
  const uint32_t n_edges = (uint32_t)(d.packed >> 56);
  const uint64_t b0 = o0 & ~3ull, b1 = (o0 + n_out + 3) & ~3ull;
  const uint32_t et_bytes = n_edges * 16;
  const uint32_t in_bytes = (uint32_t)((a1 - a0) * 4);
  const uint32_t out_bytes = (uint32_t)((b1 - b0) * 4);
  if (FILTER && need == 0u) {
    // the spatial filter found no moved box near the tile: no data, no
    // rounds (the workers take its items and find nothing to do)
    if (lane == 0) {
      write_stage_hdr(sb, jb, g0, g0, 0, 0, 0, 0, d.e_first);
      s_last[stage] = slot;
      mbar_arrive(bar);
    }
    __syncwarp();
    return;
  }
  // the stage's box records are refreshed only when its roadmap changes
  const int held = s_sjob[stage];
  const uint32_t box_bytes = (MAXJ != 1 && held != jb) ? (uint32_t)(kBoxAreaFloats * 4) : 0u;
  __syncwarp();
  uint32_t tile_rec_bytes = 0;  // record bytes this tile's copies move
  if (!FILTER || J.rcand == nullptr) {
    // whole-tile copies: lane 0 the edge table, lanes 1..4 the inner planes
    // (1..3 the link-end planes), 5..8 the outer ones, lane 9 the box area;
    // one predicated issue
    void* c_dst = sb + kStageEtabOff;
    const void* c_src = J.etab + d.etab;
    uint32_t c_bytes = et_bytes;
    if (lane >= 1 && lane <= 4) {
      c_dst = sb + J.off_in + (size_t)(lane - 1) * J.in_cap * 4;
      c_src = J.inner + (lane - 1) * J.in_stride + a0;
      c_bytes = (uint32_t)(lane - 1) < n_in ? in_bytes : 0u;
    } else if (lane >= 5 && lane <= 8) {
      c_dst = sb + J.off_out + (size_t)(lane - 5) * J.out_cap * 4;
      c_src = J.outer + (lane - 5) * J.out_stride + b0;
      c_bytes = out_bytes;
    } else if (lane == 9) {
      c_dst = s_boxes + (size_t)stage * (kBoxAreaFloats / 4);
      c_src = J.boxes;
      c_bytes = box_bytes;
    } else if (lane > 9) {
      c_bytes = 0;
    }
    if (lane == 0) {
      write_stage_hdr(sb, jb, g0, g1, n_out, n_edges, in_shift, (int)(o0 - b0), d.e_first);
      mbar_arrive_expect_tx(bar, et_bytes + n_in * in_bytes + 4 * out_bytes + box_bytes);
      s_sjob[stage] = jb;
      s_last[stage] = slot;
    }
    tile_rec_bytes = n_in * in_bytes + 4 * out_bytes;
    __syncwarp();
    fence_proxy_async_smem();
    if (c_bytes) bulk_g2s(c_dst, c_src, c_bytes, bar);
  } else if constexpr (FILTER) {
    // the runs of consecutive rounds in `need`: the lane of a run's first
    // round copies the run's 4 inner and 4 outer plane pieces, at the offsets
    // they have in a whole-tile copy (link-end planes, 12 B per sample, are
    // copied whole by lanes 1..3, since a run's near ends may lie in rounds
    // the run does not cover); lane 10 copies the tile's candidate row
    const bool starts = ((need >> lane) & 1u) && (lane == 0 || !((need >> (lane - 1)) & 1u));
    const uint32_t clear_above = ~need & ~((2u << lane) - 1u);
    const int re = clear_above ? __ffs(clear_above) - 1 : 32;  // run = rounds [lane, re)
    const uint32_t ro_last = __shfl_sync(0xffffffffu, ro, starts ? re - 1 : lane);
    uint64_t ia = a0, ib = a0, oa = b0, ob = b0;
    if (starts) {
      if (!jt) {
        ia = (K * (g0 + (uint64_t)(31 * lane))) & ~3ull;
        ib = (K * min(g0 + (uint64_t)(31 * re), g1) + 3) & ~3ull;
      }
      oa = (o0 + (ro & 0xffffu)) & ~3ull;
      ob = (o0 + (ro_last >> 16) + 3) & ~3ull;
    }
    // never outside the whole-tile window, whatever the round data say
    ia = max(ia, a0);
    ib = max(min(ib, a1), ia);
    oa = max(oa, b0);
    ob = max(min(ob, b1), oa);
    const uint32_t run_in = (uint32_t)((ib - ia) * 4);
    const uint32_t run_out = (uint32_t)((ob - oa) * 4);
    const uint32_t tile_bytes = __reduce_add_sync(0xffffffffu, 4 * (run_in + run_out)) +
                                (jt ? 3 * in_bytes : 0u);
    if (lane == 0) {
      write_stage_hdr(sb, jb, g0, g1, n_out, n_edges, in_shift, (int)(o0 - b0), d.e_first);
      mbar_arrive_expect_tx(bar, et_bytes + tile_bytes + box_bytes + 4 * kRoundSlots);
      s_sjob[stage] = jb;
      s_last[stage] = slot;
    }
    tile_rec_bytes = tile_bytes;
    __syncwarp();
    fence_proxy_async_smem();
    if (lane == 0) bulk_g2s(sb + kStageEtabOff, J.etab + d.etab, et_bytes, bar);
    if (lane == 9 && box_bytes)
      bulk_g2s(s_boxes + (size_t)stage * (kBoxAreaFloats / 4), J.boxes, box_bytes, bar);
    if (jt && lane >= 1 && lane <= 3)
      bulk_g2s(sb + J.off_in + (size_t)(lane - 1) * J.in_cap * 4,
               J.inner + (lane - 1) * J.in_stride + a0, in_bytes, bar);
    if (lane == 10)
      bulk_g2s(s_cand + stage * kRoundSlots, J.rcand + lt * kRoundSlots, 4 * kRoundSlots,
               bar);
    if (run_in)
      for (int pl = 0; pl < 4; ++pl)
        bulk_g2s(sb + J.off_in + ((size_t)pl * J.in_cap + (ia - a0)) * 4,
                 J.inner + pl * J.in_stride + ia, run_in, bar);
    if (run_out)
      for (int pl = 0; pl < 4; ++pl)
        bulk_g2s(sb + J.off_out + ((size_t)pl * J.out_cap + (oa - b0)) * 4,
                 J.outer + pl * J.out_stride + oa, run_out, bar);
  }
  // filtered instance: the record bytes this tile copied (the streaming
  // instance copies every record and does not count)
  if (FILTER && lane == 0 && J.streamed) atomicAdd(J.streamed, (unsigned long long)tile_rec_bytes);
  __syncwarp();
}

// Work items: a tile has ROUNDS rounds of 31 samples, grouped RPI rounds per
// work item; warps take items in order from a shared counter.  Slot m of a
// CTA holds the launch's tile blockIdx + m * gridDim (counting, for a job
// with the spatial filter's list, only its listed tiles).
// Round r of a tile covers the samples q = 31r .. 31r+30 on lanes 1..31;
// lane 0 takes sample 31r-1, whose following interval the round needs (for
// r = 0 that is the tile's halo interval).
//
// The ring refills itself.  Every warp is a worker.  The warp that finishes
// a tile's last item flushes the tile's per-edge bits and loads the stage
// with the tile NSTAGE slots ahead, so no warp waits for a free stage and no
// single warp issues every tile's copies.  The first NSTAGE slots are filled
// at the start.
// FILTER: the instance that serves spatially filtered jobs (listed tiles
// only, rounds copied in runs, per-round candidate masks instead of the warp
// cull); without it the jobs' filter fields are ignored and every tile is
// copied whole.
// COUNT: the instance that also counts the work it executes (rounds, outer
// sphere-box tests, inner (sample, box) pairs) into P.work.
template <int MAXJ, int NSTAGE, int STAGE_BYTES, int ROUNDS, int RPI, bool FILTER, bool COUNT = false>
__global__ void __launch_bounds__(kMaxClassifyThreads, 1) classify_kernel(const __grid_constant__ ClassifyParams<MAXJ> P) {
  static_assert(ROUNDS < kRoundSlots, "rounds per tile");
  // Shared-memory carve-up, by integer offsets from the __shared__ base so that
  // every derived pointer stays a shared-memory pointer (plain LDS/STS).
  // Box records: one area staged once for a single-roadmap launch; one per
  // stage, refilled when the stage's roadmap changes, for batched launches.
  constexpr int kBoxAreas = MAXJ == 1 ? 1 : NSTAGE;
  constexpr int IPT = (ROUNDS + RPI - 1) / RPI;  // work items per tile
  constexpr int NBAR = NSTAGE * full_barriers_per_stage(IPT);
  constexpr size_t kOffFull = (size_t)NSTAGE * STAGE_BYTES;
  constexpr size_t kOffBoxBar = kOffFull + NBAR * sizeof(uint64_t);
  constexpr size_t kOffItem = kOffBoxBar + sizeof(uint64_t);
  constexpr size_t kOffCnt = kOffItem + 8;
  constexpr size_t kOffSjob = kOffCnt + 4 * ((NSTAGE + 3) & ~3);
  constexpr size_t kOffLast = kOffSjob + 4 * ((NSTAGE + 3) & ~3);
  constexpr size_t kOffPref = kOffLast + 4 * ((NSTAGE + 3) & ~3);
  constexpr size_t kOffMetaSlot = kOffPref + 4 * (MAXJ + 1);
  constexpr size_t kOffMeta = (kOffMetaSlot + 4 * NSTAGE + 15) & ~(size_t)15;
  constexpr size_t kOffCand = (kOffMeta + 4 * (size_t)NSTAGE * kMetaWords + 15) & ~(size_t)15;
  constexpr size_t kOffBoxes =
      (kOffCand + (FILTER ? (size_t)NSTAGE * kRoundSlots * 4 : 0) + 127) & ~(size_t)127;
  constexpr size_t kOffQueues = kOffBoxes + (size_t)kBoxAreas * kBoxAreaFloats * 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffFull);
  uint64_t* boxbar = reinterpret_cast<uint64_t*>(smem + kOffBoxBar);
  uint32_t* s_item = reinterpret_cast<uint32_t*>(smem + kOffItem);     // next work item
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + kOffCnt);       // items done per stage
  int* s_sjob = reinterpret_cast<int*>(smem + kOffSjob);              // job whose boxes a stage holds
  uint32_t* s_last = reinterpret_cast<uint32_t*>(smem + kOffLast);     // last slot a stage was filled with
  // s_pref[j]: the launch's tiles before job j (the filter's listed tiles
  // for a job with a list); s_pref[njobs] = tiles of the launch
  uint32_t* s_pref = reinterpret_cast<uint32_t*>(smem + kOffPref);
  // per stage: the slot whose metadata the stage's last fill left, and that
  // metadata (see SlotMeta)
  uint32_t* s_meta_slot = reinterpret_cast<uint32_t*>(smem + kOffMetaSlot);
  uint32_t* s_meta = reinterpret_cast<uint32_t*>(smem + kOffMeta);
  // per stage (spatial filter): the moved boxes that may reach each round of
  // its tile, 0 for a round that was not copied
  uint32_t* s_cand = reinterpret_cast<uint32_t*>(smem + kOffCand);
  float4* s_boxes = reinterpret_cast<float4*>(smem + kOffBoxes);
  uint32_t* queues = reinterpret_cast<uint32_t*>(smem + kOffQueues);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;

  // An error latched by an earlier launch (on the launch's word or on one of
  // its roadmaps' own words) stops the launch before it issues anything: its
  // pass is marked skipped, so the merge leaves every per-edge set alone and
  // the host re-queues the boxes when it collects the error.
  {
    int bad = threadIdx.x == 0 ? *reinterpret_cast<volatile const int*>(P.status) : 0;
    for (uint32_t j = threadIdx.x; j < P.njobs && j < (uint32_t)MAXJ; j += blockDim.x)
      if (P.job[j].status) bad |= *reinterpret_cast<volatile const int*>(P.job[j].status);
    if (__syncthreads_or(bad != 0)) {
      if (threadIdx.x == 0) atomicCAS(P.status, 0, (int)kStatusSkipped);
      return;
    }
  }

  // zero the stages (their accumulators must start at zero) and counters
  for (uint32_t i = threadIdx.x; i < NSTAGE * STAGE_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(stages)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = threadIdx.x; i < NSTAGE; i += blockDim.x) {
    s_cnt[i] = 0;
    s_sjob[i] = -1;
    s_last[i] = 0xffffffffu;
    s_meta_slot[i] = 0xffffffffu;
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int b = 0; b < NBAR; ++b) mbar_init(&full[b], 1);
    mbar_init(boxbar, 1);
    *s_item = 0;
    fence_mbar_init();
    if (MAXJ == 1) {
      // the whole box area: the pass's box records and the link radii
      const uint32_t bytes = (uint32_t)(kBoxAreaFloats * 4);
      mbar_arrive_expect_tx(boxbar, bytes);
      bulk_g2s(s_boxes, P.job[0].boxes, bytes, boxbar);
    } else {
      mbar_arrive(boxbar);
    }
  }
  if (warp == nw - 1) {
    // tiles per job: the spatial filter's list for a job that has one (its
    // count bounded by the job's tiles), else every tile; prefix sums
    const uint32_t nj = MAXJ == 1 ? 1u : min(P.njobs, (uint32_t)MAXJ);
    uint32_t carry = 0;
    if (lane == 0) s_pref[0] = 0;
    for (uint32_t j0 = 0; j0 < nj; j0 += 32) {
      const uint32_t jj = j0 + (uint32_t)lane;
      uint32_t c = 0;
      if (jj < nj) {
        const ClassifyJob& J = P.job[MAXJ == 1 ? 0 : jj];
        c = (FILTER && J.tlist) ? min(*J.tcount, (uint32_t)J.num_tiles) : (uint32_t)J.num_tiles;
      }
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
      }
      if (jj < nj) s_pref[jj + 1] = carry + incl;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();
  // the launch's listed tiles, for the host's choice of the next pass's shape
  if (FILTER && P.listed_out && blockIdx.x == 0 && threadIdx.x == 0)
    *reinterpret_cast<volatile uint32_t*>(P.listed_out) =
        s_pref[MAXJ == 1 ? 1u : min(P.njobs, (uint32_t)MAXJ)];
  // the first NSTAGE slots, one warp each
  for (int s = warp; s < NSTAGE; s += nw) {
    const SlotMeta m = slot_meta<MAXJ, FILTER>(P, (uint32_t)s, s_pref, lane);
    fill_slot<MAXJ, NSTAGE, STAGE_BYTES, NBAR, FILTER>(P, (uint32_t)s, m, stages, full, s_sjob,
                                                       s_last, s_cand, s_boxes, lane);
    // the stage's next slot (a stage that ends here is never refilled)
    if (!m.end)
      store_meta<NSTAGE>(s_meta, s_meta_slot, s, (uint32_t)s + NSTAGE,
                         slot_meta<MAXJ, FILTER>(P, (uint32_t)s + NSTAGE, s_pref, lane), lane);
  }

  // ------------------------------------------------------------- workers
  uint32_t* queue = queues + (size_t)warp * kPairQueue;
  unsigned long long n_rounds = 0, n_outer = 0, n_pairs = 0;  // COUNT instance only
  bool run = true;
  {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(boxbar, 0, P.wait_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      if (lane == 0) atomicCAS(P.status, 0, (int)kStatusTimeoutBoxes);
      run = false;
    } else {
      mbar_wait_bounded(boxbar, 0, P.wait_ns);
    }
  }
  while (run) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(s_item, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    const uint32_t slot = item / IPT;
    const int sub = (int)(item - slot * IPT);
    const int stage = slot % NSTAGE;
    uint64_t* bar = &full[slot % NBAR];
    const uint32_t parity = (slot / NBAR) & 1;
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(bar, parity, P.wait_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      if (lane == 0) atomicCAS(P.status, 0, (int)kStatusTimeoutFull);
      break;
    }
    // completed phase: returns at once and orders the stage's data for this lane
    mbar_wait_bounded(bar, parity, P.wait_ns);
    unsigned char* sb = stages + (size_t)stage * STAGE_BYTES;
    const StageHdr hdr = *reinterpret_cast<const StageHdr*>(sb);
    if (hdr.end) break;
    // a single-roadmap launch has one job: a constant index lets every job
    // field stay a plain parameter read
    const ClassifyJob& J = P.job[MAXJ == 1 ? 0 : hdr.job];
    const int n_samp = hdr.n_samp, n_edges = hdr.n_edges;
    const int* etab = reinterpret_cast<const int*>(sb + kStageEtabOff);
    // per-stage accumulators live at a fixed place whatever the job, so a
    // stage reused by another roadmap's tile finds them zeroed
    uint32_t* acc_hit = reinterpret_cast<uint32_t*>(sb + kStageAccOff);
    uint32_t* acc_touch = acc_hit + kAccMax;
    const int K = (int)J.K;
    const int C = (int)J.C;
    const float margin = J.margin;
    const float inv_k = J.inv_k;
    const float inv_km1 = J.inv_km1;
    const float* ix = reinterpret_cast<const float*>(sb + J.off_in) + hdr.in_shift;
    const float* iy = ix + J.in_cap;
    const float* iz = iy + J.in_cap;
    const float* ir = iz + J.in_cap;
    const float* ox = reinterpret_cast<const float*>(sb + J.off_out) + hdr.out_shift;
    const float* oy = ox + J.out_cap;
    const float* oz = oy + J.out_cap;
    const float* orad = oz + J.out_cap;
    const float4* bx = MAXJ == 1 ? s_boxes : s_boxes + (size_t)stage * (kBoxAreaFloats / 4);
    // link radii of the roadmap, after its box records (link-end records)
    const float* link_r = reinterpret_cast<const float*>(bx + kBoxesPerPass * 6);
    const bool joints = J.joints != 0;
    const int r_end = min((sub + 1) * RPI, ROUNDS);
    for (int rnd = sub * RPI; rnd < r_end; ++rnd) {
      const int base = 31 * rnd;
      if (base >= n_samp) break;
      uint32_t rc = ~0u;
      if constexpr (FILTER) {
        // the spatial filter found no moved box near the round (not copied)
        if (J.rcand) rc = s_cand[stage * kRoundSlots + rnd];
        if (rc == 0u) continue;
      }
      if constexpr (COUNT) ++n_rounds;
      const int q = base - 1 + lane;
      const SampleAt at = locate_sample(etab, n_edges, q, min(base + 31, n_samp));
      const int j = at.j, n = at.n, k = at.k, o = at.o, li = at.li;
      const bool valid = at.valid, has_next = at.has_next;
      // ---- a3: the outer sphere of the interval after q, against the moved
      // boxes that may reach the round: the spatial filter's candidates for
      // the round, or those that survive a warp bounding-sphere cull
      float x = ox[o], y = oy[o], z = oz[o], r = orad[o];
      const uint32_t act = __ballot_sync(0xffffffffu, has_next);
      uint32_t bits = 0;
      uint32_t any_cand = 0;
      if (act) {
        uint32_t cand = rc;
        // the filter's test (exact box distance from a near-smallest sphere
        // about the round) is tighter than the cull, which then only costs
        if (!FILTER || J.rcand == nullptr) {
          // the bounding sphere's centre: the midpoint of the first and the
          // last active sphere centres (the round's spheres follow one link's
          // path, and the chord's midpoint gave the fewest candidates of the
          // centres tried); any centre is valid, the radius covers every sphere
          const int lo_l = __ffs(act) - 1, hi_l = 31 - __clz(act);
          const float mx = 0.5f * (__shfl_sync(0xffffffffu, x, lo_l) + __shfl_sync(0xffffffffu, x, hi_l));
          const float my = 0.5f * (__shfl_sync(0xffffffffu, y, lo_l) + __shfl_sync(0xffffffffu, y, hi_l));
          const float mz = 0.5f * (__shfl_sync(0xffffffffu, z, lo_l) + __shfl_sync(0xffffffffu, z, hi_l));
          const float dx = x - mx, dy = y - my, dz = z - mz;
          const float reach = has_next ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + r : 0.0f;
          const float rw = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(reach)));
          bool cb = false;
          if (lane < C) {
            const float4 b0 = bx[6 * lane];
            const float ex = b0.x - mx, ey = b0.y - my, ez = b0.z - mz;
            const float thr = (rw + b0.w + margin) * (1.0f + 1e-6f) + 1e-5f;
            cb = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= thr * thr;
          }
          cand = __ballot_sync(0xffffffffu, cb) & rc;
        }
        // a box already known to hit the edge of every lane in this pass is
        // done there: a hit implies a touch, so its tests could add no bit
        cand &= ~__reduce_and_sync(
            0xffffffffu, valid ? *reinterpret_cast<volatile uint32_t*>(&acc_hit[j]) : ~0u);
        any_cand = cand;
        const float rt = r + margin;
        const float rt2 = rt * rt;
        // two candidate boxes per iteration for instruction-level parallelism,
        // and a last single box on its own (cand is the same on every lane)
        while (cand) {
          const int b0 = __ffs(cand) - 1;
          cand &= cand - 1;
          if (cand) {
            const int b1 = __ffs(cand) - 1;
            cand &= cand - 1;
            const float d0 = box_dist2(x, y, z, bx + 6 * b0);
            const float d1 = box_dist2(x, y, z, bx + 6 * b1);
            bits |= (d0 <= rt2 ? 1u << b0 : 0u) | (d1 <= rt2 ? 1u << b1 : 0u);
          } else {
            bits |= box_dist2(x, y, z, bx + 6 * b0) <= rt2 ? 1u << b0 : 0u;
          }
        }
        if (!has_next) bits = 0;
        if (bits) atomicOr(&acc_touch[j], bits);
        if constexpr (COUNT) n_outer += (unsigned long long)__popc(any_cand) * __popc(act);
      }
      // no moved box near the round: nothing touched, so no inner test either
      if (!any_cand) continue;
      // ---- a4: inner spheres of q against the boxes touched by the
      // intervals next to it.  Built records (link ends): each of those outer
      // spheres holds q's capsule, so a box an inner sphere of q hits is
      // touched by both, and only boxes touched on both sides (on the one
      // side at an edge's ends) are tested.  Uploaded sphere records promise
      // only that the two together hold q's spheres: boxes touched on either
      const uint32_t prev = __shfl_up_sync(0xffffffffu, bits, 1);
      uint32_t need = 0;
      if (valid && q >= base) {
        const uint32_t after = k < n - 1 ? bits : (joints ? ~0u : 0u);
        const uint32_t before = k > 0 ? prev : (joints ? ~0u : 0u);
        need = joints ? (after & before) : (after | before);
        if (need) need &= ~*reinterpret_cast<volatile uint32_t*>(&acc_hit[j]);
      }
      // the round's (sample, box) pairs into the warp's queue, box by box: a
      // ballot per box gives each lane its place (when the pairs outnumber
      // the queue, each lane tests its own below)
      const uint32_t need_or = __reduce_or_sync(0xffffffffu, need);
      int total = 0;
      if (need_or) {
        const uint32_t lt = (1u << lane) - 1u;
        const uint32_t ent = ((uint32_t)li << 27) | ((uint32_t)q << 13) | ((uint32_t)j << 5);
        for (uint32_t m = need_or; m; m &= m - 1) {
          const int b = __ffs(m) - 1;
          const bool mine = (need >> b) & 1u;
          const uint32_t mb = __ballot_sync(0xffffffffu, mine);
          const int pos = total + __popc(mb & lt);
          if (mine && pos < kPairQueue) queue[pos] = ent | (uint32_t)b;
          total += __popc(mb);
        }
      }
      if constexpr (COUNT) n_pairs += (unsigned long long)total;
      // a (sample, box) pair packs the box (bits 0..4), the edge-table entry
      // (5..12), the local sample (13..26) and its link (27..31)
      if ((J.regular || joints) && total > 0) {
        // interpolated inner centres: one (sample, box) pair per lane,
        // compacted when the pairs fit the queue
        if (total <= kPairQueue) {
          __syncwarp();
          for (int it = lane; it < total; it += 32) {
            const uint32_t e = queue[it];
            const int qq = (int)((e >> 13) & 0x3fffu), jj = (int)((e >> 5) & 255u);
            const float4* B = bx + 6 * (int)(e & 31u);
            bool hit;
            if (joints) {
              const int le = (int)(e >> 27);
              const float rr = link_r[le] - margin;
              float ax = 0.0f, ay = 0.0f, az = 0.0f;  // link 0 starts at the base
              if (le > 0) {
                const int qn = qq - etab[4 * jj + 1];
                ax = ix[qn];
                ay = iy[qn];
                az = iz[qn];
              }
              hit = rr > 0.0f && inner_hit_joints(ax, ay, az, ix[qq], iy[qq], iz[qq], K, inv_k, rr, B);
            } else {
              const int s0 = K * qq;
              const float rr = ir[s0] - margin;
              hit = rr > 0.0f && inner_hit_regular(ix, iy, iz, s0, K, inv_km1, rr, B);
            }
            if (hit) atomicOr(&acc_hit[jj], 1u << (e & 31u));
          }
          __syncwarp();
        } else {
          // many pairs in one round: each lane tests its own
          uint32_t hits = 0;
          if (need) {
            if (joints) {
              const float rr = link_r[li] - margin;
              const float ax = li > 0 ? ix[q - n] : 0.0f, ay = li > 0 ? iy[q - n] : 0.0f,
                          az = li > 0 ? iz[q - n] : 0.0f;
              const float fx = ix[q], fy = iy[q], fz = iz[q];
              if (rr > 0.0f)
                for (uint32_t m = need; m; m &= m - 1) {
                  const int b = __ffs(m) - 1;
                  if (inner_hit_joints(ax, ay, az, fx, fy, fz, K, inv_k, rr, bx + 6 * b))
                    hits |= 1u << b;
                }
            } else {
              const float rr = ir[K * q] - margin;
              if (rr > 0.0f)
                for (uint32_t m = need; m; m &= m - 1) {
                  const int b = __ffs(m) - 1;
                  if (inner_hit_regular(ix, iy, iz, K * q, K, inv_km1, rr, bx + 6 * b))
                    hits |= 1u << b;
                }
            }
          }
          if (hits) atomicOr(&acc_hit[j], hits);
          __syncwarp();
        }
      } else if (total > 0 && total <= kPairQueue) {
        // compact the (sample, box) pairs, then test (pair, sphere) items on
        // all lanes, two items per lane per iteration
        __syncwarp();
        const int n_items = total * K;
        for (int it = lane; it < n_items; it += 64) {
          const int it2 = min(it + 32, n_items - 1);
          const int p0 = __float2int_rz(((float)it + 0.5f) * inv_k);
          const int p1 = __float2int_rz(((float)it2 + 0.5f) * inv_k);
          const uint32_t e0 = queue[p0], e1 = queue[p1];
          const int s0 = K * (int)((e0 >> 13) & 0x3fffu) + (it - p0 * K);
          const int s1 = K * (int)((e1 >> 13) & 0x3fffu) + (it2 - p1 * K);
          const float r0 = ir[s0] - margin, r1 = ir[s1] - margin;
          const float d0 = box_dist2(ix[s0], iy[s0], iz[s0], bx + 6 * (int)(e0 & 31u));
          const float d1 = box_dist2(ix[s1], iy[s1], iz[s1], bx + 6 * (int)(e1 & 31u));
          if (r0 > 0.0f && d0 <= r0 * r0) atomicOr(&acc_hit[(e0 >> 5) & 255u], 1u << (e0 & 31u));
          if (it + 32 < n_items && r1 > 0.0f && d1 <= r1 * r1)
            atomicOr(&acc_hit[(e1 >> 5) & 255u], 1u << (e1 & 31u));
        }
        __syncwarp();
      } else if (total > kPairQueue) {
        // many pairs in one round: each lane tests its own
        uint32_t hits = 0;
        for (uint32_t m = need; m; m &= m - 1) {
          const int b = __ffs(m) - 1;
          for (int s = K * q, se = K * q + K; s < se; ++s) {
            const float rin = ir[s] - margin;
            if (rin > 0.0f && box_dist2(ix[s], iy[s], iz[s], bx + 6 * b) <= rin * rin) {
              hits |= 1u << b;
              break;
            }
          }
        }
        if (hits) atomicOr(&acc_hit[j], hits);
        __syncwarp();
      }
    }
    // ---- item done; the tile's last item flushes the tile's bits and refills
    // the stage
    __syncwarp();
    uint32_t done = 0;
    if (lane == 0) {
      __threadfence_block();
      done = atomicAdd(&s_cnt[stage], 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == IPT - 1) {
      __threadfence_block();
      // ---- a5: the tile's per-edge bits into the global accumulators.  They
      // are taken into registers and the stage is refilled first: the refill
      // is on the ring's critical path, the global ORs are not
      static_assert(kAccMax <= 3 * 32, "accumulator entries per lane");
      uint32_t hv[3], tv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int jl = lane + 32 * c;
        hv[c] = 0;
        tv[c] = 0;
        if (jl < n_edges) {
          hv[c] = *reinterpret_cast<volatile uint32_t*>(&acc_hit[jl]);
          tv[c] = *reinterpret_cast<volatile uint32_t*>(&acc_touch[jl]);
          acc_hit[jl] = 0;
          acc_touch[jl] = 0;
        }
      }
      if (lane == 0) s_cnt[stage] = 0;
      __syncwarp();
      // the stage is free: this warp loads it with the slot NSTAGE ahead,
      // from the metadata the stage's last fill left (a bounded wait: that
      // fill's loads may still be in flight)
      SlotMeta m;
      if (!take_meta(s_meta, s_meta_slot, stage, slot + NSTAGE, P.wait_ns, m, lane)) {
        if (lane == 0) atomicCAS(P.status, 0, (int)kStatusTimeoutFull);
        m = SlotMeta{};
        m.end = 1;
      }
      fill_slot<MAXJ, NSTAGE, STAGE_BYTES, NBAR, FILTER>(P, slot + NSTAGE, m, stages, full, s_sjob,
                                                         s_last, s_cand, s_boxes, lane);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const uint64_t e = (uint64_t)hdr.e_first + lane + 32 * c;
        if (hv[c]) atomicOr(&J.edge_acc[2 * e], hv[c]);
        if (tv[c]) atomicOr(&J.edge_acc[2 * e + 1], tv[c]);
      }
      // and the metadata of the stage's slot after that
      if (!m.end)
        store_meta<NSTAGE>(s_meta, s_meta_slot, stage, slot + 2 * NSTAGE,
                           slot_meta<MAXJ, FILTER>(P, slot + 2 * NSTAGE, s_pref, lane), lane);
    }
  }
  if (COUNT && lane == 0 && P.work) {
    atomicAdd(&P.work[0], n_rounds);
    atomicAdd(&P.work[1], n_outer);
    atomicAdd(&P.work[2], n_pairs);
  }
  // Before the CTA exits, no bulk copy of it may still be in flight.  Every
  // warp has stopped issuing once all are here; then one thread waits
  // (bounded; at once when every filled slot has landed) for the phase of
  // each stage's last fill, whatever it was (normally an end marker, whose
  // phase is complete), and for the box records copied at the start: after
  // a wait that ran out, a slot may have been filled that no worker waited
  // for.  A stage's earlier fills were all waited for by its workers.
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s)
      if (s_last[s] != 0xffffffffu)
        mbar_wait_bounded(&full[s_last[s] % NBAR], (s_last[s] / NBAR) & 1, kDrainLimit);
    mbar_wait_bounded(boxbar, 0, kDrainLimit);
  }
}


// ===========================================================================
// a6: merge the pass's bits into the per-edge box sets (Algorithm 1's
// intersection lists) and relabel
// ===========================================================================
// One thread per edge.  Unordered passes have ascending, distinct box ids,
// so boxes sharing a 32-bit mask word are consecutive and each touched word
// is read and written once.  Ordered passes (pending requests) apply their
// positions one at a time and store the label after each request's last
// position into that request's snapshot row.  Per-edge counts of hitting and
// touching boxes give the label without reading the untouched words.
template <int MAXJ>
__global__ void __launch_bounds__(256) merge_kernel(const __grid_constant__ MergeParams<MAXJ> P) {
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= P.total_edges) return;
  int lo = 0, hi = (int)P.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.job[mid].edge_base <= g) lo = mid; else hi = mid - 1;
  }
  const MergeJob& J = P.job[lo];
  const uint64_t e = g - J.edge_base;
  uint2* accp = reinterpret_cast<uint2*>(J.edge_acc) + e;
  const uint2 acc = *accp;
  if (acc.x | acc.y) *accp = make_uint2(0u, 0u);
  if (P.status) {
    // the classify launch gave up or was skipped: its bits are partial, so
    // the sets, counts and labels stay; each roadmap of the launch latches
    // the error for the host
    const int st = *reinterpret_cast<volatile const int*>(P.status);
    if (st != 0) {
      if (e == 0 && J.status) atomicCAS(J.status, 0, st);
      return;
    }
  }
  uint32_t cnt = J.counts[e];
  int rc = (int)(cnt & 0xffffu), tc = (int)(cnt >> 16);
  uint32_t* red = J.red + e * J.Wm;
  uint32_t* tch = J.touch + e * J.Wm;
  if (J.ordered) {
    // positions in request order; a box may appear more than once, the later
    // position replacing the earlier one's bits (its later pose)
    for (uint32_t p = 0; p < J.C; ++p) {
      const uint32_t w = J.ids[p] >> 5, bit = 1u << (J.ids[p] & 31);
      const uint32_t r_old = red[w], t_old = tch[w];
      const uint32_t r_new = ((acc.x >> p) & 1u) ? (r_old | bit) : (r_old & ~bit);
      const uint32_t t_new = ((acc.y >> p) & 1u) ? (t_old | bit) : (t_old & ~bit);
      if (r_new != r_old) {
        red[w] = r_new;
        rc += (r_new & bit) ? 1 : -1;
      }
      if (t_new != t_old) {
        tch[w] = t_new;
        tc += (t_new & bit) ? 1 : -1;
      }
      if ((J.snap_mask >> p) & 1u)
        J.hist[(size_t)J.snap_slot[p] * J.num_edges + e] = rc > 0 ? 2 : (tc > 0 ? 1 : 0);
    }
    const uint32_t ncnt = (uint32_t)rc | ((uint32_t)tc << 16);
    if (ncnt != cnt) J.counts[e] = ncnt;
    J.labels[e] = rc > 0 ? 2 : (tc > 0 ? 1 : 0);
    return;
  }
  uint32_t cur = 0xffffffffu, r_old = 0, t_old = 0, r_new = 0, t_new = 0;
  for (uint32_t p = 0; p <= J.C; ++p) {
    const uint32_t w = p < J.C ? (J.ids[p] >> 5) : 0xfffffffeu;
    if (w != cur) {
      if (cur != 0xffffffffu) {
        if (r_new != r_old) {
          red[cur] = r_new;
          rc += __popc(r_new) - __popc(r_old);
        }
        if (t_new != t_old) {
          tch[cur] = t_new;
          tc += __popc(t_new) - __popc(t_old);
        }
      }
      if (p == J.C) break;
      cur = w;
      r_old = r_new = red[w];
      t_old = t_new = tch[w];
    }
    const uint32_t bit = 1u << (J.ids[p] & 31);
    r_new = ((acc.x >> p) & 1u) ? (r_new | bit) : (r_new & ~bit);
    t_new = ((acc.y >> p) & 1u) ? (t_new | bit) : (t_new & ~bit);
  }
  const uint32_t ncnt = (uint32_t)rc | ((uint32_t)tc << 16);
  if (ncnt != cnt) J.counts[e] = ncnt;
  J.labels[e] = rc > 0 ? 2 : (tc > 0 ? 1 : 0);
}

// ===========================================================================
// Non-lazy resolution of gray edges (Algorithm 1, lazy = false)
// ===========================================================================
// Squared distance from the segment p -> p + dlt to the box [-h, h] (box
// frame), exactly.  Along the segment each axis contributes
// max(0, |x_k(t)| - h_k)^2, so the sum is a convex piecewise quadratic in t
// whose pieces end where a coordinate crosses -h_k or +h_k.  The six
// crossings, clamped to [0, 1], are sorted by a fixed 12-comparator network;
// on each of the seven pieces the quadratic sum_k (o_k + t d_k)^2 over the
// axes outside the box there is minimised in closed form.
__device__ __forceinline__ float seg_box_dist2(const float p[3], const float dlt[3],
                                               const float h[3]) {
  float t[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float lo = 0.0f, hi = 0.0f;
    if (dlt[k] != 0.0f) {
      lo = (-h[k] - p[k]) / dlt[k];
      hi = (h[k] - p[k]) / dlt[k];
    }
    t[2 * k] = fminf(fmaxf(lo, 0.0f), 1.0f);
    t[2 * k + 1] = fminf(fmaxf(hi, 0.0f), 1.0f);
  }
#define RGG_CX(i, j)                                    \
  {                                                     \
    const float lo_ = fminf(t[i], t[j]), hi_ = fmaxf(t[i], t[j]); \
    t[i] = lo_;                                         \
    t[j] = hi_;                                         \
  }
  RGG_CX(1, 2) RGG_CX(4, 5) RGG_CX(0, 2) RGG_CX(3, 5) RGG_CX(0, 1) RGG_CX(3, 4)
  RGG_CX(2, 5) RGG_CX(0, 3) RGG_CX(1, 4) RGG_CX(2, 4) RGG_CX(1, 3) RGG_CX(2, 3)
#undef RGG_CX
  float best = INFINITY;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const float ta = i == 0 ? 0.0f : t[i - 1];
    const float tb = i == 6 ? 1.0f : t[i];
    const float tm = 0.5f * (ta + tb);
    float A = 0.0f, B = 0.0f, o[3];
    bool out[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float x = fmaf(tm, dlt[k], p[k]);
      out[k] = x > h[k] || x < -h[k];
      o[k] = x > h[k] ? p[k] - h[k] : p[k] + h[k];
      if (out[k]) {
        A = fmaf(dlt[k], dlt[k], A);
        B = fmaf(o[k], dlt[k], B);
      }
    }
    const float ts = A > 0.0f ? fminf(fmaxf(-B / A, ta), tb) : ta;
    float f = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (out[k]) {
        const float v = fmaf(ts, dlt[k], o[k]);
        f = fmaf(v, v, f);
      }
    best = fminf(best, f);
  }
  return best;
}

// Edges that are not gray keep their label.  A gray edge's block gathers up
// to 32 boxes of its touch set at a time (only boxes an outer sphere touched
// can meet the capsules) and thread k takes the configurations k, k+256, ...
// of t_c = c / ((n_e - 1) F): FP32 kinematics, then, per link and box, the
// capsule-axis-to-box distance minus the link radius.  A (link, box) pair
// whose bounding spheres cannot beat the best so far is skipped, so the
// minimum is exact.  The block stops after the first step with a clearance
// below -thr (RED); otherwise the edge is GREEN when the minimum is at least
// thr, and stays GRAY in between.
// Order-preserving map of a float onto an unsigned int (for atomicMin).
__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Lists the gray edges (one warp-aggregated atomic per warp, in no
// particular order) for resolve_gray_kernel, and passes every other edge's
// label through.
__global__ void __launch_bounds__(256) gray_list_kernel(const __grid_constant__ ResolveParams p) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x; e0 < p.n_edges;
       e0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = e0 + threadIdx.x;
    const uint8_t lab = e < p.n_edges ? p.labels[e] : 0;
    const bool gray = e < p.n_edges && lab == 1;
    if (e < p.n_edges && !gray) {
      p.out[e] = lab;
      p.clearance[e] = __int_as_float(0x7fc00000);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, gray);
    unsigned long long at = 0;
    if (lane == 0 && m) at = atomicAdd(&p.work[4], (unsigned long long)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (gray) p.gray[at + __popc(m & ((1u << lane) - 1u))] = (uint32_t)e;
  }
}

__global__ void __launch_bounds__(256) resolve_gray_kernel(const __grid_constant__ ResolveParams p) {
  // One block per gray edge at a time: its 256 threads take the edge's
  // configurations in steps of 256 (a long edge no longer runs on one warp).
  // Blocks take the listed gray edges one at a time from a shared cursor, so
  // that the long edges do not pile up on a few blocks.
  __shared__ float s_box[32][16];
  __shared__ uint64_t s_e;
  // per joint: the start angle and the step per configuration, each as an
  // FP32 pair (high part, remainder) of its FP64 value
  __shared__ float4 s_q[kMaxBuildLinks];
  __shared__ uint32_t s_best;                 // block's running minimum (float_key)
  __shared__ float s_red_best[8];
  __shared__ unsigned long long s_evals[8];
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31;
  const uint32_t wib = tid >> 5;
  const uint32_t L = p.L, Wm = p.Wm;
  const uint64_t n_gray = min((uint64_t)p.work[4], p.n_edges);
  for (;;) {
    if (tid == 0) {
      const unsigned long long i = atomicAdd(&p.work[5], 1ull);
      s_e = i < n_gray ? (uint64_t)p.gray[i] : ~0ull;
    }
    __syncthreads();
    const uint64_t e = s_e;
    if (e == ~0ull) break;
    const uint64_t n = p.soff[e + 1] - p.soff[e];
    const uint64_t m = (n - 1) * (uint64_t)p.F;
    const uint32_t* tw = p.touch + e * Wm;
    if (tid == 0) s_best = float_key(INFINITY);
    if (tid < L) {
      const double a = p.qa[e * L + tid];
      const double d = (p.qb[e * L + tid] - a) / (double)m;
      const float ah = (float)a, dh = (float)d;
      s_q[tid] = make_float4(ah, (float)(a - (double)ah), dh, (float)(d - (double)dh));
    }
    float best = INFINITY;
    unsigned long long evals = 0;
    bool red = false;
    uint32_t w = 0, word = Wm ? tw[0] : 0u;
    for (;;) {
      // the next up to 32 boxes of the touch set (every thread walks the words)
      int cnt = 0;
      __syncthreads();  // the previous batch's boxes are no longer read
      while (cnt < 32 && w < Wm) {
        if (word == 0u) {
          if (++w < Wm) word = tw[w];
          continue;
        }
        const uint32_t b = 32u * w + (uint32_t)(__ffs(word) - 1);
        word &= word - 1u;
        if ((uint32_t)cnt == tid) {
          const float4* src = reinterpret_cast<const float4*>(p.table + 16 * (size_t)b);
          float4* dst = reinterpret_cast<float4*>(s_box[tid]);
          for (int c = 0; c < 4; ++c) dst[c] = src[c];
        }
        ++cnt;
      }
      __syncthreads();
      if (cnt == 0) break;
      for (uint64_t c0 = 0; c0 <= m && !red; c0 += 256) {
        const uint64_t c = c0 + tid;
        // prune against the block's best so far, not only this thread's
        best = fminf(best, key_float(*reinterpret_cast<volatile uint32_t*>(&s_best)));
        if (c <= m) {
          const float cf = (float)c;  // exact: c < 2^24
          float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
          float o[3] = {0, 0, 0};
          for (uint32_t i = 0; i < L; ++i) {
            // q = a + c d, rounded once to FP32 (as the FP64 value would be,
            // without FP64 arithmetic): c * d_high exactly as p + pe (an FMA
            // gives the product's rounding error), a_high + p exactly as
            // s + se (Knuth's two-sum), then the small terms added to s
            const float4 z = s_q[i];
            const float pp = __fmul_rn(cf, z.z);
            const float pe = fmaf(cf, z.z, -pp);
            const float s = __fadd_rn(z.x, pp);
            const float sb = __fsub_rn(s, z.x);
            const float se = __fadd_rn(__fsub_rn(z.x, __fsub_rn(s, sb)), __fsub_rn(pp, sb));
            const float q = __fadd_rn(s, __fadd_rn(se, __fadd_rn(pe, fmaf(cf, z.w, z.y))));
            float st, ct;
            sincosf(q, &st, &ct);
            const float v0 = p.a[i] * ct, v1 = p.a[i] * st, v2 = p.d[i];
            float on[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
              on[r] = fmaf(R[3 * r], v0, fmaf(R[3 * r + 1], v1, fmaf(R[3 * r + 2], v2, o[r])));
            const float mx = 0.5f * (o[0] + on[0]), my = 0.5f * (o[1] + on[1]),
                        mz = 0.5f * (o[2] + on[2]);
            const float hl = 0.5f * sqrtf((on[0] - o[0]) * (on[0] - o[0]) +
                                          (on[1] - o[1]) * (on[1] - o[1]) +
                                          (on[2] - o[2]) * (on[2] - o[2]));
            const float rad = p.radius[i];
            for (int b = 0; b < cnt; ++b) {
              const float* B = s_box[b];
              const float hx = B[12], hy = B[13], hz = B[14];
              const float dx = mx - B[0], dy = my - B[1], dz = mz - B[2];
              // lower bound of the pair's clearance from the two bounding spheres
              const float lb = sqrtf(dx * dx + dy * dy + dz * dz) - hl -
                               sqrtf(hx * hx + hy * hy + hz * hz) - rad;
              if (lb > best + 1e-5f) continue;
              // the segment in the box frame: coordinate k = column k of R_b . (x - c_b)
              float pb[3], db[3];
              const float h3[3] = {hx, hy, hz};
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float ax = B[3 + k], ay = B[6 + k], az = B[9 + k];
                pb[k] = ax * (o[0] - B[0]) + ay * (o[1] - B[1]) + az * (o[2] - B[2]);
                db[k] = ax * (on[0] - o[0]) + ay * (on[1] - o[1]) + az * (on[2] - o[2]);
              }
              const float cl = sqrtf(seg_box_dist2(pb, db, h3)) - rad;
              best = fminf(best, cl);
              ++evals;
            }
            // R <- R * Rz(q) Rx(alpha)
            const float ca = p.ca[i], sa = p.sa[i];
            const float A[9] = {ct, -st * ca, st * sa, st, ct * ca, -ct * sa, 0.0f, sa, ca};
            float Rn[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
              for (int cc = 0; cc < 3; ++cc)
                Rn[3 * r + cc] = fmaf(R[3 * r], A[cc], fmaf(R[3 * r + 1], A[3 + cc], R[3 * r + 2] * A[6 + cc]));
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k] = Rn[k];
#pragma unroll
            for (int r = 0; r < 3; ++r) o[r] = on[r];
          }
        }
        if (best < INFINITY) atomicMin(&s_best, float_key(best));
        red = __syncthreads_or(best <= -p.thr) != 0;
      }
      if (red) break;
    }
    // block minimum of the clearances and sum of the evaluation counts
    for (int off = 16; off; off >>= 1) {
      best = fminf(best, __shfl_xor_sync(0xffffffffu, best, off));
      evals += __shfl_xor_sync(0xffffffffu, evals, off);
    }
    if (lane == 0) {
      s_red_best[wib] = best;
      s_evals[wib] = evals;
    }
    __syncthreads();
    if (tid == 0) {
      for (int k = 1; k < 8; ++k) {
        best = fminf(best, s_red_best[k]);
        evals += s_evals[k];
      }
      const uint8_t res = best <= -p.thr ? 2 : (best >= p.thr ? 0 : 1);
      p.out[e] = res;
      p.clearance[e] = best;
      atomicAdd(&p.work[0], 1ull);
      if (res == 2) atomicAdd(&p.work[1], 1ull);
      if (res == 0) atomicAdd(&p.work[2], 1ull);
      atomicAdd(&p.work[3], evals);
    }
    __syncthreads();  // the shared results are read before the next edge
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

template <int MAXJ, int NSTAGE, int STAGE_BYTES, int IPT, bool FILTER>
static size_t smem_bytes_t(uint32_t consumer_warps) {
  // mirrors the carve-up at the top of classify_kernel; every warp is a
  // worker with its own pair queue
  constexpr int kBoxAreas = MAXJ == 1 ? 1 : NSTAGE;
  constexpr int NBAR = NSTAGE * full_barriers_per_stage(IPT);
  constexpr size_t kOffFull = (size_t)NSTAGE * STAGE_BYTES;
  constexpr size_t kOffCnt = kOffFull + (NBAR + 1) * sizeof(uint64_t) + 8;
  constexpr size_t kOffMeta = (kOffCnt + 3 * 4 * ((NSTAGE + 3) & ~3) + 4 * (MAXJ + 1) + 4 * NSTAGE + 15) & ~(size_t)15;
  constexpr size_t kOffCand = (kOffMeta + 4 * (size_t)NSTAGE * kMetaWords + 15) & ~(size_t)15;
  constexpr size_t kOffBoxes =
      (kOffCand + (FILTER ? (size_t)NSTAGE * kRoundSlots * 4 : 0) + 127) & ~(size_t)127;
  constexpr size_t kOffQueues = kOffBoxes + (size_t)kBoxAreas * kBoxAreaFloats * 4;
  return kOffQueues + (size_t)(consumer_warps + 1) * 4 * kPairQueue;
}

size_t classify_smem_bytes(int variant, uint32_t consumer_warps) {
  // the batched kernel's (larger) footprint, which bounds both
  switch (variant) {
#define RGG_VARIANT(id, ns, sb, rd, rpi) \
  case id: return smem_bytes_t<kMaxJobs, ns, sb, (rd + rpi - 1) / rpi, filter_variant(id)>(consumer_warps);
    RGG_VARIANTS(RGG_VARIANT)
#undef RGG_VARIANT
    default: return 0;
  }
}

template <int MAXJ, int NSTAGE, int STAGE_BYTES, int ROUNDS, int RPI, bool FILTER, bool COUNT = false>
static cudaError_t launch_classify_v(const ClassifyParams<MAXJ>& p, const ClassifyLaunch& lc,
                                     cudaStream_t s) {
  auto kern = classify_kernel<MAXJ, NSTAGE, STAGE_BYTES, ROUNDS, RPI, FILTER, COUNT>;
  const size_t smem = smem_bytes_t<MAXJ, NSTAGE, STAGE_BYTES, (ROUNDS + RPI - 1) / RPI, FILTER>(lc.consumer_warps);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<lc.grid, 32 * (1 + lc.consumer_warps), smem, s>>>(p);
  return cudaGetLastError();
}

// The filtered instance exists for the two default pipeline variants only.
template <int MAXJ, int ID, int NS, int SB, int RD, int RPI>
static cudaError_t launch_variant(const ClassifyParams<MAXJ>& p, const ClassifyLaunch& lc,
                                  bool filtered, cudaStream_t s) {
  if constexpr (filter_variant(ID)) {
    // the counting instances exist for single-roadmap launches of the
    // default shapes
    if constexpr (MAXJ == 1) {
      if (p.work) {
        if (filtered) return launch_classify_v<MAXJ, NS, SB, RD, RPI, true, true>(p, lc, s);
        return launch_classify_v<MAXJ, NS, SB, RD, RPI, false, true>(p, lc, s);
      }
    }
    if (filtered) return launch_classify_v<MAXJ, NS, SB, RD, RPI, true>(p, lc, s);
  } else {
    if (filtered) return cudaErrorInvalidValue;
  }
  return launch_classify_v<MAXJ, NS, SB, RD, RPI, false>(p, lc, s);
}

template <int MAXJ>
static cudaError_t launch_classify_t(const ClassifyParams<MAXJ>& p, const ClassifyLaunch& lc,
                                     cudaStream_t s) {
  // the spatial filter's per-pass test, when a job uses it
  bool filtered = false;
  for (uint32_t j = 0; j < p.njobs && j < (uint32_t)MAXJ; ++j) filtered |= p.job[j].rcand != nullptr;
  if (filtered && p.total_tiles) {
    // a warp per kFilterTilesPerWarp tiles, 8 warps per block
    constexpr uint64_t per_block = 8 * (uint64_t)kFilterTilesPerWarp;
    round_filter_kernel<MAXJ>
        <<<(unsigned)((p.total_tiles + per_block - 1) / per_block), 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  switch (lc.variant) {
#define RGG_VARIANT(id, ns, sb, rd, rpi) \
  case id: return launch_variant<MAXJ, id, ns, sb, rd, rpi>(p, lc, filtered, s);
    RGG_VARIANTS(RGG_VARIANT)
#undef RGG_VARIANT
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_classify_single(const ClassifyParams<1>& p, const ClassifyLaunch& lc,
                                   cudaStream_t s) {
  return launch_classify_t<1>(p, lc, s);
}

cudaError_t launch_classify_batched(const ClassifyParams<kMaxJobs>& p, const ClassifyLaunch& lc,
                                    cudaStream_t s) {
  return launch_classify_t<kMaxJobs>(p, lc, s);
}

template <int MAXJ>
static cudaError_t launch_merge_t(const MergeParams<MAXJ>& p, cudaStream_t s) {
  if (p.total_edges == 0) return cudaSuccess;
  const uint32_t blk = 256;
  merge_kernel<MAXJ><<<(unsigned)((p.total_edges + blk - 1) / blk), blk, 0, s>>>(p);
  return cudaGetLastError();
}

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(MergeParams<kMaxJobs>) <= 32764, "merge parameters too large");
static_assert(sizeof(BoxPrepParams) <= 32764, "box-prep parameters too large");
static_assert(sizeof(BoxUpdateParams) <= 32764, "box-update parameters too large");
static_assert(sizeof(ClassifyParams<kMaxJobs>) <= 32764, "classify parameters too large");

cudaError_t launch_round_bounds(const RoundBoundsParams& p, int num_sms, cudaStream_t s) {
  if (p.T == 0) return cudaSuccess;
  const uint64_t want = (p.T + 7) / 8;  // a warp per tile
  const uint64_t cap = (uint64_t)num_sms * 16;
  round_bounds_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_resolve_gray(const ResolveParams& p, int num_sms, cudaStream_t s) {
  if (p.n_edges == 0) return cudaSuccess;
  // the gray edges first (work[4] and work[5] start at zero)
  const uint64_t lb = (p.n_edges + 255) / 256, lcap = (uint64_t)num_sms * 8;
  gray_list_kernel<<<(unsigned)(lb < lcap ? lb : lcap), 256, 0, s>>>(p);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return le;
  // a block per gray edge at a time; as many blocks as are resident at once,
  // so that every block starts with the launch
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resolve_gray_kernel, 256, 0) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const uint64_t want = p.n_edges;
  const uint64_t cap = (uint64_t)num_sms * (uint64_t)per_sm;
  resolve_gray_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_merge_single(const MergeParams<1>& p, cudaStream_t s) {
  return launch_merge_t<1>(p, s);
}

cudaError_t launch_merge_batched(const MergeParams<kMaxJobs>& p, cudaStream_t s) {
  return launch_merge_t<kMaxJobs>(p, s);
}

}  // namespace rgg
