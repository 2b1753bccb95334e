// The paper's own primitives on the GPU (Sec. 4.2, Sec. 4.3): per (edge,
// body) OBB outer approximations, shortcut splines through the inscribed
// spheres' centres as inner approximations, a one-layer uniform grid over the
// OBBs, and the per-pass queries (OBB-OBB separating-axis tests, spline
// segment - obstacle sphere tests) that feed the shared merge kernel.
//
//   obb_build_kernel    offline: FP64 kinematics, boxes, greedy shortcuts
//   obb_bounds_kernel   offline: extent of the OBBs (grid sizing)
//   obb_grid_kernel     offline: cell incidences (count, then fill)
//   obb_pairs_kernel    per pass: chunk size, (moved box, grid cell, chunk) work list
//   obb_query_kernel    per pass: the tests, OR-ed into the per-edge bits
#include <cstdio>

#include "rgg_device.cuh"
#include "rgg_kernels.h"

namespace rgg {

// ===========================================================================
// offline build
// ===========================================================================
// Joint positions at q = qa + t (qb - qa): J[0] = 0 (base), then down the DH
// chain o_{i+1} = o_i + R_i (a_i cos q_i, a_i sin q_i, d_i),
// R_{i+1} = R_i Rz(q_i) Rx(alpha_i).
__device__ void obb_joints_at(const ObbBuildParams& p, const double* ca, const double* sa,
                              const double* qa, const double* qb, double t, double* J) {
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double o[3] = {0, 0, 0};
  J[0] = J[1] = J[2] = 0.0;
  for (uint32_t i = 0; i < p.L; ++i) {
    const double q = qa[i] + t * (qb[i] - qa[i]);
    double st, ct;
    sincos(q, &st, &ct);
    const double v0 = p.a[i] * ct, v1 = p.a[i] * st, v2 = p.d[i];
    double on[3];
    for (int r = 0; r < 3; ++r) on[r] = o[r] + R[3 * r] * v0 + R[3 * r + 1] * v1 + R[3 * r + 2] * v2;
    for (int r = 0; r < 3; ++r) J[3 * (i + 1) + r] = on[r];
    const double A[9] = {ct, -st * ca[i], st * sa[i], st, ct * ca[i], -ct * sa[i], 0.0, sa[i], ca[i]};
    double Rn[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Rn[3 * r + c] = R[3 * r] * A[c] + R[3 * r + 1] * A[3 + c] + R[3 * r + 2] * A[6 + c];
    for (int k = 0; k < 9; ++k) R[k] = Rn[k];
    for (int r = 0; r < 3; ++r) o[r] = on[r];
  }
}

__device__ __forceinline__ double seg_point_dist_d(const double* p0, const double* p1,
                                                   const double* x) {
  double dd[3], w[3], c[3];
  for (int k = 0; k < 3; ++k) {
    dd[k] = p1[k] - p0[k];
    w[k] = x[k] - p0[k];
  }
  const double len2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
  double t = len2 > 0.0 ? (w[0] * dd[0] + w[1] * dd[1] + w[2] * dd[2]) / len2 : 0.0;
  t = fmin(fmax(t, 0.0), 1.0);
  for (int k = 0; k < 3; ++k) c[k] = p0[k] + t * dd[k] - x[k];
  return sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}

// Centre of inscribed sphere (fraction f of link i) at configuration m.
__device__ __forceinline__ void sphere_centre(const double* J, uint32_t stride, uint32_t i, double f,
                                              uint64_t m, double* v) {
  const double* jm = J + m * stride;
  for (int r = 0; r < 3; ++r) v[r] = jm[3 * i + r] + f * (jm[3 * (i + 1) + r] - jm[3 * i + r]);
}

// One warp per edge.  Lanes compute the joint positions of the edge's n
// configurations into the warp's scratch (and lane 0 those at q(1/2)).
// Pass 0: lane i < L fixes body i's box axes -- u1 the link direction at
// q(1/2), u2 the part normal to u1 of the link midpoint's displacement from
// q_a to q_b (the world axis least aligned with u1 when that is shorter than
// 1e-9 m), u3 = u1 x u2 -- then, body by body, the lanes project both link
// endpoints at every configuration on the axes, the warp reduces the ranges,
// and each half-extent grows by R_i plus half the largest motion of a link
// point between consecutive configurations (1/2 sum_{j<=i} |dq_j| rho_{j,i}).
// The box is stored in FP32 with its half-extents rounded up past the
// rounding of centre and axes.  Both passes then run the greedy shortcut of
// every (body, sphere) spline: from the last kept vertex j the warp tests,
// lanes over the dropped vertices m, whether the segment to candidate p + 1
// stays closer than R_i to all of them, and keeps extending while it does.
// Pass 0 counts the kept vertices; pass 1 writes them.
__global__ void __launch_bounds__(256) obb_build_kernel(const __grid_constant__ ObbBuildParams p) {
  __shared__ double s_ca[32], s_sa[32], s_len[32];
  __shared__ double s_mid[8][3 * 33];
  __shared__ double s_ax[8][32][9];
  if (threadIdx.x < p.L) {
    double sn, cs;
    sincos(p.alpha[threadIdx.x], &sn, &cs);
    s_ca[threadIdx.x] = cs;
    s_sa[threadIdx.x] = sn;
    s_len[threadIdx.x] = sqrt(p.a[threadIdx.x] * p.a[threadIdx.x] + p.d[threadIdx.x] * p.d[threadIdx.x]);
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t L = p.L, K = p.K, stride = 3 * (L + 1);
  double* J = p.scratch + warp * p.scratch_per_warp;
  double* mid = s_mid[wib];
  for (uint64_t e = warp; e < p.n_edges; e += nwarps) {
    const uint64_t n = p.soff[e + 1] - p.soff[e];
    const double* qa = p.qa + e * L;
    const double* qb = p.qb + e * L;
    for (uint64_t c = lane; c < n; c += 32)
      obb_joints_at(p, s_ca, s_sa, qa, qb, (double)c / (double)(n - 1), J + c * stride);
    if (lane == 0) obb_joints_at(p, s_ca, s_sa, qa, qb, 0.5, mid);
    __syncwarp();
    if (p.pass == 0) {
      if (lane < L) {
        const uint32_t i = lane;
        double* u = s_ax[wib][i];
        double len = 0.0;
        for (int r = 0; r < 3; ++r) {
          u[r] = mid[3 * (i + 1) + r] - mid[3 * i + r];
          len += u[r] * u[r];
        }
        len = sqrt(len);
        if (len < 1e-12) {
          u[0] = 1.0;
          u[1] = u[2] = 0.0;
        } else {
          for (int r = 0; r < 3; ++r) u[r] /= len;
        }
        const double* ja = J;
        const double* jb = J + (n - 1) * stride;
        double w[3];
        for (int r = 0; r < 3; ++r)
          w[r] = 0.5 * (jb[3 * i + r] + jb[3 * (i + 1) + r]) - 0.5 * (ja[3 * i + r] + ja[3 * (i + 1) + r]);
        const double wu = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
        double* v = u + 3;
        for (int r = 0; r < 3; ++r) v[r] = w[r] - wu * u[r];
        double l2 = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (l2 < 1e-9) {
          int kmin = 0;
          for (int k = 1; k < 3; ++k)
            if (fabs(u[k]) < fabs(u[kmin])) kmin = k;
          for (int r = 0; r < 3; ++r) v[r] = (r == kmin ? 1.0 : 0.0) - u[kmin] * u[r];
          l2 = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        }
        for (int r = 0; r < 3; ++r) v[r] /= l2;
        double* x = u + 6;
        x[0] = u[1] * v[2] - u[2] * v[1];
        x[1] = u[2] * v[0] - u[0] * v[2];
        x[2] = u[0] * v[1] - u[1] * v[0];
      }
      __syncwarp();
      double prefix = 0.0, sweep = 0.0;
      for (uint32_t i = 0; i < L; ++i) {
        prefix += fabs(qb[i] - qa[i]) / (double)(n - 1);
        sweep += s_len[i] * prefix;
        const double* u = s_ax[wib][i];
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (uint64_t c = lane; c < n; c += 32)
          for (uint32_t ep = i; ep <= i + 1; ++ep) {
            const double* pt = J + c * stride + 3 * ep;
            const double d0 = pt[0] - mid[3 * i], d1 = pt[1] - mid[3 * i + 1],
                         d2 = pt[2] - mid[3 * i + 2];
            for (int k = 0; k < 3; ++k) {
              const double s = d0 * u[3 * k] + d1 * u[3 * k + 1] + d2 * u[3 * k + 2];
              lo[k] = fmin(lo[k], s);
              hi[k] = fmax(hi[k], s);
            }
          }
        for (int off = 16; off; off >>= 1)
          for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
          }
        if (lane == 0) {
          const double grow = p.radius[i] + 0.5 * sweep;
          double c[3];
          for (int r = 0; r < 3; ++r) {
            c[r] = mid[3 * i + r];
            for (int k = 0; k < 3; ++k) c[r] += 0.5 * (lo[k] + hi[k]) * u[3 * k + r];
          }
          // FP32 rounding of centre and axes moves a box point by at most
          // ~6e-8 (|c| + sum h); 1e-6 m of extra half-extent covers it
          float4* ob = p.obb + 4 * (e * L + i);
          ob[0] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.0f);
          for (int k = 0; k < 3; ++k)
            ob[1 + k] = make_float4((float)u[3 * k], (float)u[3 * k + 1], (float)u[3 * k + 2],
                                    __double2float_ru(0.5 * (hi[k] - lo[k]) + grow + 1e-6));
        }
      }
    }
    // shortcut splines
    for (uint32_t i = 0; i < L; ++i) {
      const double R = p.radius[i];
      for (uint32_t s = 0; s < K; ++s) {
        const double f = ((double)s + 0.5) / (double)K;
        const uint64_t sp = (e * L + i) * K + s;
        const uint64_t off = p.pass == 1 ? p.spl_off[sp] : 0;
        uint32_t count = 0;
        double vj[3], vp[3], vm[3];
        auto emit = [&](uint64_t c) {
          if (p.pass == 1 && lane == 0) {
            double v[3];
            sphere_centre(J, stride, i, f, c, v);
            p.spl_v[off + count] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.0f);
          }
          ++count;
        };
        emit(0);
        uint64_t j = 0;
        while (j < n - 1) {
          uint64_t q = j + 1;
          while (q + 1 <= n - 1) {
            sphere_centre(J, stride, i, f, j, vj);
            sphere_centre(J, stride, i, f, q + 1, vp);
            bool ok = true;
            for (uint64_t m = j + 1 + lane; m <= q; m += 32) {
              sphere_centre(J, stride, i, f, m, vm);
              ok = ok && seg_point_dist_d(vj, vp, vm) < R;
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            ++q;
          }
          emit(q);
          j = q;
        }
        if (p.pass == 0 && lane == 0) p.spl_count[sp] = count;
      }
    }
    __syncwarp();
  }
}

// ===========================================================================
// offline grid
// ===========================================================================
__device__ __forceinline__ void obb_aabb(const float4* ob, float lo[3], float hi[3]) {
  const float4 c = ob[0], u1 = ob[1], u2 = ob[2], u3 = ob[3];
  const float ex = fabsf(u1.x) * u1.w + fabsf(u2.x) * u2.w + fabsf(u3.x) * u3.w;
  const float ey = fabsf(u1.y) * u1.w + fabsf(u2.y) * u2.w + fabsf(u3.y) * u3.w;
  const float ez = fabsf(u1.z) * u1.w + fabsf(u2.z) * u2.w + fabsf(u3.z) * u3.w;
  lo[0] = c.x - ex;
  lo[1] = c.y - ey;
  lo[2] = c.z - ez;
  hi[0] = c.x + ex;
  hi[1] = c.y + ey;
  hi[2] = c.z + ez;
}

__device__ __forceinline__ int cell_coord(float x, float o, float cell, uint32_t g) {
  const int c = (int)floorf((x - o) / cell);
  return c < 0 ? 0 : (c >= (int)g ? (int)g - 1 : c);
}

// Per block: min corner, max corner, and the sum of the boxes' largest
// AABB side (grid sizing); 8 floats per block.
__global__ void __launch_bounds__(256) obb_bounds_kernel(const float4* obb, uint64_t n_obb,
                                                         float* partial) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  float side = 0.0f;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n_obb;
       o += (uint64_t)gridDim.x * blockDim.x) {
    float a[3], b[3];
    obb_aabb(obb + 4 * o, a, b);
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], a[k]);
      hi[k] = fmaxf(hi[k], b[k]);
    }
    side += fmaxf(b[0] - a[0], fmaxf(b[1] - a[1], b[2] - a[2]));
  }
  __shared__ float s[8][8];
  for (int off = 16; off; off >>= 1) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
    }
    side += __shfl_xor_sync(0xffffffffu, side, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) {
      s[w][k] = lo[k];
      s[w][3 + k] = hi[k];
    }
    s[w][6] = side;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float r[7];
    for (int k = 0; k < 7; ++k) r[k] = s[0][k];
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) {
      for (int k = 0; k < 3; ++k) {
        r[k] = fminf(r[k], s[ww][k]);
        r[3 + k] = fmaxf(r[3 + k], s[ww][3 + k]);
      }
      r[6] += s[ww][6];
    }
    for (int k = 0; k < 7; ++k) partial[8 * blockIdx.x + k] = r[k];
    partial[8 * blockIdx.x + 7] = 0.0f;
  }
}

// Pass 0 counts, per cell, the boxes whose AABB meets it; pass 1 writes each
// box into every such cell's list as two float4: (AABB low corner, index
// bits) and (AABB high corner, 0), so that a query streams the AABBs of a
// cell's boxes contiguously and loads a box record only when the AABBs meet.
__global__ void __launch_bounds__(256) obb_grid_kernel(const __grid_constant__ ObbGridParams p) {
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < p.n_obb;
       o += (uint64_t)gridDim.x * blockDim.x) {
    float a[3], b[3];
    obb_aabb(p.obb + 4 * o, a, b);
    const int x0 = cell_coord(a[0], p.g.ox, p.g.cell, p.g.gx), x1 = cell_coord(b[0], p.g.ox, p.g.cell, p.g.gx);
    const int y0 = cell_coord(a[1], p.g.oy, p.g.cell, p.g.gy), y1 = cell_coord(b[1], p.g.oy, p.g.cell, p.g.gy);
    const int z0 = cell_coord(a[2], p.g.oz, p.g.cell, p.g.gz), z1 = cell_coord(b[2], p.g.oz, p.g.cell, p.g.gz);
    for (int z = z0; z <= z1; ++z)
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          const uint32_t cell = ((uint32_t)z * p.g.gy + (uint32_t)y) * p.g.gx + (uint32_t)x;
          if (p.pass == 0) {
            atomicAdd(&p.cell_count[cell], 1u);
          } else {
            const uint32_t k = atomicAdd(&p.cell_cursor[cell], 1u);
            const size_t at = 2 * ((size_t)p.cell_off[cell] + k);
            p.cell_items[at] = make_float4(a[0], a[1], a[2], __uint_as_float((uint32_t)o));
            p.cell_items[at + 1] = make_float4(b[0], b[1], b[2], 0.0f);
          }
        }
  }
}

// ===========================================================================
// per-pass queries
// ===========================================================================
// World AABB of a moved box's derived record (r1..r3 = axes, r4 = half-extents)
// grown by the margin.
__device__ __forceinline__ void box_aabb(const float4* B, float margin, float lo[3], float hi[3]) {
  const float4 c = B[0], a0 = B[1], a1 = B[2], a2 = B[3], h = B[4];
  const float ex = fabsf(a0.x) * h.x + fabsf(a1.x) * h.y + fabsf(a2.x) * h.z + margin;
  const float ey = fabsf(a0.y) * h.x + fabsf(a1.y) * h.y + fabsf(a2.y) * h.z + margin;
  const float ez = fabsf(a0.z) * h.x + fabsf(a1.z) * h.y + fabsf(a2.z) * h.z + margin;
  lo[0] = c.x - ex;
  lo[1] = c.y - ey;
  lo[2] = c.z - ez;
  hi[0] = c.x + ex;
  hi[1] = c.y + ey;
  hi[2] = c.z + ez;
}

// One block: the (moved box, cell, chunk) work items -- every chunk of
// boxes of each non-empty cell that a moved box's AABB meets (every non-empty
// cell without the spatial filter).  Chunks keep crowded cells (the ones near
// the robot's base hold most edges' first bodies) from landing on a single
// block.  A first sweep sums the boxes of the pass's (box, cell) pairs and
// picks the chunk size: the smallest power of two in [kObbChunkMin,
// kObbChunkMax] that gives at most target_items work items.  Fixed sizes
// showed why: on the 7-DOF roadmap chunks of 1,024 instead of 4,096 halved
// the query time (more items balance the blocks' long test chains), and on
// the large one chunks of 512 doubled it (per-item overhead).
__global__ void __launch_bounds__(256) obb_pairs_kernel(const __grid_constant__ ObbQueryParams p) {
  __shared__ unsigned long long s_total;
  __shared__ uint32_t s_chunk;
  if (threadIdx.x == 0) s_total = 0;
  __syncthreads();
  for (int sweep = 0; sweep < 2; ++sweep) {
    const uint32_t chunk = sweep ? s_chunk : 0u;
    unsigned long long mine = 0;
    for (uint32_t b = 0; b < p.C; ++b) {
      const float4* B = reinterpret_cast<const float4*>(p.boxes) + 6 * b;
      float lo[3], hi[3];
      box_aabb(B, p.margin, lo, hi);
      int x0 = 0, y0 = 0, z0 = 0, x1 = (int)p.g.gx - 1, y1 = (int)p.g.gy - 1, z1 = (int)p.g.gz - 1;
      if (p.filter) {
        x0 = cell_coord(lo[0], p.g.ox, p.g.cell, p.g.gx);
        x1 = cell_coord(hi[0], p.g.ox, p.g.cell, p.g.gx);
        y0 = cell_coord(lo[1], p.g.oy, p.g.cell, p.g.gy);
        y1 = cell_coord(hi[1], p.g.oy, p.g.cell, p.g.gy);
        z0 = cell_coord(lo[2], p.g.oz, p.g.cell, p.g.gz);
        z1 = cell_coord(hi[2], p.g.oz, p.g.cell, p.g.gz);
      }
      const uint32_t nx = (uint32_t)(x1 - x0 + 1), ny = (uint32_t)(y1 - y0 + 1);
      const uint32_t ncell = nx * ny * (uint32_t)(z1 - z0 + 1);
      for (uint32_t k = threadIdx.x; k < ncell; k += blockDim.x) {
        const uint32_t x = x0 + k % nx, y = y0 + (k / nx) % ny, z = z0 + k / (nx * ny);
        const uint32_t cell = (z * p.g.gy + y) * p.g.gx + x;
        const uint32_t items = p.cell_off[cell + 1] - p.cell_off[cell];
        if (items == 0) continue;
        if (sweep == 0) {
          mine += items;
          continue;
        }
        const uint32_t chunks = (items + chunk - 1) / chunk;
        const uint32_t slot = atomicAdd(&p.counters[0], chunks);
        for (uint32_t c = 0; c < chunks; ++c)
          if (slot + c < p.pair_cap) p.pairs[slot + c] = make_uint2(b | (c << 5), cell);
      }
    }
    if (sweep == 0) {
      if (mine) atomicAdd(&s_total, mine);
      __syncthreads();
      if (threadIdx.x == 0) {
        const uint64_t t = p.target_items ? p.target_items : 1u;
        const uint64_t want = (s_total + t - 1) / t;
        uint32_t c = kObbChunkMin;
        while (c < kObbChunkMax && c < want) c <<= 1;
        s_chunk = c;
        p.counters[2] = c;
      }
      __syncthreads();
    }
  }
}

// Does the FP32 box `ob` (centre, axes with half-extents) come within `margin`
// of the moved box B along every one of the 15 separating axes?  Any unit
// axis whose projections are disjoint proves separation, so a skipped
// (near-parallel) cross product can only make the answer "touch".
__device__ __forceinline__ bool obb_box_touch(const float4* ob, const float4* B, float margin) {
  float u[3][3], hu[3], b[3][3], hb[3], t[3];
  for (int k = 0; k < 3; ++k) {
    const float4 uk = ob[1 + k], bk = B[1 + k];
    u[k][0] = uk.x;
    u[k][1] = uk.y;
    u[k][2] = uk.z;
    hu[k] = uk.w;
    b[k][0] = bk.x;
    b[k][1] = bk.y;
    b[k][2] = bk.z;
  }
  hb[0] = B[4].x;
  hb[1] = B[4].y;
  hb[2] = B[4].z;
  t[0] = B[0].x - ob[0].x;
  t[1] = B[0].y - ob[0].y;
  t[2] = B[0].z - ob[0].z;
  auto sep = [&](const float* l) {
    float s = fabsf(t[0] * l[0] + t[1] * l[1] + t[2] * l[2]);
    for (int k = 0; k < 3; ++k) {
      s -= hu[k] * fabsf(u[k][0] * l[0] + u[k][1] * l[1] + u[k][2] * l[2]);
      s -= hb[k] * fabsf(b[k][0] * l[0] + b[k][1] * l[1] + b[k][2] * l[2]);
    }
    return s;
  };
  for (int k = 0; k < 3; ++k)
    if (sep(u[k]) > margin || sep(b[k]) > margin) return false;
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      float l[3] = {u[j][1] * b[k][2] - u[j][2] * b[k][1], u[j][2] * b[k][0] - u[j][0] * b[k][2],
                    u[j][0] * b[k][1] - u[j][1] * b[k][0]};
      const float len = sqrtf(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
      if (len < 1e-6f) continue;
      if (sep(l) > margin * len) return false;
    }
  return true;
}

__device__ __forceinline__ float seg_point_dist_f(float4 p0, float4 p1, float4 x) {
  const float dx = p1.x - p0.x, dy = p1.y - p0.y, dz = p1.z - p0.z;
  const float wx = x.x - p0.x, wy = x.y - p0.y, wz = x.z - p0.z;
  const float len2 = dx * dx + dy * dy + dz * dz;
  float t = len2 > 0.0f ? (wx * dx + wy * dy + wz * dz) / len2 : 0.0f;
  t = fminf(fmaxf(t, 0.0f), 1.0f);
  const float cx = fmaf(t, dx, p0.x) - x.x, cy = fmaf(t, dy, p0.y) - x.y, cz = fmaf(t, dz, p0.z) - x.z;
  return sqrtf(cx * cx + cy * cy + cz * cz);
}

// Persistent blocks take (box, cell, chunk) items.  A (OBB, box) pair is
// tested only in the cell holding the low corner of the two AABBs' overlap,
// so a pair listed in several cells counts once.  A touching pair
// (separation <= margin) sets the edge's touch bit for the pass position;
// then the body's splines are tested against the box's inner sphere (its
// centre, radius = smallest half-extent): a segment within radius - margin
// sets the hit bit.  (A spline lies inside its body's box, so only touching
// pairs can hit.)  Each stage compacts its survivors into a block queue, so
// that whole warps run the next test: the chunk's AABBs (one per thread),
// then the separating-axis tests of the pairs whose AABBs meet (one pair per
// thread), then the splines of the touching pairs (one spline per thread).
__global__ void __launch_bounds__(256) obb_query_kernel(const __grid_constant__ ObbQueryParams p) {
  __shared__ uint2 s_pair;
  __shared__ unsigned long long s_work[2];
  __shared__ uint32_t s_n[2];                  // pairs queued for SAT, touching pairs queued
  __shared__ uint32_t s_sat[kObbChunkMax];     // OBBs whose AABB meets the box's in this cell
  __shared__ uint32_t s_spl[kObbChunkMax];     // touching OBBs whose splines are tested
  const uint32_t total = min(p.counters[0], p.pair_cap);
  const uint32_t chunk = min(p.counters[2], kObbChunkMax);  // chosen by obb_pairs_kernel
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t k = atomicAdd(&p.counters[1], 1u);
      s_pair = k < total ? p.pairs[k] : make_uint2(0xffffffffu, 0u);
      s_work[0] = s_work[1] = 0;
      s_n[0] = s_n[1] = 0;
    }
    __syncthreads();
    const uint2 pr = s_pair;
    if (pr.x == 0xffffffffu) break;
    const uint32_t bpos = pr.x & 31u, cell = pr.y;
    const uint32_t k0 = p.cell_off[cell] + (pr.x >> 5) * chunk;
    const uint32_t k1 = min(p.cell_off[cell + 1], k0 + chunk);
    const float4* B = reinterpret_cast<const float4*>(p.boxes) + 6 * bpos;
    float blo[3], bhi[3];
    box_aabb(B, p.margin, blo, bhi);
    const float4 bc = B[0];
    const float rin = fminf(B[4].x, fminf(B[4].y, B[4].z)) - p.margin;
    const uint32_t bit = 1u << bpos;
    // 1. AABBs, and the cell that owns the pair
    for (uint32_t kb = k0; kb < k1; kb += blockDim.x) {
      const uint32_t k = kb + threadIdx.x;
      bool keep = false;
      uint32_t o = 0;
      if (k < k1) {
        const float4 ia = p.cell_items[2 * (size_t)k], ib = p.cell_items[2 * (size_t)k + 1];
        const float lo[3] = {ia.x, ia.y, ia.z}, hi[3] = {ib.x, ib.y, ib.z};
        if (!(lo[0] > bhi[0] || lo[1] > bhi[1] || lo[2] > bhi[2] || blo[0] > hi[0] ||
              blo[1] > hi[1] || blo[2] > hi[2])) {
          const uint32_t rx = cell_coord(fmaxf(lo[0], blo[0]), p.g.ox, p.g.cell, p.g.gx);
          const uint32_t ry = cell_coord(fmaxf(lo[1], blo[1]), p.g.oy, p.g.cell, p.g.gy);
          const uint32_t rz = cell_coord(fmaxf(lo[2], blo[2]), p.g.oz, p.g.cell, p.g.gz);
          keep = (rz * p.g.gy + ry) * p.g.gx + rx == cell;
          o = __float_as_uint(ia.w);
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      uint32_t at = 0;
      if (lane == 0 && m) at = atomicAdd(&s_n[0], (uint32_t)__popc(m));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (keep) s_sat[at + __popc(m & ((1u << lane) - 1u))] = o;
    }
    __syncthreads();
    const uint32_t n_sat = s_n[0];
    // 2. separating-axis tests
    for (uint32_t i = threadIdx.x; i < n_sat; i += blockDim.x) {
      const uint32_t o = s_sat[i];
      if (!obb_box_touch(p.obb + 4 * (size_t)o, B, p.margin)) continue;
      atomicOr(&p.edge_acc[2 * (uint64_t)(o / p.L) + 1], bit);
      if (rin > 0.0f) s_spl[atomicAdd(&s_n[1], 1u)] = o;
    }
    __syncthreads();
    const uint32_t n_spl = s_n[1];
    // 3. the touching bodies' splines against the box's inner sphere
    unsigned long long n_seg = 0;
    for (uint32_t i = threadIdx.x; i < n_spl * p.K; i += blockDim.x) {
      const uint32_t o = s_spl[i / p.K];
      const uint64_t sp = (uint64_t)o * p.K + (i % p.K);
      bool hit = false;
      for (uint64_t v = p.spl_off[sp]; v + 1 < p.spl_off[sp + 1]; ++v) {
        ++n_seg;
        if (seg_point_dist_f(p.spl_v[v], p.spl_v[v + 1], bc) <= rin) {
          hit = true;
          break;
        }
      }
      if (hit) atomicOr(&p.edge_acc[2 * (uint64_t)(o / p.L)], bit);
    }
    if (p.work) {
      if (threadIdx.x == 0) s_work[0] = n_sat;
      atomicAdd(&s_work[1], n_seg);
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicAdd(&p.work[0], s_work[0]);
        atomicAdd(&p.work[1], s_work[1]);
      }
    }
    __syncthreads();
  }
}

// ===========================================================================
// launchers
// ===========================================================================
cudaError_t launch_obb_build(const ObbBuildParams& p, uint32_t warps, cudaStream_t s) {
  if (p.n_edges == 0) return cudaSuccess;
  obb_build_kernel<<<(warps + 7) / 8, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_obb_bounds(const float4* obb, uint64_t n_obb, float* partial, uint32_t blocks,
                              cudaStream_t s) {
  if (n_obb == 0) return cudaSuccess;
  obb_bounds_kernel<<<blocks, 256, 0, s>>>(obb, n_obb, partial);
  return cudaGetLastError();
}

cudaError_t launch_obb_grid(const ObbGridParams& p, cudaStream_t s) {
  if (p.n_obb == 0) return cudaSuccess;
  const uint64_t want = (p.n_obb + 255) / 256;
  obb_grid_kernel<<<(unsigned)(want < 65535 ? want : 65535), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_obb_query(const ObbQueryParams& p, int num_sms, cudaStream_t s) {
  if (p.C == 0) return cudaSuccess;
  // the query grid: as many blocks as are resident at once; the chunk size
  // aims at about 4 work items per block
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, obb_query_kernel, 256, 0) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const uint32_t blocks = (uint32_t)num_sms * (uint32_t)per_sm;
  ObbQueryParams q = p;
  q.target_items = 4 * blocks;
  obb_pairs_kernel<<<1, 256, 0, s>>>(q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  obb_query_kernel<<<blocks, 256, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace rgg
