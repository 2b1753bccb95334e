/*
 * FP64 CPU oracle for the Red-Green-Gray (RGG) edge classification.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library; it
 * recomputes everything (sample counts, forward kinematics, inner and outer
 * spheres, box distances, labels) from the robot, the edge endpoints and the
 * box poses.
 *
 * It is deliberately plain: loops over edges, samples, links, spheres and
 * boxes in the order the definitions state them, every sphere tested against
 * every present box, no culling, no blocking.  The only parallelism is an
 * OpenMP loop over independent edges.
 *
 * Definitions followed (paper sections):
 *   - Sec. 3.2: an edge is discretised into configurations cfg(e) spaced by
 *     the resolution eps; FK maps a configuration to the robot's volume; an
 *     outer (inner) approximation is a superset (subset) of that volume.
 *   - Sec. 4.1: inner-approximation hit => red, outer-approximation miss =>
 *     green, otherwise gray.
 *   - Sec. 4.2: each body is under-approximated by inscribed spheres that are
 *     carried to every intermediate configuration (the vertices of the
 *     splines L_{e,i}).
 *   - Algorithm 1: per component, the set of obstacles it overlaps.
 * Readings where the paper is silent (geometry of the outer sphere, closed
 * contact, sample count, clearance) are stated next to each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LINKS 32

enum { OR_GREEN = 0, OR_GRAY = 1, OR_RED = 2 };

static int g_threads = 0; /* 0: OpenMP default */

void or_set_threads(int n) { g_threads = n; }

int or_max_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Number of configurations of an edge (Sec. 3.2: ||e||/eps configurations).
 * Reading: the length is the max-norm of the joint displacement, both
 * endpoints are included, and at least two samples are kept:
 *     n = max(2, ceil(max_j |qb_j - qa_j| / step) + 1).
 * Returns -1 for a non-positive or non-finite step.
 */
int64_t or_num_samples(int dof, const double* qa, const double* qb, double step) {
  if (!(step > 0.0) || !isfinite(step)) return -1;
  double m = 0.0;
  for (int j = 0; j < dof; ++j) {
    double v = fabs(qb[j] - qa[j]);
    if (v > m) m = v;
  }
  double c = ceil(m / step);
  int64_t n = (int64_t)c + 1;
  return n < 2 ? 2 : n;
}

/*
 * Forward kinematics of a serial arm in standard Denavit-Hartenberg form
 * (Sec. 3.2's FK, made concrete).  Joint i contributes the homogeneous
 * transform Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i); the base frame is the world
 * frame.  Output: the L+1 frame origins o_0 = 0, o_1, ..., o_L; link i is the
 * segment o_i -> o_{i+1} (0-based).
 */
void or_forward_kinematics(int L, const double* a, const double* alpha, const double* d,
                           const double* q, double* joints) {
  double T[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  joints[0] = joints[1] = joints[2] = 0.0;
  for (int i = 0; i < L; ++i) {
    double ct = cos(q[i]), st = sin(q[i]);
    double ca = cos(alpha[i]), sa = sin(alpha[i]);
    double A[4][4] = {{ct, -st * ca, st * sa, a[i] * ct},
                      {st, ct * ca, -ct * sa, a[i] * st},
                      {0.0, sa, ca, d[i]},
                      {0.0, 0.0, 0.0, 1.0}};
    double N[4][4];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        for (int m = 0; m < 4; ++m) s += T[r][m] * A[m][c];
        N[r][c] = s;
      }
    memcpy(T, N, sizeof(T));
    joints[3 * (i + 1) + 0] = T[0][3];
    joints[3 * (i + 1) + 1] = T[1][3];
    joints[3 * (i + 1) + 2] = T[2][3];
  }
}

/*
 * Euclidean distance from a point to a solid oriented box (Arvo's method in
 * the box frame).  box = [centre(3), R(9, row-major; columns are the box
 * axes in world coordinates), half-extents(3)].  p = R^T (x - centre);
 * d = || p - clamp(p, -h, h) ||, zero inside the box.
 */
double or_box_distance(const double* box, const double* x) {
  const double* c = box;
  const double* R = box + 3;
  const double* h = box + 12;
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    double p = 0.0;
    for (int m = 0; m < 3; ++m) p += R[3 * m + k] * (x[m] - c[m]);
    double cl = p < -h[k] ? -h[k] : (p > h[k] ? h[k] : p);
    double e = p - cl;
    s += e * e;
  }
  return sqrt(s);
}

/* Link length l_i = |o_{i+1} - o_i| = sqrt(a_i^2 + d_i^2) for a DH link. */
static double link_length(const double* a, const double* d, int i) {
  return sqrt(a[i] * a[i] + d[i] * d[i]);
}

/* Configuration at fraction t of the edge: q = qa + t (qb - qa). */
static void lerp_config(int L, const double* qa, const double* qb, double t, double* q) {
  for (int j = 0; j < L; ++j) q[j] = qa[j] + t * (qb[j] - qa[j]);
}

/*
 * Inner spheres at one configuration (Sec. 4.2): K spheres of radius R_i
 * inscribed in link i's capsule, centred on the link axis at fractions
 * (j + 1/2)/K of the segment o_i -> o_{i+1}.  Written as [L][K][4] (x,y,z,r).
 */
static void inner_spheres_at(int L, int K, const double* radius, const double* joints,
                             double* out) {
  for (int i = 0; i < L; ++i) {
    const double* o0 = joints + 3 * i;
    const double* o1 = joints + 3 * (i + 1);
    for (int j = 0; j < K; ++j) {
      double f = (j + 0.5) / (double)K;
      double* s = out + 4 * (i * K + j);
      s[0] = o0[0] + f * (o1[0] - o0[0]);
      s[1] = o0[1] + f * (o1[1] - o0[1]);
      s[2] = o0[2] + f * (o1[2] - o0[2]);
      s[3] = radius[i];
    }
  }
}

/*
 * Outer sphere of link i over one sample interval [q_k, q_{k+1}] (the outer
 * approximation of Sec. 3.2 / 4.2, here a sphere instead of the paper's OBB).
 * Reading: centre = midpoint of link i at q_mid = (q_k + q_{k+1})/2;
 *   radius = l_i/2 + R_i + 1/2 * sum_{j<=i} |dq_j| * rho_{j,i},
 *   rho_{j,i} = sum_{m=j..i} l_m   (a bound on the distance from joint j's
 * axis to any point of link i), dq = q_{k+1} - q_k.  Along the straight
 * joint-space path every point of link i moves at speed at most
 * sum_j |dq_j| dist(point, axis_j), so over half an interval it stays within
 * the last term of its position at q_mid; the first two terms enclose the
 * capsule at q_mid.  Written as [L][4].
 */
static void outer_spheres_at(int L, const double* a, const double* d, const double* radius,
                             const double* joints_mid, const double* dq, double* out) {
  for (int i = 0; i < L; ++i) {
    const double* o0 = joints_mid + 3 * i;
    const double* o1 = joints_mid + 3 * (i + 1);
    double sweep = 0.0;
    for (int j = 0; j <= i; ++j) {
      double rho = 0.0;
      for (int m = j; m <= i; ++m) rho += link_length(a, d, m);
      sweep += fabs(dq[j]) * rho;
    }
    double* s = out + 4 * i;
    s[0] = 0.5 * (o0[0] + o1[0]);
    s[1] = 0.5 * (o0[1] + o1[1]);
    s[2] = 0.5 * (o0[2] + o1[2]);
    s[3] = 0.5 * link_length(a, d, i) + radius[i] + 0.5 * sweep;
  }
}

/*
 * All spheres of one edge.  inner: [n][L][K][4]; outer: [n-1][L][4].
 * Sample k is q_k = qa + (k/(n-1)) (qb - qa), k = 0..n-1.  Returns n, or -1
 * if n exceeds cap_samples (the caller's buffer size) or the step is bad.
 */
int64_t or_edge_spheres(int L, const double* a, const double* alpha, const double* d,
                        const double* radius, int K, const double* qa, const double* qb,
                        double step, int64_t cap_samples, double* inner, double* outer) {
  if (L <= 0 || L > OR_MAX_LINKS) return -1;
  int64_t n = or_num_samples(L, qa, qb, step);
  if (n < 0 || n > cap_samples) return -1;
  double q[OR_MAX_LINKS], q1[OR_MAX_LINKS], qm[OR_MAX_LINKS], dq[OR_MAX_LINKS];
  double joints[3 * (OR_MAX_LINKS + 1)];
  for (int64_t k = 0; k < n; ++k) {
    lerp_config(L, qa, qb, (double)k / (double)(n - 1), q);
    or_forward_kinematics(L, a, alpha, d, q, joints);
    inner_spheres_at(L, K, radius, joints, inner + 4 * (size_t)(k * L * K));
    if (k + 1 < n) {
      lerp_config(L, qa, qb, (double)(k + 1) / (double)(n - 1), q1);
      for (int j = 0; j < L; ++j) {
        qm[j] = 0.5 * (q[j] + q1[j]);
        dq[j] = q1[j] - q[j];
      }
      or_forward_kinematics(L, a, alpha, d, qm, joints);
      outer_spheres_at(L, a, d, radius, joints, dq, outer + 4 * (size_t)(k * L));
    }
  }
  return n;
}

/*
 * Plain-definition classification of every edge against the current pose of
 * every present box (Sec. 4.1 labelling rule, with the per-box overlap sets of
 * Algorithm 1):
 *   hit_b(e)   <=> some inner sphere (x, r) of e has d(x, b) <= r
 *   touch_b(e) <=> some outer sphere (x, r) of e has d(x, b) <= r
 *   label = RED if some hit_b; else GREEN if no touch_b; else GRAY.
 * Contact counts (closed sets).  Clearance (how far the edge is from any
 * decision boundary): h_in = max over boxes and inner spheres of (r - d),
 * h_out = the same over outer spheres; kappa = h_in if h_in >= 0, else
 * min(-h_in, |h_out|).  With no present box, h_in = h_out = -inf.
 *
 * boxes: [n_boxes][15]; present: [n_boxes] (0/1) or NULL for all present.
 * Outputs may be NULL except labels.  hit_bits / touch_bits: [n_edges][W],
 * W = ceil(n_boxes/32), bit b of word b/32 for box b.
 * Returns 0, or -1 on a bad argument (sample count over max_samples, bad L).
 */
int or_classify(int L, const double* a, const double* alpha, const double* d,
                const double* radius, int K, int64_t n_edges, const double* qa,
                const double* qb, double step, int64_t max_samples, int n_boxes,
                const double* boxes, const uint8_t* present, uint8_t* labels, double* kappa,
                double* h_in_out, double* h_out_out, uint32_t* hit_bits, uint32_t* touch_bits) {
  if (L <= 0 || L > OR_MAX_LINKS || K <= 0 || n_boxes < 0) return -1;
  const int W = (n_boxes + 31) / 32;
  int bad = 0;
#pragma omp parallel num_threads(or_max_threads())
  {
    double* inner = (double*)malloc(sizeof(double) * 4 * (size_t)(max_samples * L * K));
    double* outer = (double*)malloc(sizeof(double) * 4 * (size_t)(max_samples * L));
    uint32_t* hb = (uint32_t*)calloc(W > 0 ? W : 1, sizeof(uint32_t));
    uint32_t* tb = (uint32_t*)calloc(W > 0 ? W : 1, sizeof(uint32_t));
#pragma omp for schedule(dynamic, 16)
    for (int64_t e = 0; e < n_edges; ++e) {
      const double* ea = qa + (size_t)e * L;
      const double* eb = qb + (size_t)e * L;
      int64_t n = or_edge_spheres(L, a, alpha, d, radius, K, ea, eb, step, max_samples,
                                  inner, outer);
      if (n < 0 || !inner || !outer) {
#pragma omp atomic write
        bad = 1;
        continue;
      }
      memset(hb, 0, sizeof(uint32_t) * (W > 0 ? W : 1));
      memset(tb, 0, sizeof(uint32_t) * (W > 0 ? W : 1));
      double h_in = -INFINITY, h_out = -INFINITY;
      for (int b = 0; b < n_boxes; ++b) {
        if (present && !present[b]) continue;
        const double* box = boxes + 15 * (size_t)b;
        for (int64_t s = 0; s < n * L * K; ++s) {
          const double* sp = inner + 4 * s;
          double v = sp[3] - or_box_distance(box, sp);
          if (v > h_in) h_in = v;
          if (v >= 0.0) hb[b >> 5] |= 1u << (b & 31);
        }
        for (int64_t s = 0; s < (n - 1) * L; ++s) {
          const double* sp = outer + 4 * s;
          double v = sp[3] - or_box_distance(box, sp);
          if (v > h_out) h_out = v;
          if (v >= 0.0) tb[b >> 5] |= 1u << (b & 31);
        }
      }
      int any_hit = 0, any_touch = 0;
      for (int w = 0; w < W; ++w) {
        any_hit |= hb[w] != 0;
        any_touch |= tb[w] != 0;
      }
      labels[e] = any_hit ? OR_RED : (any_touch ? OR_GRAY : OR_GREEN);
      if (kappa) kappa[e] = h_in >= 0.0 ? h_in : fmin(-h_in, fabs(h_out));
      if (h_in_out) h_in_out[e] = h_in;
      if (h_out_out) h_out_out[e] = h_out;
      if (hit_bits) memcpy(hit_bits + (size_t)e * W, hb, sizeof(uint32_t) * W);
      if (touch_bits) memcpy(touch_bits + (size_t)e * W, tb, sizeof(uint32_t) * W);
    }
    free(inner);
    free(outer);
    free(hb);
    free(tb);
  }
  return bad ? -1 : 0;
}

/*
 * Labels of edges whose approximations are given as sphere sets rather than
 * built from a robot (Sec. 4.1 applied to caller-supplied approximations):
 * edge e owns the inner spheres [in_off[e], in_off[e+1]) of inner[.][4] and
 * the outer spheres [out_off[e], out_off[e+1]) of outer[.][4], each sphere
 * (x, y, z, r).  Same rules as or_classify: box b is hit when some inner
 * sphere reaches it (d <= r), touched when some outer sphere does; red if
 * any box is hit, else green if none is touched, else gray; the clearance
 * kappa as in or_classify.  Outputs other than labels may be NULL.
 */
int or_classify_spheres(int64_t n_edges, const int64_t* in_off, const double* inner,
                        const int64_t* out_off, const double* outer, int n_boxes,
                        const double* boxes, const uint8_t* present, uint8_t* labels,
                        double* kappa, uint32_t* hit_bits, uint32_t* touch_bits) {
  if (n_edges < 0 || n_boxes < 0) return -1;
  const int W = (n_boxes + 31) / 32;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_max_threads())
  for (int64_t e = 0; e < n_edges; ++e) {
    double h_in = -INFINITY, h_out = -INFINITY;
    int any_hit = 0, any_touch = 0;
    for (int b = 0; b < n_boxes; ++b) {
      if (present && !present[b]) continue;
      const double* box = boxes + 15 * (size_t)b;
      int hit = 0, touch = 0;
      for (int64_t s = in_off[e]; s < in_off[e + 1]; ++s) {
        const double v = inner[4 * s + 3] - or_box_distance(box, inner + 4 * s);
        if (v > h_in) h_in = v;
        if (v >= 0.0) hit = 1;
      }
      for (int64_t s = out_off[e]; s < out_off[e + 1]; ++s) {
        const double v = outer[4 * s + 3] - or_box_distance(box, outer + 4 * s);
        if (v > h_out) h_out = v;
        if (v >= 0.0) touch = 1;
      }
      any_hit |= hit;
      any_touch |= touch;
      if (hit_bits && hit) hit_bits[(size_t)e * W + (b >> 5)] |= 1u << (b & 31);
      if (touch_bits && touch) touch_bits[(size_t)e * W + (b >> 5)] |= 1u << (b & 31);
    }
    labels[e] = any_hit ? OR_RED : (any_touch ? OR_GRAY : OR_GREEN);
    if (kappa) kappa[e] = h_in >= 0.0 ? h_in : fmin(-h_in, fabs(h_out));
  }
  return 0;
}

/*
 * Distance from the segment p0 -> p1 to a solid box: the minimum over
 * t in [0, 1] of d(p0 + t (p1 - p0), box).  That function is convex in t (a
 * convex distance composed with an affine map), so a golden-section search
 * on [0, 1] converges to its minimum; it runs until the bracket is below
 * 1e-12.  Used by the brute-force check below, not by the labels.
 */
double or_segment_box_distance(const double* p0, const double* p1, const double* box) {
  const double g = 0.5 * (sqrt(5.0) - 1.0);
  double lo = 0.0, hi = 1.0;
  double x[3];
#define OR_SEG_AT(t, out)                            \
  do {                                               \
    for (int m = 0; m < 3; ++m) x[m] = p0[m] + (t) * (p1[m] - p0[m]); \
    out = or_box_distance(box, x);                   \
  } while (0)
  double t1 = hi - g * (hi - lo), t2 = lo + g * (hi - lo), f1, f2;
  OR_SEG_AT(t1, f1);
  OR_SEG_AT(t2, f2);
  while (hi - lo > 1e-12) {
    if (f1 <= f2) {
      hi = t2;
      t2 = t1;
      f2 = f1;
      t1 = hi - g * (hi - lo);
      OR_SEG_AT(t1, f1);
    } else {
      lo = t1;
      t1 = t2;
      f1 = f2;
      t2 = lo + g * (hi - lo);
      OR_SEG_AT(t2, f2);
    }
  }
  double fa, fb, fm;
  OR_SEG_AT(0.0, fa);
  OR_SEG_AT(1.0, fb);
  OR_SEG_AT(0.5 * (lo + hi), fm);
#undef OR_SEG_AT
  double best = fm;
  if (f1 < best) best = f1;
  if (f2 < best) best = f2;
  if (fa < best) best = fa;
  if (fb < best) best = fb;
  return best;
}

/*
 * Brute-force check of one edge against the exact robot geometry: resample
 * the edge with `factor` times as many intervals (every original sample is
 * among the new ones), and at every configuration compute, for each link
 * capsule (segment o_i -> o_{i+1} with radius R_i) and each present box,
 * segdist - R_i.  Returns the minimum (<= 0 means the robot collides at some
 * resampled configuration), and writes to *argmin_t the edge fraction where it
 * occurs.  Returns +inf with no present box; NaN on a bad argument.
 */
double or_edge_dense_clearance(int L, const double* a, const double* alpha, const double* d,
                               const double* radius, const double* qa, const double* qb,
                               double step, int factor, int n_boxes, const double* boxes,
                               const uint8_t* present, double* argmin_t) {
  if (L <= 0 || L > OR_MAX_LINKS || factor < 1) return NAN;
  int64_t n = or_num_samples(L, qa, qb, step);
  if (n < 0) return NAN;
  int64_t m = (n - 1) * (int64_t)factor;
  double q[OR_MAX_LINKS], joints[3 * (OR_MAX_LINKS + 1)];
  double best = INFINITY, best_t = -1.0;
  for (int64_t k = 0; k <= m; ++k) {
    double t = (double)k / (double)m;
    lerp_config(L, qa, qb, t, q);
    or_forward_kinematics(L, a, alpha, d, q, joints);
    for (int b = 0; b < n_boxes; ++b) {
      if (present && !present[b]) continue;
      for (int i = 0; i < L; ++i) {
        double v = or_segment_box_distance(joints + 3 * i, joints + 3 * (i + 1),
                                           boxes + 15 * (size_t)b) -
                   radius[i];
        if (v < best) {
          best = v;
          best_t = t;
        }
      }
    }
  }
  if (argmin_t) *argmin_t = best_t;
  return best;
}

/* ========================================================================
 * The paper's own primitives (Sec. 4.2, Sec. 4.3): per (edge, body) OBB
 * outer approximations tested with the separating-axis test against the
 * obstacles' boxes, and shortcut splines through the inscribed spheres'
 * centres tested against the obstacles' inner spheres.
 * ======================================================================== */

static double dot3(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

static void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

/* Distance from point x to the segment p0 -> p1 (closest point by projection,
 * clamped to the segment). */
double or_segment_point_distance(const double* p0, const double* p1, const double* x) {
  double dd[3], w[3], c[3];
  for (int k = 0; k < 3; ++k) {
    dd[k] = p1[k] - p0[k];
    w[k] = x[k] - p0[k];
  }
  const double len2 = dot3(dd, dd);
  double t = len2 > 0.0 ? dot3(w, dd) / len2 : 0.0;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  for (int k = 0; k < 3; ++k) c[k] = p0[k] + t * dd[k] - x[k];
  return sqrt(dot3(c, c));
}

/*
 * Separation of two boxes along the 15 axes of the separating-axis test
 * (Sec. 4.3).  Each box is 15 doubles: centre, R (row-major; column k is
 * axis k), half-extents.  For a unit axis l the separation is
 *   |(c_B - c_A).l| - sum_k hA_k |a_k.l| - sum_k hB_k |b_k.l|,
 * over the 3 + 3 box axes and the 9 cross products a_j x b_k scaled to unit
 * length (a product shorter than 1e-6 comes from a parallel pair and is
 * skipped: the face axes cover it).  Returns the largest: > 0 means that axis
 * separates the boxes, <= 0 that no axis does and the boxes meet.
 */
double or_obb_separation(const double* A, const double* B) {
  double ax[3][3], bx[3][3], t[3];
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < 3; ++r) {
      ax[k][r] = A[3 + 3 * r + k];
      bx[k][r] = B[3 + 3 * r + k];
    }
  for (int r = 0; r < 3; ++r) t[r] = B[r] - A[r];
  double best = -INFINITY;
  double axes[15][3];
  int na = 0;
  for (int k = 0; k < 3; ++k) {
    for (int r = 0; r < 3; ++r) axes[na][r] = ax[k][r];
    ++na;
  }
  for (int k = 0; k < 3; ++k) {
    for (int r = 0; r < 3; ++r) axes[na][r] = bx[k][r];
    ++na;
  }
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      double w[3];
      cross3(ax[j], bx[k], w);
      const double len = sqrt(dot3(w, w));
      if (len < 1e-6) continue;
      for (int r = 0; r < 3; ++r) axes[na][r] = w[r] / len;
      ++na;
    }
  for (int i = 0; i < na; ++i) {
    const double* l = axes[i];
    double s = fabs(dot3(t, l));
    for (int k = 0; k < 3; ++k) {
      s -= A[12 + k] * fabs(dot3(ax[k], l));
      s -= B[12 + k] * fabs(dot3(bx[k], l));
    }
    if (s > best) best = s;
  }
  return best;
}

/* Joint positions of the edge's n configurations: joints[c][L+1][3]. */
static double* edge_joints(int L, const double* a, const double* alpha, const double* d,
                           const double* qa, const double* qb, int64_t n) {
  double* J = (double*)malloc(sizeof(double) * 3 * (size_t)(L + 1) * (size_t)n);
  if (!J) return NULL;
  double q[OR_MAX_LINKS];
  for (int64_t c = 0; c < n; ++c) {
    lerp_config(L, qa, qb, (double)c / (double)(n - 1), q);
    or_forward_kinematics(L, a, alpha, d, q, J + 3 * (size_t)(L + 1) * (size_t)c);
  }
  return J;
}

/*
 * OBB of each body over an edge (Sec. 4.2's outer approximation: an OBB
 * around the point cloud of the body's intermediates; the paper fits an
 * approximately optimal-volume box, here the axes come from the motion):
 *   u1 = link i's direction at the middle configuration q(1/2) (world x if
 *        the link has zero length);
 *   u2 = the part normal to u1 of the displacement of the link's midpoint
 *        from q_a to q_b; when shorter than 1e-9 m, the world axis least
 *        aligned with u1 (lowest index on ties) made normal to u1;
 *   u3 = u1 x u2.
 * The box spans the projections of both link endpoints at every
 * configuration of cfg(e) on those axes; each half-extent then grows by
 * R_i (the capsule) plus 1/2 sum_{j<=i} |dq_j| rho_{j,i}, half the largest
 * motion of a link point between consecutive configurations (the bound the
 * outer spheres use), so that the box holds the capsule over the whole edge.
 * obbs receives L boxes of 15 doubles (centre, R row-major with columns
 * u1 u2 u3, half-extents).  Returns n, or -1 on a bad argument.
 */
int64_t or_edge_obbs(int L, const double* a, const double* alpha, const double* d,
                     const double* radius, const double* qa, const double* qb, double step,
                     double* obbs) {
  if (L <= 0 || L > OR_MAX_LINKS) return -1;
  const int64_t n = or_num_samples(L, qa, qb, step);
  if (n < 2) return -1;
  double* J = edge_joints(L, a, alpha, d, qa, qb, n);
  if (!J) return -1;
  double q[OR_MAX_LINKS], jm[3 * (OR_MAX_LINKS + 1)];
  lerp_config(L, qa, qb, 0.5, q);
  or_forward_kinematics(L, a, alpha, d, q, jm);
  const double* ja = J;
  const double* jb = J + 3 * (size_t)(L + 1) * (size_t)(n - 1);
  double prefix = 0.0, sweep = 0.0;
  for (int i = 0; i < L; ++i) {
    double u[3][3];
    double len = 0.0;
    for (int r = 0; r < 3; ++r) {
      u[0][r] = jm[3 * (i + 1) + r] - jm[3 * i + r];
      len += u[0][r] * u[0][r];
    }
    len = sqrt(len);
    if (len < 1e-12) {
      u[0][0] = 1.0;
      u[0][1] = u[0][2] = 0.0;
    } else {
      for (int r = 0; r < 3; ++r) u[0][r] /= len;
    }
    double w[3];
    for (int r = 0; r < 3; ++r)
      w[r] = 0.5 * (jb[3 * i + r] + jb[3 * (i + 1) + r]) - 0.5 * (ja[3 * i + r] + ja[3 * (i + 1) + r]);
    double wu = dot3(w, u[0]);
    for (int r = 0; r < 3; ++r) u[1][r] = w[r] - wu * u[0][r];
    double l2 = sqrt(dot3(u[1], u[1]));
    if (l2 < 1e-9) {
      int kmin = 0;
      for (int k = 1; k < 3; ++k)
        if (fabs(u[0][k]) < fabs(u[0][kmin])) kmin = k;
      for (int r = 0; r < 3; ++r) u[1][r] = (r == kmin ? 1.0 : 0.0) - u[0][kmin] * u[0][r];
      l2 = sqrt(dot3(u[1], u[1]));
    }
    for (int r = 0; r < 3; ++r) u[1][r] /= l2;
    cross3(u[0], u[1], u[2]);
    /* motion bound: the same prefix sums as the outer spheres */
    prefix += fabs(qb[i] - qa[i]) / (double)(n - 1);
    sweep += link_length(a, d, i) * prefix;
    const double grow = radius[i] + 0.5 * sweep;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t c = 0; c < n; ++c) {
      const double* jc = J + 3 * (size_t)(L + 1) * (size_t)c;
      for (int e = 0; e < 2; ++e) {
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = jc[3 * (i + e) + r] - jm[3 * i + r];
        for (int k = 0; k < 3; ++k) {
          const double s = dot3(p, u[k]);
          if (s < lo[k]) lo[k] = s;
          if (s > hi[k]) hi[k] = s;
        }
      }
    }
    double* out = obbs + 15 * (size_t)i;
    for (int r = 0; r < 3; ++r) {
      double c = jm[3 * i + r];
      for (int k = 0; k < 3; ++k) c += 0.5 * (lo[k] + hi[k]) * u[k][r];
      out[r] = c;
      for (int k = 0; k < 3; ++k) out[3 + 3 * r + k] = u[k][r];
    }
    for (int k = 0; k < 3; ++k) out[12 + k] = 0.5 * (hi[k] - lo[k]) + grow;
  }
  free(J);
  return n;
}

/*
 * Shortcut splines (Sec. 4.2).  For body i and its inscribed sphere s (centre
 * at fraction (s + 1/2)/K of the link axis, radius R_i), the centre's
 * positions at the n configurations of cfg(e) form a polyline.  Vertices are
 * dropped greedily: from the last kept vertex j, the next kept vertex is the
 * largest p for which every vertex m strictly between j and p lies closer
 * than R_i to the segment v_j v_p (the paper's shortcut criterion), and the
 * last vertex is always kept.  verts receives, for (i, s) at slot
 * (i*K + s)*max_vertices, the kept vertices (x, y, z); counts[i*K + s] their
 * number.  Returns n, or -1 on a bad argument or too small a buffer.
 */
int64_t or_edge_splines(int L, const double* a, const double* alpha, const double* d,
                        const double* radius, int K, const double* qa, const double* qb,
                        double step, int64_t max_vertices, double* verts, int64_t* counts) {
  if (L <= 0 || L > OR_MAX_LINKS || K <= 0) return -1;
  const int64_t n = or_num_samples(L, qa, qb, step);
  if (n < 2 || max_vertices < n) return -1;
  double* J = edge_joints(L, a, alpha, d, qa, qb, n);
  double* V = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!J || !V) {
    free(J);
    free(V);
    return -1;
  }
  for (int i = 0; i < L; ++i)
    for (int s = 0; s < K; ++s) {
      const double f = ((double)s + 0.5) / (double)K;
      for (int64_t c = 0; c < n; ++c) {
        const double* jc = J + 3 * (size_t)(L + 1) * (size_t)c;
        for (int r = 0; r < 3; ++r)
          V[3 * c + r] = jc[3 * i + r] + f * (jc[3 * (i + 1) + r] - jc[3 * i + r]);
      }
      double* out = verts + 3 * (size_t)((size_t)(i * K + s) * (size_t)max_vertices);
      int64_t nk = 0;
      for (int r = 0; r < 3; ++r) out[r] = V[r];
      nk = 1;
      int64_t j = 0;
      while (j < n - 1) {
        int64_t p = j + 1;
        while (p + 1 <= n - 1) {
          int ok = 1;
          for (int64_t m = j + 1; m <= p && ok; ++m)
            ok = or_segment_point_distance(V + 3 * j, V + 3 * (p + 1), V + 3 * m) < radius[i];
          if (!ok) break;
          ++p;
        }
        for (int r = 0; r < 3; ++r) out[3 * nk + r] = V[3 * p + r];
        ++nk;
        j = p;
      }
      counts[i * K + s] = nk;
    }
  free(J);
  free(V);
  return n;
}

/*
 * Labels with the paper's primitives (Sec. 4.1 rule, Sec. 4.3 queries):
 * box b is touched when some body's OBB meets it (separation <= 0), hit when
 * some spline segment comes within its inner sphere (the largest inscribed
 * sphere: the box centre, radius its smallest half-extent; distance <= that
 * radius).  Red if any box is hit, else green if none is touched, else gray.
 * Clearance: h_in = max over segments and boxes of (radius - distance); sep =
 * the smallest |separation| over bodies and boxes; kappa = h_in when >= 0,
 * else min(-h_in, sep).  Outputs other than labels may be NULL.
 */
int or_classify_obb(int L, const double* a, const double* alpha, const double* d,
                    const double* radius, int K, int64_t n_edges, const double* qa,
                    const double* qb, double step, int64_t max_samples, int n_boxes,
                    const double* boxes, const uint8_t* present, uint8_t* labels,
                    double* kappa, uint32_t* hit_bits, uint32_t* touch_bits) {
  if (L <= 0 || L > OR_MAX_LINKS || K <= 0 || n_boxes < 0) return -1;
  const int W = (n_boxes + 31) / 32;
  int bad = 0;
#pragma omp parallel num_threads(or_max_threads())
  {
    double* obbs = (double*)malloc(sizeof(double) * 15 * (size_t)L);
    double* verts = (double*)malloc(sizeof(double) * 3 * (size_t)L * (size_t)K * (size_t)max_samples);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)L * (size_t)K);
#pragma omp for schedule(dynamic, 8)
    for (int64_t e = 0; e < n_edges; ++e) {
      const double* ea = qa + (size_t)e * L;
      const double* eb = qb + (size_t)e * L;
      if (!obbs || !verts || !cnt ||
          or_edge_obbs(L, a, alpha, d, radius, ea, eb, step, obbs) < 0 ||
          or_edge_splines(L, a, alpha, d, radius, K, ea, eb, step, max_samples, verts, cnt) < 0) {
#pragma omp atomic write
        bad = 1;
        continue;
      }
      double h_in = -INFINITY, sep_min = INFINITY;
      int any_hit = 0, any_touch = 0;
      for (int b = 0; b < n_boxes; ++b) {
        if (present && !present[b]) continue;
        const double* box = boxes + 15 * (size_t)b;
        double rb = box[12];
        if (box[13] < rb) rb = box[13];
        if (box[14] < rb) rb = box[14];
        int hit = 0, touch = 0;
        for (int i = 0; i < L; ++i) {
          const double sp = or_obb_separation(obbs + 15 * (size_t)i, box);
          if (fabs(sp) < sep_min) sep_min = fabs(sp);
          if (sp <= 0.0) touch = 1;
          for (int s = 0; s < K; ++s) {
            const double* v = verts + 3 * (size_t)((size_t)(i * K + s) * (size_t)max_samples);
            for (int64_t g = 0; g + 1 < cnt[i * K + s]; ++g) {
              const double h = rb - or_segment_point_distance(v + 3 * g, v + 3 * (g + 1), box);
              if (h > h_in) h_in = h;
              if (h >= 0.0) hit = 1;
            }
          }
        }
        any_hit |= hit;
        any_touch |= touch;
        if (hit_bits && hit) hit_bits[(size_t)e * W + (b >> 5)] |= 1u << (b & 31);
        if (touch_bits && touch) touch_bits[(size_t)e * W + (b >> 5)] |= 1u << (b & 31);
      }
      labels[e] = any_hit ? OR_RED : (any_touch ? OR_GRAY : OR_GREEN);
      if (kappa) kappa[e] = h_in >= 0.0 ? h_in : fmin(-h_in, sep_min);
    }
    free(obbs);
    free(verts);
    free(cnt);
  }
  return bad ? -1 : 0;
}
