/*
 * vt_oracle.c -- CPU oracle for discrete Voronoi, Laguerre and Johnson-Mehl
 * diagrams on a regular grid (Moulinec, arxiv 2201.13234).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * itself never does, and it shares no code with the library.
 *
 * What it computes (Section 2 and Appendix A of the paper), in the fixed-point
 * convention of this project (Q = 512 units per voxel):
 *   voxel centre          c_i = 512 k_i + 256              (k_i = voxel index)
 *   per-axis delta        d_i = c_i - q_i, and on a periodic axis the
 *                         L-periodic form of Appendix A, Eq. (dL):
 *                         d_i - N(d_i / L_i) L_i with N(x) = floor(x + 1/2)
 *   squared distance      D = sum_i d_i^2                      (exact int64)
 *   Voronoi score         D                                    (Eq. Voronoi_Cell, squared)
 *   Laguerre score        D - w_s                              (power distance, Section 2.3)
 *   Johnson-Mehl score    t_s + sqrt(D) / (512 v_s)            (Eq. JMAK2, IEEE double,
 *                         in that order: sqrt, then the divide, then the add)
 *   label(voxel)          the site with the smallest score; among equal scores
 *                         the lowest 0-based id (the strict "<" with increasing s
 *                         of Algorithms 1-3).
 *
 * Two independent ways of reaching that label:
 *   vto_brute    -- Algorithm 1: every voxel against every site
 *                   (vto_brute_scores: the same, with the best score per voxel).
 *   vto_twostep  -- Algorithms 2 and 3 and the Laguerre variant (Section 3):
 *                   step 1 visits, site by site in increasing order, the voxels
 *                   of the site's investigation ball and keeps the best score;
 *                   step 2 runs the brute force on the voxels no ball reached.
 *                   The ball of site s is the set of voxels whose score is at
 *                   most a threshold (r0^2 for Voronoi, G t0 for Laguerre, t0 for
 *                   Johnson-Mehl), which is the paper's ball written in the
 *                   score's own arithmetic, so the result equals the brute force
 *                   for any threshold.
 * and the paper's cost model that picks the threshold (Eqs. nstep12_3d,
 * v0_3d, v', nstep12_jmak, rs JM, rs Laguerre).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math, so
 * the Johnson-Mehl arithmetic is plain IEEE round-to-nearest with no fused
 * multiply-add).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { VTO_VORONOI = 0, VTO_LAGUERRE = 1, VTO_JM = 2 };

typedef struct {
  int nd;
  int64_t n[3];
  int64_t L[3];
  int per[3];
  int kind;
  int64_t ns;
  const int32_t *q; /* [ns][nd] */
  const int64_t *w; /* [ns] */
  const double *t;  /* [ns] */
  const double *v;  /* [ns] */
} vto_prob;

static int64_t floordiv64(int64_t a, int64_t b) {
  int64_t r = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) r--;
  return r;
}

static int64_t mod64(int64_t a, int64_t b) { return a - floordiv64(a, b) * b; }

/* Appendix A, Eq. (dL): the nearest-image delta on a periodic axis. */
static int64_t axis_delta(const vto_prob *P, int ax, int64_t c, int64_t q) {
  int64_t d = c - q;
  if (P->per[ax]) d -= floordiv64(2 * d + P->L[ax], 2 * P->L[ax]) * P->L[ax];
  return d;
}

static int64_t sq_dist(const vto_prob *P, const int64_t *c, int64_t s) {
  int64_t D = 0;
  for (int a = 0; a < P->nd; a++) {
    int64_t d = axis_delta(P, a, c[a], (int64_t)P->q[s * P->nd + a]);
    D += d * d;
  }
  return D;
}

/* Integer scores (Voronoi, Laguerre). */
static int64_t score_i(const vto_prob *P, const int64_t *c, int64_t s) {
  int64_t D = sq_dist(P, c, s);
  return P->kind == VTO_LAGUERRE ? D - P->w[s] : D;
}

/* Johnson-Mehl arrival time, Eq. (JMAK2): t_s + d / G with d in voxels. */
static double score_jm(const vto_prob *P, const int64_t *c, int64_t s) {
  double D = (double)sq_dist(P, c, s);
  double den = 512.0 * P->v[s];
  double d = sqrt(D);
  double x = d / den;
  return P->t[s] + x;
}

static int setup(vto_prob *P, int nd, const int64_t *n, int per_mask, int kind, int64_t ns,
                 const int32_t *q, const int64_t *w, const double *t, const double *v) {
  if (nd < 2 || nd > 3 || ns < 1) return 1;
  memset(P, 0, sizeof(*P));
  P->nd = nd;
  for (int a = 0; a < 3; a++) {
    P->n[a] = a < nd ? n[a] : 1;
    P->L[a] = 512 * P->n[a];
    P->per[a] = a < nd ? ((per_mask >> a) & 1) : 0;
  }
  P->kind = kind;
  P->ns = ns;
  P->q = q;
  P->w = w;
  P->t = t;
  P->v = v;
  if (kind == VTO_LAGUERRE && !w) return 1;
  if (kind == VTO_JM && (!t || !v)) return 1;
  return 0;
}

/* Voxel of flat index `idx` inside the slab [z0, z1) of the last axis. */
static void voxel_centre(const vto_prob *P, int64_t z0, int64_t idx, int64_t *c) {
  for (int a = 0; a < P->nd; a++) {
    int64_t k;
    if (a < P->nd - 1) {
      k = idx % P->n[a];
      idx /= P->n[a];
    } else {
      k = z0 + idx;
    }
    c[a] = 512 * k + 256;
  }
}

static int64_t slab_voxels(const vto_prob *P, int64_t z0, int64_t z1) {
  int64_t m = z1 - z0;
  for (int a = 0; a < P->nd - 1; a++) m *= P->n[a];
  return m;
}

/* The winner at centre c, and (when the pointers are given) its score: the
 * integer score for Voronoi and Laguerre, the arrival time for Johnson-Mehl. */
static void brute_one_scored(const vto_prob *P, const int64_t *c, int32_t *lab, int64_t *iscore,
                             double *dscore) {
  if (P->kind == VTO_JM) {
    double best = score_jm(P, c, 0);
    int64_t arg = 0;
    for (int64_t s = 1; s < P->ns; s++) {
      double sc = score_jm(P, c, s);
      if (sc < best) { best = sc; arg = s; }
    }
    *lab = (int32_t)arg;
    if (dscore) *dscore = best;
  } else {
    int64_t best = score_i(P, c, 0);
    int64_t arg = 0;
    for (int64_t s = 1; s < P->ns; s++) {
      int64_t sc = score_i(P, c, s);
      if (sc < best) { best = sc; arg = s; }
    }
    *lab = (int32_t)arg;
    if (iscore) *iscore = best;
  }
}

static void brute_one(const vto_prob *P, const int64_t *c, int32_t *lab) {
  brute_one_scored(P, c, lab, NULL, NULL);
}

/* Algorithm 1 on the slab z0 <= k_last < z1.  Labels are written for the slab
 * only, x fastest.  Returns 0 on success. */
int vto_brute(int nd, const int64_t *n, int per_mask, int kind, int64_t ns, const int32_t *q,
              const int64_t *w, const double *t, const double *v, int64_t z0, int64_t z1,
              int32_t *labels, int nthreads) {
  vto_prob P;
  if (setup(&P, nd, n, per_mask, kind, ns, q, w, t, v)) return 1;
  if (z0 < 0 || z1 > P.n[nd - 1] || z0 >= z1) return 2;
  int64_t m = slab_voxels(&P, z0, z1);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < m; i++) {
    int64_t c[3];
    voxel_centre(&P, z0, i, c);
    brute_one(&P, c, &labels[i]);
  }
  return 0;
}

/* Algorithm 1 on the slab, with each voxel's best score as well (the score
 * image the paper notes comes with the labels: for Voronoi the squared
 * Euclidean distance transform of the sites).  iscore (Voronoi, Laguerre) or
 * dscore (Johnson-Mehl) receives it, x fastest.  Returns 0 on success. */
int vto_brute_scores(int nd, const int64_t *n, int per_mask, int kind, int64_t ns,
                     const int32_t *q, const int64_t *w, const double *t, const double *v,
                     int64_t z0, int64_t z1, int32_t *labels, int64_t *iscore, double *dscore,
                     int nthreads) {
  vto_prob P;
  if (setup(&P, nd, n, per_mask, kind, ns, q, w, t, v)) return 1;
  if (z0 < 0 || z1 > P.n[nd - 1] || z0 >= z1) return 2;
  if (kind == VTO_JM ? !dscore : !iscore) return 3;
  int64_t m = slab_voxels(&P, z0, z1);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < m; i++) {
    int64_t c[3];
    voxel_centre(&P, z0, i, c);
    brute_one_scored(&P, c, &labels[i], iscore ? &iscore[i] : NULL, dscore ? &dscore[i] : NULL);
  }
  return 0;
}

/* Brute force at an explicit list of voxels (flat indices into the full grid). */
int vto_brute_points(int nd, const int64_t *n, int per_mask, int kind, int64_t ns,
                     const int32_t *q, const int64_t *w, const double *t, const double *v,
                     int64_t npts, const int64_t *flat, int32_t *labels, int nthreads) {
  vto_prob P;
  if (setup(&P, nd, n, per_mask, kind, ns, q, w, t, v)) return 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < npts; i++) {
    int64_t c[3];
    voxel_centre(&P, 0, flat[i], c);
    brute_one(&P, c, &labels[i]);
  }
  return 0;
}

/* Bound R (fixed-point units) on |d_i| for every voxel inside the ball of site
 * s; returns -1 when the ball is empty. */
static int64_t isqrt64(int64_t x) {
  if (x <= 0) return 0;
  int64_t r = (int64_t)sqrt((double)x);
  while (r * r > x) r--;
  while ((r + 1) * (r + 1) <= x) r++;
  return r;
}

static int64_t ball_axis_bound(const vto_prob *P, int64_t s, int64_t thr_i, double thr_d) {
  if (P->kind == VTO_VORONOI) return thr_i < 0 ? -1 : isqrt64(thr_i);
  if (P->kind == VTO_LAGUERRE) {
    int64_t r2 = thr_i + P->w[s];
    return r2 < 0 ? -1 : isqrt64(r2);
  }
  /* Johnson-Mehl: arrival >= t_s, so the ball is empty when t_s > t0.  Otherwise
   * sqrt(D) <= (t0 - t_s) * 512 v_s up to rounding; the margin below is generous
   * because each voxel of the box is then tested exactly. */
  double t = P->t[s];
  if (!(t <= thr_d)) return -1;
  double r = (thr_d - t) * 512.0 * P->v[s];
  r = r * (1.0 + 1e-9) + 4.0;
  if (r > 4.0e15) r = 4.0e15;
  return (int64_t)r;
}

/* Voxel index range of the ball along axis a; returns the count and fills
 * idx[] with the wrapped indices (each at most once). */
static int64_t axis_range(const vto_prob *P, int a, int64_t q, int64_t R, int64_t *idx) {
  int64_t lo = -floordiv64(-(q - R - 256), 512); /* ceil((q-R-256)/512) */
  int64_t hi = floordiv64(q + R - 256, 512);
  if (hi < lo) return 0;
  int64_t n = P->n[a], m = 0;
  if (P->per[a]) {
    if (hi - lo + 1 >= n) {
      for (int64_t k = 0; k < n; k++) idx[m++] = k;
    } else {
      for (int64_t k = lo; k <= hi; k++) idx[m++] = mod64(k, n);
    }
  } else {
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    for (int64_t k = lo; k <= hi; k++) idx[m++] = k;
  }
  return m;
}

/* Algorithms 2/3 (and the Laguerre variant) on the slab z0 <= k_last < z1.
 * thr_i is the Voronoi/Laguerre ball threshold on the integer score, thr_d the
 * Johnson-Mehl threshold t0 on the arrival time.  counts (nullable) receives
 * {distance evaluations inside balls (step 1), distance evaluations of step 2,
 *  voxels left for step 2, voxels tested in ball bounding boxes}. */
int vto_twostep(int nd, const int64_t *n, int per_mask, int kind, int64_t ns, const int32_t *q,
                const int64_t *w, const double *t, const double *v, int64_t thr_i, double thr_d,
                int64_t z0, int64_t z1, int32_t *labels, int64_t *counts, int nthreads) {
  vto_prob P;
  if (setup(&P, nd, n, per_mask, kind, ns, q, w, t, v)) return 1;
  if (z0 < 0 || z1 > P.n[nd - 1] || z0 >= z1) return 2;
  const int last = nd - 1;
  const int64_t m = slab_voxels(&P, z0, z1);
  const int64_t plane = m / (z1 - z0);
  int is_jm = kind == VTO_JM;
  int64_t *Di = NULL;
  double *Dd = NULL;
  unsigned char *hit = (unsigned char *)calloc((size_t)m, 1);
  if (is_jm)
    Dd = (double *)malloc(sizeof(double) * (size_t)m);
  else
    Di = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  if (!hit || (!Dd && !Di)) {
    free(hit); free(Dd); free(Di);
    return 3;
  }
  int64_t c_step1 = 0, c_step2 = 0, c_left = 0, c_tested = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif

  /* Step 1.  Each thread owns a contiguous range of the last axis and visits
   * every site in increasing order, so no two threads touch the same voxel and
   * the strict "<" keeps the lowest id among equal scores. */
#pragma omp parallel reduction(+ : c_step1, c_tested)
  {
    int nth = 1, tid = 0;
#ifdef _OPENMP
    nth = omp_get_num_threads();
    tid = omp_get_thread_num();
#endif
    int64_t span = z1 - z0;
    int64_t za = z0 + span * tid / nth, zb = z0 + span * (tid + 1) / nth;
    int64_t nmax = P.n[0];
    for (int a = 1; a < 3; a++) if (P.n[a] > nmax) nmax = P.n[a];
    int64_t *ix[3];
    int64_t *d2[3];
    for (int a = 0; a < 3; a++) {
      ix[a] = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
      d2[a] = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
    }
    int64_t cnt[3];
    for (int64_t s = 0; s < ns && za < zb; s++) {
      int64_t R = ball_axis_bound(&P, s, thr_i, thr_d);
      if (R < 0) continue;
      int empty = 0;
      for (int a = 0; a < nd; a++) {
        int64_t qa = (int64_t)q[s * nd + a];
        cnt[a] = axis_range(&P, a, qa, R, ix[a]);
        if (a == last) { /* keep this thread's part of the slab only */
          int64_t k2 = 0;
          for (int64_t k = 0; k < cnt[a]; k++)
            if (ix[a][k] >= za && ix[a][k] < zb) ix[a][k2++] = ix[a][k];
          cnt[a] = k2;
        }
        if (cnt[a] == 0) { empty = 1; break; }
        for (int64_t k = 0; k < cnt[a]; k++) {
          int64_t d = axis_delta(&P, a, 512 * ix[a][k] + 256, qa);
          d2[a][k] = d * d;
        }
      }
      if (empty) continue;
      int64_t c1 = nd == 3 ? cnt[1] : 1;
      int64_t c2 = cnt[last];
      for (int64_t kz = 0; kz < c2; kz++) {
        for (int64_t ky = 0; ky < c1; ky++) {
          int64_t base;
          int64_t dyz;
          if (nd == 3) {
            base = ((ix[2][kz] - z0) * P.n[1] + ix[1][ky]) * P.n[0];
            dyz = d2[1][ky] + d2[2][kz];
          } else {
            base = (ix[1][kz] - z0) * P.n[0];
            dyz = d2[1][kz];
          }
          for (int64_t kx = 0; kx < cnt[0]; kx++) {
            int64_t k = base + ix[0][kx];
            int64_t D = d2[0][kx] + dyz;
            c_tested++;
            if (is_jm) {
              double a = t[s] + sqrt((double)D) / (512.0 * v[s]);
              if (a <= thr_d) {
                c_step1++;
                if (!hit[k] || a < Dd[k]) { Dd[k] = a; labels[k] = (int32_t)s; hit[k] = 1; }
              }
            } else {
              int64_t sc = kind == VTO_LAGUERRE ? D - w[s] : D;
              if (sc <= thr_i) {
                c_step1++;
                if (!hit[k] || sc < Di[k]) { Di[k] = sc; labels[k] = (int32_t)s; hit[k] = 1; }
              }
            }
          }
        }
      }
    }
    for (int a = 0; a < 3; a++) { free(ix[a]); free(d2[a]); }
  }

  /* Step 2: brute force on the voxels that no ball reached. */
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : c_left)
  for (int64_t i = 0; i < m; i++) {
    if (hit[i]) continue;
    int64_t c[3];
    voxel_centre(&P, z0, i, c);
    brute_one(&P, c, &labels[i]);
    c_left++;
  }
  c_step2 = c_left * ns;
  (void)plane;
  if (counts) {
    counts[0] = c_step1;
    counts[1] = c_step2;
    counts[2] = c_left;
    counts[3] = c_tested;
  }
  free(hit); free(Dd); free(Di);
  return 0;
}

/* ---------------- cost model (Section 3.2.3 and 3.3.2) ---------------- */

static const double VTO_PI = 3.14159265358979323846;
static double ball_coeff(int nd) { return nd == 2 ? VTO_PI : 4.0 * VTO_PI / 3.0; }

/* Eq. (v0_3d): the ball volume fraction v0/V that minimises Eq. (nstep12_3d). */
double vto_v0_fraction(int64_t ns) {
  if (ns < 2) return 1.0;
  return -expm1(-log((double)ns) / (double)(ns - 1));
}

/* Eq. (nstep12_3d) divided by N_v N_s: expected distance evaluations per voxel
 * and per site for a ball volume fraction f = v0/V. */
double vto_voronoi_cost(int64_t ns, double f) { return f + pow(1.0 - f, (double)ns); }

/* Radius r0 (voxels) of the Voronoi investigation ball on a grid of nd dims. */
double vto_voronoi_r0(int nd, const int64_t *n, int64_t ns) {
  double V = 1.0;
  for (int a = 0; a < nd; a++) V *= (double)n[a];
  double v0 = vto_v0_fraction(ns) * V;
  return pow(v0 / ball_coeff(nd), 1.0 / nd);
}

/* Ball volume (voxels^d) of site s at parameter x: Johnson-Mehl x = t0 with
 * radius v_s (t0 - t_s)^+ (Eq. rs JM); Laguerre x = G t0 in voxel^2 with
 * r_s^2 = x + w_s / 512^2 (Eq. rs Laguerre with G t_s = -r_s^2). */
static double ball_volume(int nd, int kind, double x, double ts, double vs, double ws) {
  double r;
  if (kind == VTO_JM) {
    r = vs * (x - ts);
    if (r <= 0) return 0.0;
  } else {
    double r2 = x + ws / (512.0 * 512.0);
    if (r2 <= 0) return 0.0;
    r = sqrt(r2);
  }
  return ball_coeff(nd) * pow(r, (double)nd);
}

/* Eq. (nstep12_jmak) divided by N_v, with v'_s = min(V, v_s) (Eq. v'). */
double vto_growth_cost(int nd, const int64_t *n, int kind, int64_t ns, const int64_t *w,
                       const double *t, const double *v, double x) {
  double V = 1.0;
  for (int a = 0; a < nd; a++) V *= (double)n[a];
  double s1 = 0.0, logp = 0.0;
  int zero = 0;
  for (int64_t s = 0; s < ns; s++) {
    double vs = ball_volume(nd, kind, x, kind == VTO_JM ? t[s] : 0.0,
                            kind == VTO_JM ? v[s] : 0.0, kind == VTO_JM ? 0.0 : (double)w[s]);
    double f = vs / V;
    if (f >= 1.0) { f = 1.0; zero = 1; }
    s1 += f;
    if (!zero) logp += log1p(-f);
  }
  return s1 + (zero ? 0.0 : (double)ns * exp(logp));
}

/* Search interval of the growth threshold (end of Section 3.3.2 and of 3.4). */
static void growth_bounds(int nd, const int64_t *n, int per_mask, int kind, int64_t ns,
                          const int64_t *w, const double *t, const double *v, double *lo,
                          double *hi) {
  double sum_l2 = 0.0;
  for (int a = 0; a < nd; a++) sum_l2 += (double)n[a] * (double)n[a];
  int periodic = (per_mask & ((1 << nd) - 1)) != 0;
  if (kind == VTO_JM) {
    double tmin = t[0], vmin = v[0];
    for (int64_t s = 1; s < ns; s++) {
      if (t[s] < tmin) tmin = t[s];
      if (v[s] < vmin) vmin = v[s];
    }
    *lo = tmin;
    *hi = tmin + (periodic ? 0.5 : 1.0) * sqrt(sum_l2) / vmin;
  } else {
    double wmax = (double)w[0];
    for (int64_t s = 1; s < ns; s++)
      if ((double)w[s] > wmax) wmax = (double)w[s];
    *lo = -wmax / (512.0 * 512.0);
    *hi = *lo + (periodic ? 0.25 : 1.0) * sum_l2;
  }
}

/* Minimiser of Eq. (nstep12_jmak) over its interval: a uniform scan followed
 * by golden-section refinement of the best bracket (the paper only asks for a
 * one-dimensional search, e.g. a dichotomy). */
double vto_growth_threshold(int nd, const int64_t *n, int per_mask, int kind, int64_t ns,
                            const int64_t *w, const double *t, const double *v) {
  double lo, hi;
  growth_bounds(nd, n, per_mask, kind, ns, w, t, v, &lo, &hi);
  const int G = 128;
  int best = 0;
  double bestc = INFINITY;
  for (int i = 0; i <= G; i++) {
    double x = lo + (hi - lo) * i / G;
    double c = vto_growth_cost(nd, n, kind, ns, w, t, v, x);
    if (c < bestc) { bestc = c; best = i; }
  }
  double a = lo + (hi - lo) * (best > 0 ? best - 1 : 0) / G;
  double b = lo + (hi - lo) * (best < G ? best + 1 : G) / G;
  const double gr = 0.6180339887498949;
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double f1 = vto_growth_cost(nd, n, kind, ns, w, t, v, x1);
  double f2 = vto_growth_cost(nd, n, kind, ns, w, t, v, x2);
  for (int it = 0; it < 40; it++) {
    if (f1 < f2) {
      b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a);
      f1 = vto_growth_cost(nd, n, kind, ns, w, t, v, x1);
    } else {
      a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a);
      f2 = vto_growth_cost(nd, n, kind, ns, w, t, v, x2);
    }
  }
  double xm = 0.5 * (a + b);
  return vto_growth_cost(nd, n, kind, ns, w, t, v, xm) <= bestc ? xm : lo + (hi - lo) * best / G;
}
