/*
 * tpct_oracle.c -- plain FP64 CPU oracle of TPC sector track finding.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); the CUDA
 * library never calls it and shares no code with it.
 *
 * The paper (Tables 1-3) names "TPC Processing (Tracking)" as the dominant
 * reconstruction step but gives no algorithm; this file follows the stated
 * reading of the steps, one function per step, in the order they run:
 *   S1 row lists (the oracle's own search structure: clusters of a row sorted
 *      by y, scanned between two binary-searched bounds),
 *   S2 neighbour finding (best straight-line pair in rows r-1, r+1),
 *   S3 removal of non-reciprocal links,
 *   S4 start hits (chain bottoms with a chain of at least three hits),
 *   S5 tracklet growth with a Kalman filter, upward then downward,
 *   S6 selection by owned-cluster count and shared fraction,
 *   S7 iterated FP64 refit of the owned clusters.
 * Matrices are full 5x5 row-major arrays and every product is a plain loop.
 * Each decision that compares a computed value with a cut or with another
 * candidate logs its relative margin; the parity checker uses these margins.
 */
#include "tpct_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KB_PER_TESLA 0.299792458e-2   /* curvature [1/cm] per (q/pT [c/GeV]) per T */
#define EXT 1.001                      /* windows widened by this factor for margin logging */

/* ------------------------------------------------------------ growable arrays */
typedef struct { char* p; int64_t n, cap; size_t es; } vec;

static void vec_init(vec* v, size_t es) { v->p = NULL; v->n = 0; v->cap = 0; v->es = es; }
static int vec_push(vec* v, const void* e) {
  if (v->n == v->cap) {
    int64_t nc = v->cap ? 2 * v->cap : 256;
    char* q = (char*)realloc(v->p, (size_t)nc * v->es);
    if (!q) return 1;
    v->p = q; v->cap = nc;
  }
  memcpy(v->p + (size_t)v->n * v->es, e, v->es);
  v->n++;
  return 0;
}
static void vec_free(vec* v) { free(v->p); v->p = NULL; v->n = v->cap = 0; }

/* ------------------------------------------------------------ result */
struct orc_result {
  int64_t n;
  int n_rows;
  int32_t *up, *down, *upc, *downc;
  double* nf_margin;
  uint32_t* weight;
  vec a[ORC_N_ARRAYS];     /* tracklet and track arrays, indexed by the ORC_* enum */
};

static int is_per_cluster(int w) {
  return w == ORC_UP || w == ORC_DOWN || w == ORC_UPC || w == ORC_DOWNC || w == ORC_NF_MARGIN ||
         w == ORC_WEIGHT;
}

int64_t orc_count(const orc_result* r, int w) {
  if (!r || w < 0 || w >= ORC_N_ARRAYS) return -1;
  if (is_per_cluster(w)) return r->n;
  return r->a[w].n;
}

const void* orc_array(const orc_result* r, int w) {
  if (!r || w < 0 || w >= ORC_N_ARRAYS) return NULL;
  switch (w) {
    case ORC_UP: return r->up;
    case ORC_DOWN: return r->down;
    case ORC_UPC: return r->upc;
    case ORC_DOWNC: return r->downc;
    case ORC_NF_MARGIN: return r->nf_margin;
    case ORC_WEIGHT: return r->weight;
    default: return r->a[w].p;
  }
}

void orc_free(orc_result* r) {
  if (!r) return;
  free(r->up); free(r->down); free(r->upc); free(r->downc); free(r->nf_margin); free(r->weight);
  for (int i = 0; i < ORC_N_ARRAYS; ++i) vec_free(&r->a[i]);
  free(r);
}

/* ------------------------------------------------------------ small helpers */
static double rel_margin(double a, double cut) {
  double d = fabs(a - cut);
  double s = fabs(cut);
  return s > 0.0 ? d / s : d;
}
static double dmin(double a, double b) { return a < b ? a : b; }

/* cluster resolution: linear in drift length d = clamp(z_max - |z|, 0, z_max) */
static double sigma_at(const orc_geometry* g, const orc_cuts* c, double z) {
  double d = g->z_max - fabs(z);
  if (d < 0.0) d = 0.0;
  if (d > g->z_max) d = g->z_max;
  return c->sig_readout + (c->sig_cathode - c->sig_readout) * d / g->z_max;
}

/* asin(h)/h and its derivative; below |h| = 0.01 by the Taylor series of
 * asin (coefficients (2n)! / (4^n (n!)^2 (2n+1))), truncation < 1e-25 */
static double asin_over(double h) {
  if (fabs(h) < 1e-2) {
    double u = h * h;
    return 1.0 + u * (1.0 / 6.0 + u * (3.0 / 40.0 + u * (5.0 / 112.0 + u * (35.0 / 1152.0 + u * (63.0 / 2816.0)))));
  }
  return asin(h) / h;
}
static double asin_over_deriv(double h) {
  if (fabs(h) < 1e-2) {
    double u = h * h;
    return h * (2.0 / 6.0 + u * (4.0 * 3.0 / 40.0 + u * (6.0 * 5.0 / 112.0 + u * (8.0 * 35.0 / 1152.0 + u * (10.0 * 63.0 / 2816.0)))));
  }
  return (1.0 / sqrt(1.0 - h * h) - asin(h) / h) / h;
}

/* ------------------------------------------------------------ propagation */
/* Exact helix in x: s1 = s0 + rho dx (rho = -k_B q/pT); the chord's slope is the
 * tangent of the mean direction, dy = dx (s0+s1)/(c0+c1); the arc length of a
 * chord L is L asin(h)/h with h = rho L / 2; dz = tan(lambda) * arc.  L carries
 * the sign of dx, so transport towards smaller x has a negative path length. */
static int propagate_m(double bz, double s_max, double x0, double x1, double p[5], double F[25],
                       double* margin) {
  double kb = KB_PER_TESLA * bz;
  double dx = x1 - x0;
  double rho = -kb * p[4];
  double s0 = p[2];
  double s1 = s0 + rho * dx;
  if (margin) *margin = dmin(*margin, dmin(rel_margin(fabs(s0), s_max), rel_margin(fabs(s1), s_max)));
  if (fabs(s0) >= s_max || fabs(s1) >= s_max) return 1;
  double c0 = sqrt(1.0 - s0 * s0), c1 = sqrt(1.0 - s1 * s1);
  double A = s0 + s1, B = c0 + c1;
  double dy = dx * A / B;
  double L = copysign(sqrt(dx * dx + dy * dy), dx);
  double h = 0.5 * rho * L;
  double g = asin_over(h);
  double arc = L * g;
  double dz = p[3] * arc;
  if (F) {
    for (int i = 0; i < 25; ++i) F[i] = 0.0;
    for (int i = 0; i < 5; ++i) F[i * 5 + i] = 1.0;
    /* s1 */
    F[2 * 5 + 4] = -kb * dx;
    /* dy = dx A / B, with A, B functions of (s0, q/pT) */
    double dA_ds0 = 2.0, dA_dq = -kb * dx;
    double dB_ds0 = -s0 / c0 - s1 / c1;
    double dB_dq = -(s1 / c1) * (-kb * dx);
    double ddy_ds0 = dx * (dA_ds0 * B - A * dB_ds0) / (B * B);
    double ddy_dq = dx * (dA_dq * B - A * dB_dq) / (B * B);
    F[0 * 5 + 2] = ddy_ds0;
    F[0 * 5 + 4] = ddy_dq;
    /* arc = L g(h), h = rho L / 2, L = sqrt(dx^2 + dy^2) */
    double gp = asin_over_deriv(h);
    double darc_dL = g + h * gp;
    double darc_drho = 0.5 * L * L * gp;
    double dL_ddy = L != 0.0 ? dy / L : 0.0;
    double darc_ds0 = darc_dL * dL_ddy * ddy_ds0;
    double darc_dq = darc_dL * dL_ddy * ddy_dq + darc_drho * (-kb);
    F[1 * 5 + 2] = p[3] * darc_ds0;
    F[1 * 5 + 3] = arc;
    F[1 * 5 + 4] = p[3] * darc_dq;
  }
  p[0] += dy;
  p[1] += dz;
  p[2] = s1;
  return 0;
}

int orc_propagate(double bz, double s_max, double x0, double x1, double p[5], double F[25]) {
  return propagate_m(bz, s_max, x0, x1, p, F, NULL);
}

/* Rotation of the local frame by dalpha.  A point (x, y) becomes
 * (x cos d + y sin d, -x sin d + y cos d) and the direction angle phi becomes
 * phi - d.  Perturbing y at fixed x moves the point off the new plane x' =
 * const; sliding back along the track by dl = -sin(d) dy / cos(phi') gives
 * dy' = dy cos(phi)/cos(phi'), dz' = dz - t sin(d) dy / cos(phi'), and turns
 * the direction by rho dl, dsin(phi') = -rho sin(d) dy.  A change of sin(phi)
 * at a fixed point changes phi' equally: dsin(phi') = cos(phi')/cos(phi) ds. */
int orc_rotate(double bz, double s_max, double dalpha, double x0, const double p0[5], double* x1,
               double p1[5], double F[25]) {
  double ca = cos(dalpha), sa = sin(dalpha);
  double s = p0[2];
  if (fabs(s) >= 1.0) return 1;
  double c = sqrt(1.0 - s * s);
  double s1 = s * ca - c * sa;          /* sin(phi - d) */
  double c1 = c * ca + s * sa;          /* cos(phi - d) */
  if (!(c1 > 0.0) || fabs(s1) >= s_max) return 1;
  *x1 = x0 * ca + p0[0] * sa;
  p1[0] = -x0 * sa + p0[0] * ca;
  p1[1] = p0[1];
  p1[2] = s1;
  p1[3] = p0[3];
  p1[4] = p0[4];
  if (F) {
    double rho = -KB_PER_TESLA * bz * p0[4];
    for (int i = 0; i < 25; ++i) F[i] = 0.0;
    for (int i = 0; i < 5; ++i) F[i * 5 + i] = 1.0;
    F[0 * 5 + 0] = c / c1;
    F[1 * 5 + 0] = -p0[3] * sa / c1;
    F[2 * 5 + 0] = -rho * sa;
    F[2 * 5 + 2] = c1 / c;
  }
  return 0;
}

/* C <- F C F^T */
static void transport_cov(const double F[25], double C[25]) {
  double T[25], R[25];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += F[i * 5 + k] * C[k * 5 + j];
      T[i * 5 + j] = s;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += T[i * 5 + k] * F[j * 5 + k];
      R[i * 5 + j] = s;
    }
  memcpy(C, R, sizeof(R));
}

/* Predict p, C from x0 to x1. */
static int predict(double bz, double s_max, double x0, double x1, double p[5], double C[25],
                   double* margin) {
  double F[25];
  if (propagate_m(bz, s_max, x0, x1, p, F, margin)) return 1;
  transport_cov(F, C);
  return 0;
}

/* ------------------------------------------------------------ Kalman filter */
/* H = [I2 0], V = diag(vy, vz), S = H C H^T + V */
static double kf_chi2(const double p[5], const double C[25], double my, double mz, double vy, double vz) {
  double S00 = C[0] + vy, S01 = C[1], S11 = C[6] + vz;
  double det = S00 * S11 - S01 * S01;
  double r0 = my - p[0], r1 = mz - p[1];
  return (r0 * (S11 * r0 - S01 * r1) + r1 * (S00 * r1 - S01 * r0)) / det;
}

double orc_kf_update(double p[5], double C[25], double my, double mz, double vy, double vz) {
  double S00 = C[0] + vy, S01 = C[1], S11 = C[6] + vz;
  double det = S00 * S11 - S01 * S01;
  double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  double r0 = my - p[0], r1 = mz - p[1];
  double chi2 = r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
  double K[5][2], HC[2][5];
  for (int i = 0; i < 5; ++i) {
    K[i][0] = C[i * 5 + 0] * I00 + C[i * 5 + 1] * I01;
    K[i][1] = C[i * 5 + 0] * I01 + C[i * 5 + 1] * I11;
  }
  for (int j = 0; j < 5; ++j) { HC[0][j] = C[0 * 5 + j]; HC[1][j] = C[1 * 5 + j]; }
  for (int i = 0; i < 5; ++i) p[i] += K[i][0] * r0 + K[i][1] * r1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C[i * 5 + j] -= K[i][0] * HC[0][j] + K[i][1] * HC[1][j];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < i; ++j) {
      double s = 0.5 * (C[i * 5 + j] + C[j * 5 + i]);
      C[i * 5 + j] = s;
      C[j * 5 + i] = s;
    }
  return chi2;
}

/* ------------------------------------------------------------ S1: row lists */
typedef struct {
  const orc_geometry* g;
  const orc_cuts* c;
  const double *y, *z;
  const int32_t* row;      /* per cluster */
  int64_t base, n;         /* instance cluster range */
  int64_t* ids;            /* instance ids grouped by row, sorted by (y, id) within row */
  int64_t roff[ORC_MAX_ROWS + 1];
  int brute;
} inst_ctx;

static const double* g_sort_y;
static int cmp_y_id(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  double yi = g_sort_y[i], yj = g_sort_y[j];
  if (yi < yj) return -1;
  if (yi > yj) return 1;
  return (i > j) - (i < j);
}

static int build_rows(inst_ctx* t) {
  int R = t->g->n_rows;
  int64_t cnt[ORC_MAX_ROWS];
  memset(cnt, 0, sizeof(cnt));
  for (int64_t i = t->base; i < t->base + t->n; ++i) cnt[t->row[i]]++;
  t->roff[0] = 0;
  for (int r = 0; r < R; ++r) t->roff[r + 1] = t->roff[r] + cnt[r];
  t->ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(t->n > 0 ? t->n : 1));
  if (!t->ids) return 1;
  int64_t fill[ORC_MAX_ROWS];
  for (int r = 0; r < R; ++r) fill[r] = t->roff[r];
  for (int64_t i = t->base; i < t->base + t->n; ++i) t->ids[fill[t->row[i]]++] = i;
  g_sort_y = t->y;
  for (int r = 0; r < R; ++r)
    qsort(t->ids + t->roff[r], (size_t)cnt[r], sizeof(int64_t), cmp_y_id);
  return 0;
}

/* first position in row r with y >= ylo (or the row start for brute force) */
static int64_t row_lower(const inst_ctx* t, int r, double ylo) {
  int64_t lo = t->roff[r], hi = t->roff[r + 1];
  if (t->brute) return lo;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (t->y[t->ids[mid]] < ylo) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* ------------------------------------------------------------ S2: neighbours */
/* Candidates of hit h in row rn: |y - yh| <= wy dxn and |z - zh| <= wz dxn.
 * Collects them (ids) and logs the edge margins of everything in the widened window. */
static int64_t nf_candidates(const inst_ctx* t, int64_t h, int rn, double dxn, int64_t* out,
                             int64_t cap, double* margin) {
  double wy = t->c->nf_wy * dxn, wz = t->c->nf_wz * dxn;
  double yh = t->y[h], zh = t->z[h];
  int64_t k = row_lower(t, rn, yh - wy * EXT), n = 0;
  for (; k < t->roff[rn + 1]; ++k) {
    int64_t i = t->ids[k];
    double ady = fabs(t->y[i] - yh), adz = fabs(t->z[i] - zh);
    if (!t->brute && t->y[i] > yh + wy * EXT) break;
    if (ady <= wy * EXT && adz <= wz * EXT) {
      *margin = dmin(*margin, dmin(rel_margin(ady, wy), rel_margin(adz, wz)));
    }
    if (ady <= wy && adz <= wz) {
      if (n < cap) out[n] = i;
      n++;
    }
  }
  return n;
}

static int neighbours(inst_ctx* t, orc_result* res) {
  const double* X = t->g->row_x;
  int R = t->g->n_rows;
  int64_t cap = 4096;
  int64_t* cu = (int64_t*)malloc(sizeof(int64_t) * cap);
  int64_t* cd = (int64_t*)malloc(sizeof(int64_t) * cap);
  if (!cu || !cd) { free(cu); free(cd); return 1; }
  for (int64_t h = t->base; h < t->base + t->n; ++h) {
    res->up[h] = res->down[h] = -1;
    res->nf_margin[h] = INFINITY;
  }
  for (int r = 1; r + 1 < R; ++r) {
    double dxu = X[r + 1] - X[r], dxd = X[r] - X[r - 1];
    double f = (X[r] - X[r - 1]) / (X[r + 1] - X[r - 1]);
    for (int64_t k = t->roff[r]; k < t->roff[r + 1]; ++k) {
      int64_t h = t->ids[k];
      double margin = INFINITY;
      int64_t nu = nf_candidates(t, h, r + 1, dxu, cu, cap, &margin);
      int64_t nd = nf_candidates(t, h, r - 1, dxd, cd, cap, &margin);
      if (nu > cap || nd > cap) { free(cu); free(cd); return 1; }
      double D1 = INFINITY, D2 = INFINITY;
      int64_t bu = -1, bd = -1;
      for (int64_t a = 0; a < nu; ++a)
        for (int64_t b = 0; b < nd; ++b) {
          int64_t u = cu[a], d = cd[b];
          double yhat = t->y[d] + f * (t->y[u] - t->y[d]);
          double zhat = t->z[d] + f * (t->z[u] - t->z[d]);
          double D = (yhat - t->y[h]) * (yhat - t->y[h]) + (zhat - t->z[h]) * (zhat - t->z[h]);
          int better = bu < 0 || D < D1 || (D == D1 && (u < bu || (u == bu && d < bd)));
          if (better) {
            if (bu >= 0) D2 = D1;
            D1 = D; bu = u; bd = d;
          } else if (D < D2) {
            D2 = D;
          }
        }
      if (bu >= 0) {
        margin = dmin(margin, rel_margin(D1, t->c->nf_dmax));
        if (D2 < INFINITY) margin = dmin(margin, D2 > 0.0 ? (D2 - D1) / D2 : 0.0);
        if (D1 <= t->c->nf_dmax) { res->up[h] = (int32_t)bu; res->down[h] = (int32_t)bd; }
      }
      res->nf_margin[h] = margin;
    }
  }
  free(cu); free(cd);
  return 0;
}

/* ------------------------------------------------------------ S3: clean */
static void clean_links(const inst_ctx* t, orc_result* res) {
  for (int64_t h = t->base; h < t->base + t->n; ++h) {
    int32_t u = res->up[h], d = res->down[h];
    res->upc[h] = (u >= 0 && res->down[u] == h) ? u : -1;
    res->downc[h] = (d >= 0 && res->up[d] == h) ? d : -1;
  }
}

/* ------------------------------------------------------------ S5: tracklets */
enum { STOP_END = 0, STOP_PROP = 1, STOP_EDGE = 2, STOP_MISS = 3, STOP_SINPHI = 4 };

/* Search row r around the prediction: candidate c is inside iff
 * |dy| <= k sqrt(Cyy + s_c^2) and |dz| <= k sqrt(Czz + s_c^2), s_c = sigma(z_c);
 * the best minimises dy^2/(Cyy+s_c^2) + dz^2/(Czz+s_c^2), ties to the smaller id. */
static int64_t search_row(const inst_ctx* t, int r, const double p[5], const double C[25], double* margin) {
  const orc_cuts* c = t->c;
  double smax = c->sig_readout > c->sig_cathode ? c->sig_readout : c->sig_cathode;
  double ybound = c->search_k * sqrt(C[0] + smax * smax) * EXT;
  int64_t k = row_lower(t, r, p[0] - ybound);
  int64_t best = -1;
  double d1 = INFINITY, d2 = INFINITY;
  for (; k < t->roff[r + 1]; ++k) {
    int64_t i = t->ids[k];
    if (!t->brute && t->y[i] > p[0] + ybound) break;
    double s = sigma_at(t->g, c, t->z[i]);
    double vy = C[0] + s * s, vz = C[6] + s * s;
    double wy = c->search_k * sqrt(vy), wz = c->search_k * sqrt(vz);
    double ady = fabs(t->y[i] - p[0]), adz = fabs(t->z[i] - p[1]);
    if (ady <= wy * EXT && adz <= wz * EXT)
      *margin = dmin(*margin, dmin(rel_margin(ady, wy), rel_margin(adz, wz)));
    if (ady > wy || adz > wz) continue;
    double d = ady * ady / vy + adz * adz / vz;
    if (best < 0 || d < d1 || (d == d1 && i < best)) {
      if (best >= 0) d2 = d1;
      d1 = d; best = i;
    } else if (d < d2) {
      d2 = d;
    }
  }
  if (best >= 0 && d2 < INFINITY) *margin = dmin(*margin, d2 > 0.0 ? (d2 - d1) / d2 : 0.0);
  return best;
}

static void init_cov(const inst_ctx* t, double C[25], double zc) {
  double s = sigma_at(t->g, t->c, zc);
  for (int i = 0; i < 25; ++i) C[i] = 0.0;
  C[0] = s * s;
  C[6] = s * s;
  C[12] = t->c->c_s;
  C[18] = t->c->c_t;
  C[24] = t->c->c_qpt;
}

/* Refit prior: diffuse in every parameter, centred on the previous estimate. */
static void init_cov_refit_c(const orc_cuts* c, double C[25]) {
  for (int i = 0; i < 25; ++i) C[i] = 0.0;
  C[0] = c->c_yz_refit;
  C[6] = c->c_yz_refit;
  C[12] = c->c_s;
  C[18] = c->c_t;
  C[24] = c->c_qpt_refit;
}

static void init_cov_refit(const inst_ctx* t, double C[25]) {
  for (int i = 0; i < 25; ++i) C[i] = 0.0;
  C[0] = t->c->c_yz_refit;
  C[6] = t->c->c_yz_refit;
  C[12] = t->c->c_s;
  C[18] = t->c->c_t;
  C[24] = t->c->c_qpt_refit;
}

/* Try cluster i at the current prediction: chi2 cut, then update. */
static int try_hit(const inst_ctx* t, int64_t i, double p[5], double C[25], double* margin) {
  double s = sigma_at(t->g, t->c, t->z[i]);
  double chi2 = kf_chi2(p, C, t->y[i], t->z[i], s * s, s * s);
  *margin = dmin(*margin, rel_margin(chi2, t->c->chi2_max));
  if (!(chi2 <= t->c->chi2_max)) return 0;
  orc_kf_update(p, C, t->y[i], t->z[i], s * s, s * s);
  return 1;
}

typedef struct {
  int64_t hits[ORC_MAX_ROWS];
  int nhits, stop_up, stop_down, row_ref;
  double x_ref, param[5], margin;
} tracklet;

static void grow(const inst_ctx* t, const orc_result* res, int64_t h0, tracklet* tl) {
  const orc_cuts* c = t->c;
  const double* X = t->g->row_x;
  int R = t->g->n_rows;
  double tanh_ = t->g->tan_half_sector;
  double margin = INFINITY;
  int64_t up_hit[ORC_MAX_ROWS];
  for (int r = 0; r < R; ++r) { up_hit[r] = -1; tl->hits[r] = -1; }

  /* init from the first link of the chain */
  int r0 = t->row[h0];
  int64_t h1 = res->upc[h0];
  int r1 = t->row[h1];
  double dx = X[r1] - X[r0], dy = t->y[h1] - t->y[h0], dz = t->z[h1] - t->z[h0];
  double L = sqrt(dx * dx + dy * dy);
  double p[5] = {t->y[h0], t->z[h0], dy / L, dz / L, 0.0};
  double C[25];
  init_cov(t, C, t->z[h0]);
  up_hit[r0] = h0;

  /* upward */
  int prev_row = r0;
  int64_t prev = h0;
  int miss = 0;
  int stop = STOP_END;
  int top_row = r0;
  double top_p[5];
  memcpy(top_p, p, sizeof(top_p));
  for (int r = r0 + 1; r < R; ++r) {
    if (predict(c->bz, c->s_max, X[r - 1], X[r], p, C, &margin)) { stop = STOP_PROP; break; }
    double edge = X[r] * tanh_ + c->edge_margin;
    margin = dmin(margin, rel_margin(fabs(p[0]), edge));
    if (fabs(p[0]) > edge) { stop = STOP_EDGE; break; }
    int64_t cand;
    if (prev_row == r - 1 && res->upc[prev] >= 0) cand = res->upc[prev];
    else cand = search_row(t, r, p, C, &margin);
    if (cand >= 0 && try_hit(t, cand, p, C, &margin)) {
      up_hit[r] = cand; prev = cand; prev_row = r; miss = 0;
      top_row = r; memcpy(top_p, p, sizeof(top_p));
      margin = dmin(margin, rel_margin(fabs(p[2]), c->s_max));
      if (fabs(p[2]) >= c->s_max) { stop = STOP_SINPHI; break; }
    } else {
      if (++miss > c->max_miss) { stop = STOP_MISS; break; }
    }
  }
  tl->stop_up = stop;

  /* downward from the outermost accepted hit, covariance reset */
  memcpy(p, top_p, sizeof(top_p));
  init_cov(t, C, t->z[up_hit[top_row]]);
  tl->hits[top_row] = up_hit[top_row];
  int in_row = top_row;
  double in_p[5];
  memcpy(in_p, p, sizeof(in_p));
  miss = 0;
  stop = STOP_END;
  for (int r = top_row - 1; r >= 0; --r) {
    if (predict(c->bz, c->s_max, X[r + 1], X[r], p, C, &margin)) { stop = STOP_PROP; break; }
    double edge = X[r] * tanh_ + c->edge_margin;
    margin = dmin(margin, rel_margin(fabs(p[0]), edge));
    if (fabs(p[0]) > edge) { stop = STOP_EDGE; break; }
    int64_t cand = up_hit[r] >= 0 ? up_hit[r] : search_row(t, r, p, C, &margin);
    if (cand >= 0 && try_hit(t, cand, p, C, &margin)) {
      tl->hits[r] = cand; miss = 0;
      in_row = r; memcpy(in_p, p, sizeof(in_p));
      margin = dmin(margin, rel_margin(fabs(p[2]), c->s_max));
      if (fabs(p[2]) >= c->s_max) { stop = STOP_SINPHI; break; }
    } else {
      if (++miss > c->max_miss) { stop = STOP_MISS; break; }
    }
  }
  tl->stop_down = stop;
  tl->nhits = 0;
  for (int r = 0; r < R; ++r) tl->nhits += tl->hits[r] >= 0;
  tl->row_ref = in_row;
  tl->x_ref = X[in_row];
  memcpy(tl->param, in_p, sizeof(in_p));
  tl->margin = margin;
}

/* ------------------------------------------------------------ S7: refit */
/* Each pass linearises around a reference trajectory: the previous estimate
 * transported exactly to every owned cluster.  A Kalman filter of the
 * deviation d from that trajectory (d transported by the Jacobian at the
 * reference, diffuse prior centred on d = 0) runs from the outermost cluster
 * inward; reference + d at the innermost cluster is the next estimate.  One
 * pass is one Gauss-Newton step of the least-squares fit, so the exact helix is
 * the fixed point for noiseless clusters. */
static int refit(const inst_ctx* t, const int64_t* ids, int n, const double p_in[5], double x_in,
                 double p_out[5], double cov_out[15], double* chi2_out, double* x_out, double* margin) {
  const orc_cuts* c = t->c;
  const double* X = t->g->row_x;
  double est[5], ref[5], d[5], C[25], F[25], chi2 = 0.0, x_cur = x_in;
  memcpy(est, p_in, sizeof(est));
  for (int pass = 0; pass < c->n_refit; ++pass) {
    int64_t last = ids[n - 1];
    memcpy(ref, est, sizeof(ref));
    if (propagate_m(c->bz, c->s_max, x_cur, X[t->row[last]], ref, NULL, margin)) return 1;
    for (int q = 0; q < 5; ++q) d[q] = 0.0;
    init_cov_refit(t, C);
    chi2 = 0.0;
    for (int k = n - 1; k >= 0; --k) {
      int64_t i = ids[k];
      if (k < n - 1) {
        if (propagate_m(c->bz, c->s_max, X[t->row[ids[k + 1]]], X[t->row[i]], ref, F, margin)) return 1;
        double dn[5];
        for (int a = 0; a < 5; ++a) {
          dn[a] = 0.0;
          for (int b = 0; b < 5; ++b) dn[a] += F[a * 5 + b] * d[b];
        }
        memcpy(d, dn, sizeof(d));
        transport_cov(F, C);
      }
      double s = sigma_at(t->g, c, t->z[i]);
      chi2 += orc_kf_update(d, C, t->y[i] - ref[0], t->z[i] - ref[1], s * s, s * s);
    }
    for (int q = 0; q < 5; ++q) est[q] = ref[q] + d[q];
    x_cur = X[t->row[ids[0]]];
  }
  memcpy(p_out, est, sizeof(est));
  int m = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) cov_out[m++] = C[i * 5 + j];
  *chi2_out = chi2;
  *x_out = x_cur;
  return 0;
}

/* ------------------------------------------------------------ S4, S5, S6, S7 per instance */
static const inst_ctx* g_sort_ctx;
static int cmp_row_id(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  int ri = g_sort_ctx->row[i], rj = g_sort_ctx->row[j];
  if (ri != rj) return ri < rj ? -1 : 1;
  return (i > j) - (i < j);
}

#define PUSH(res, w, val) do { __typeof__(val) v_ = (val); if (vec_push(&(res)->a[w], &v_)) goto oom; } while (0)

static int track_instance(inst_ctx* t, int64_t inst, orc_result* res) {
  int R = t->g->n_rows;
  int64_t* starts = NULL;
  tracklet* tls = NULL;
  int64_t ns = 0;
  if (neighbours(t, res)) return 1;
  clean_links(t, res);

  /* S4: start hits, ordered by (row, id) */
  starts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(t->n > 0 ? t->n : 1));
  if (!starts) return 1;
  for (int64_t h = t->base; h < t->base + t->n; ++h) {
    int32_t u = res->upc[h];
    if (res->downc[h] < 0 && u >= 0 && res->upc[u] >= 0) starts[ns++] = h;
  }
  g_sort_ctx = t;
  qsort(starts, (size_t)ns, sizeof(int64_t), cmp_row_id);
  if (ns >= (1 << 20)) { free(starts); return 1; }

  /* S5 */
  tls = (tracklet*)malloc(sizeof(tracklet) * (size_t)(ns > 0 ? ns : 1));
  if (!tls) { free(starts); return 1; }
  for (int64_t k = 0; k < ns; ++k) grow(t, res, starts[k], &tls[k]);

  /* S6: weights, owned clusters, cuts */
  for (int64_t h = t->base; h < t->base + t->n; ++h) res->weight[h] = 0;
  for (int64_t k = 0; k < ns; ++k) {
    uint32_t w = ((uint32_t)tls[k].nhits << 20) | (uint32_t)((1 << 20) - 1 - k);
    for (int r = 0; r < R; ++r) {
      int64_t i = tls[k].hits[r];
      if (i >= 0 && res->weight[i] < w) res->weight[i] = w;
    }
  }
  int64_t own_ids[ORC_MAX_ROWS];
  for (int64_t k = 0; k < ns; ++k) {
    tracklet* tl = &tls[k];
    int32_t tl_index = (int32_t)(res->a[ORC_TL_INST].n);
    /* record the tracklet */
    PUSH(res, ORC_TL_INST, (int32_t)inst);
    PUSH(res, ORC_TL_START, (int32_t)starts[k]);
    PUSH(res, ORC_TL_NHITS, (int32_t)tl->nhits);
    PUSH(res, ORC_TL_STOP_UP, (int32_t)tl->stop_up);
    PUSH(res, ORC_TL_STOP_DOWN, (int32_t)tl->stop_down);
    PUSH(res, ORC_TL_ROWREF, (int32_t)tl->row_ref);
    PUSH(res, ORC_TL_XREF, tl->x_ref);
    PUSH(res, ORC_TL_MARGIN, tl->margin);
    for (int i = 0; i < 5; ++i) PUSH(res, ORC_TL_PARAM, tl->param[i]);
    for (int r = 0; r < R; ++r) PUSH(res, ORC_TL_HITS, (int32_t)tl->hits[r]);

    uint32_t w = ((uint32_t)tl->nhits << 20) | (uint32_t)((1 << 20) - 1 - k);
    int own = 0;
    for (int r = 0; r < R; ++r) {
      int64_t i = tl->hits[r];
      if (i >= 0 && res->weight[i] == w) own_ids[own++] = i;
    }
    int shared = tl->nhits - own;
    if (!(own >= t->c->n_min && (double)shared <= t->c->f_shared * (double)tl->nhits)) continue;

    /* S7 */
    double pout[5], cov[15], chi2 = 0.0, xout = 0.0, margin = INFINITY;
    int status = refit(t, own_ids, own, tl->param, tl->x_ref, pout, cov, &chi2, &xout, &margin);
    if (status) {
      memcpy(pout, tl->param, sizeof(pout));
      for (int i = 0; i < 15; ++i) cov[i] = 0.0;
      xout = tl->x_ref;
    }
    PUSH(res, ORC_TR_INST, (int32_t)inst);
    PUSH(res, ORC_TR_TRACKLET, tl_index);
    PUSH(res, ORC_TR_NCL, (int32_t)own);
    PUSH(res, ORC_TR_OFFSET, (int32_t)res->a[ORC_TR_IDS].n);
    PUSH(res, ORC_TR_NDF, (int32_t)(2 * own - 5));
    PUSH(res, ORC_TR_STATUS, (int32_t)status);
    PUSH(res, ORC_TR_XREF, xout);
    PUSH(res, ORC_TR_CHI2, chi2);
    PUSH(res, ORC_TR_MARGIN, margin);
    for (int i = 0; i < 5; ++i) PUSH(res, ORC_TR_PARAM, pout[i]);
    for (int i = 0; i < 15; ++i) PUSH(res, ORC_TR_COV, cov[i]);
    for (int i = 0; i < own; ++i) PUSH(res, ORC_TR_IDS, (int32_t)own_ids[i]);
  }
  free(starts);
  free(tls);
  return 0;
oom:
  free(starts);
  free(tls);
  return 1;
}

/* ------------------------------------------------------------ entry */
static const size_t elem_size[ORC_N_ARRAYS] = {
  [ORC_TL_INST] = 4, [ORC_TL_START] = 4, [ORC_TL_NHITS] = 4, [ORC_TL_STOP_UP] = 4,
  [ORC_TL_STOP_DOWN] = 4, [ORC_TL_ROWREF] = 4, [ORC_TL_XREF] = 8, [ORC_TL_MARGIN] = 8,
  [ORC_TL_PARAM] = 8, [ORC_TL_HITS] = 4,
  [ORC_TR_INST] = 4, [ORC_TR_TRACKLET] = 4, [ORC_TR_NCL] = 4, [ORC_TR_OFFSET] = 4,
  [ORC_TR_NDF] = 4, [ORC_TR_STATUS] = 4, [ORC_TR_XREF] = 8, [ORC_TR_CHI2] = 8,
  [ORC_TR_MARGIN] = 8, [ORC_TR_PARAM] = 8, [ORC_TR_COV] = 8, [ORC_TR_IDS] = 4,
};

orc_result* orc_track(const orc_geometry* g, const orc_cuts* c, int64_t n_inst,
                      const int64_t* inst_offsets, const double* x, const double* y,
                      const double* z, const int32_t* row, int brute_force_nf) {
  if (!g || !c || !inst_offsets || !y || !z || g->n_rows < 3 || g->n_rows > ORC_MAX_ROWS || n_inst < 0)
    return NULL;
  if (!row && !x) return NULL;
  int64_t n = inst_offsets[n_inst];
  for (int64_t i = 0; i < n_inst; ++i)
    if (inst_offsets[i + 1] < inst_offsets[i]) return NULL;
  orc_result* res = (orc_result*)calloc(1, sizeof(orc_result));
  if (!res) return NULL;
  res->n = n;
  res->n_rows = g->n_rows;
  for (int i = 0; i < ORC_N_ARRAYS; ++i) vec_init(&res->a[i], elem_size[i] ? elem_size[i] : 4);
  size_t nn = (size_t)(n > 0 ? n : 1);
  res->up = (int32_t*)malloc(4 * nn);
  res->down = (int32_t*)malloc(4 * nn);
  res->upc = (int32_t*)malloc(4 * nn);
  res->downc = (int32_t*)malloc(4 * nn);
  res->nf_margin = (double*)malloc(8 * nn);
  res->weight = (uint32_t*)malloc(4 * nn);
  int32_t* rows = (int32_t*)malloc(4 * nn);
  if (!res->up || !res->down || !res->upc || !res->downc || !res->nf_margin || !res->weight || !rows) {
    free(rows); orc_free(res); return NULL;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (row) {
      rows[i] = row[i];
    } else {
      int best = 0;
      for (int r = 1; r < g->n_rows; ++r)
        if (fabs(x[i] - g->row_x[r]) < fabs(x[i] - g->row_x[best])) best = r;
      rows[i] = best;
    }
    if (rows[i] < 0 || rows[i] >= g->n_rows) { free(rows); orc_free(res); return NULL; }
  }
  for (int64_t k = 0; k < n_inst; ++k) {
    inst_ctx t;
    memset(&t, 0, sizeof(t));
    t.g = g; t.c = c; t.y = y; t.z = z; t.row = rows;
    t.base = inst_offsets[k]; t.n = inst_offsets[k + 1] - inst_offsets[k];
    t.brute = brute_force_nf;
    if (build_rows(&t) || track_instance(&t, k, res)) {
      free(t.ids); free(rows); orc_free(res); return NULL;
    }
    free(t.ids);
  }
  free(rows);
  return res;
}


/* ============================================================ cross-sector merging
 * Reading: a particle that crosses a sector boundary leaves one track in each
 * sector.  For tracks a, b in adjacent sectors (same side, same collision) the
 * inner one I has the smaller radius of its reference point (ties: smaller
 * track index).  The pair is tested if |tanl_I - tanl_O| <= max_dtanl and I's
 * outermost and O's innermost owned clusters are within max_gap in the
 * transverse plane.  I's refit state is transported to its outermost
 * cluster, rotated into O's frame and transported to O's reference x; chi2 =
 * dp^T (C_I + C_O)^-1 dp with dp the parameter difference; accepted iff chi2
 * <= chi2_max.  Each track keeps its best outer and its best inner partner
 * (smallest chi2, ties to the smaller track index); mutual best pairs are
 * linked.  Linked tracks form chains, inner to outer, refitted together:
 * the sector refit (reference trajectory, diffuse prior, 3 passes) with the
 * reference rotated exactly and deviation and covariance rotated by the
 * Jacobian wherever consecutive clusters lie in different sectors. */

struct orc_merge_result {
  int64_t k;
  vec a[ORM_N_ARRAYS];
};

static const size_t orm_elem[ORM_N_ARRAYS] = {
  [ORM_LINK_OUT] = 4, [ORM_LINK_IN] = 4, [ORM_MARGIN] = 8, [ORM_CH_HEAD] = 4, [ORM_CH_NSEG] = 4,
  [ORM_CH_NCL] = 4, [ORM_CH_OFFSET] = 4, [ORM_CH_NDF] = 4, [ORM_CH_STATUS] = 4, [ORM_CH_INST] = 4,
  [ORM_CH_XREF] = 8, [ORM_CH_CHI2] = 8, [ORM_CH_MARGIN] = 8, [ORM_CH_PARAM] = 8, [ORM_CH_COV] = 8,
  [ORM_CH_SEGS] = 4, [ORM_CH_IDS] = 4, [ORM_PAIRS] = 8,
};

int64_t orm_count(const orc_merge_result* r, int w) {
  if (!r || w < 0 || w >= ORM_N_ARRAYS) return -1;
  return r->a[w].n;
}
const void* orm_array(const orc_merge_result* r, int w) {
  if (!r || w < 0 || w >= ORM_N_ARRAYS) return NULL;
  return r->a[w].p;
}
void orm_free(orc_merge_result* r) {
  if (!r) return;
  for (int i = 0; i < ORM_N_ARRAYS; ++i) vec_free(&r->a[i]);
  free(r);
}

typedef struct {
  int32_t inst, sector, n, status;
  const int32_t* ids;
  double alpha, x_ref, r_ref, x_out;
  double p[5], C[25];
  double in_x, in_y, out_x, out_y;   /* transverse positions of the innermost / outermost clusters */
} mtrack;

static double wrap_angle(double a) {
  while (a > M_PI) a -= 2.0 * M_PI;
  while (a <= -M_PI) a += 2.0 * M_PI;
  return a;
}

/* Solve S x = b (5x5, plain Gaussian elimination with partial pivoting); 1 if singular */
static int solve5(const double S_in[25], const double b_in[5], double x[5]) {
  double A[5][6];
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j < 5; ++j) A[i][j] = S_in[i * 5 + j];
    A[i][5] = b_in[i];
  }
  for (int col = 0; col < 5; ++col) {
    int piv = col;
    for (int i = col + 1; i < 5; ++i)
      if (fabs(A[i][col]) > fabs(A[piv][col])) piv = i;
    if (A[piv][col] == 0.0) return 1;
    if (piv != col)
      for (int j = 0; j < 6; ++j) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
    for (int i = col + 1; i < 5; ++i) {
      double f = A[i][col] / A[col][col];
      for (int j = col; j < 6; ++j) A[i][j] -= f * A[col][j];
    }
  }
  for (int i = 4; i >= 0; --i) {
    double sum = A[i][5];
    for (int j = i + 1; j < 5; ++j) sum -= A[i][j] * x[j];
    x[i] = sum / A[i][i];
  }
  return 0;
}

/* chi2 of the pair (I inner, O outer); 1 if a transport or rotation fails */
static int pair_chi2(const orc_cuts* c, const mtrack* I, const mtrack* O, double* chi2) {
  double p[5], C[25], F[25], x1;
  memcpy(p, I->p, sizeof(p));
  memcpy(C, I->C, sizeof(C));
  if (propagate_m(c->bz, c->s_max, I->x_ref, I->x_out, p, F, NULL)) return 1;
  transport_cov(F, C);
  double pr[5];
  if (orc_rotate(c->bz, c->s_max, wrap_angle(O->alpha - I->alpha), I->x_out, p, &x1, pr, F)) return 1;
  transport_cov(F, C);
  if (propagate_m(c->bz, c->s_max, x1, O->x_ref, pr, F, NULL)) return 1;
  transport_cov(F, C);
  double S[25], dp[5], sol[5];
  for (int i = 0; i < 25; ++i) S[i] = C[i] + O->C[i];
  for (int i = 0; i < 5; ++i) dp[i] = pr[i] - O->p[i];
  if (solve5(S, dp, sol)) return 1;
  double q = 0.0;
  for (int i = 0; i < 5; ++i) q += dp[i] * sol[i];
  *chi2 = q;
  return 0;
}

typedef struct { int32_t id; int seg; } mcl;

/* Global refit of one chain (segments inner to outer). */
static int chain_refit(const orc_geometry* g, const orc_cuts* c, const mtrack* T, const int32_t* segs, int m,
                       const double* y, const double* z, const int32_t* row, const mcl* L, int n,
                       double p_out[5], double cov_out[15], double* chi2_out, double* x_out, double* margin) {
  const double* X = g->row_x;
  double est[5], ref[5], d[5], C[25], F[25], chi2 = 0.0, x_cur, x1;
  /* pass 0: reference from the outermost segment's own fit, carried within
   * its frame to its outermost cluster */
  const mtrack* So = &T[segs[m - 1]];
  double ref_out[5];
  memcpy(ref_out, So->p, sizeof(ref_out));
  if (propagate_m(c->bz, c->s_max, So->x_ref, So->x_out, ref_out, NULL, margin)) return 1;
  const double x_outer = So->x_out;
  memcpy(est, T[segs[0]].p, sizeof(est));
  x_cur = T[segs[0]].x_ref;
  for (int pass = 0; pass < c->n_refit; ++pass) {
    /* later passes: the estimate carried outward through the chain; if that
     * carry fails, the previous pass's outer reference is kept */
    if (pass > 0) {
      double carry[5];
      memcpy(carry, est, sizeof(carry));
      double xf = x_cur;
      int ok = 1;
      for (int j = 0; j < m && ok; ++j) {
        const mtrack* S = &T[segs[j]];
        if (propagate_m(c->bz, c->s_max, xf, S->x_out, carry, NULL, margin)) { ok = 0; break; }
        xf = S->x_out;
        if (j < m - 1) {
          double pr[5];
          if (orc_rotate(c->bz, c->s_max, wrap_angle(T[segs[j + 1]].alpha - S->alpha), xf, carry, &x1, pr,
                         NULL)) { ok = 0; break; }
          memcpy(carry, pr, sizeof(carry));
          xf = x1;
        }
      }
      if (ok) memcpy(ref_out, carry, sizeof(ref_out));
    }
    memcpy(ref, ref_out, sizeof(ref));
    double xf = x_outer;
    for (int q = 0; q < 5; ++q) d[q] = 0.0;
    init_cov_refit_c(c, C);
    chi2 = 0.0;
    double x_prev = xf;
    for (int k = n - 1; k >= 0; --k) {
      int32_t i = L[k].id;
      double xk = X[row[i]];
      if (k < n - 1) {
        if (L[k].seg != L[k + 1].seg) {
          double pr[5], R[25];
          if (orc_rotate(c->bz, c->s_max, wrap_angle(T[segs[L[k].seg]].alpha - T[segs[L[k + 1].seg]].alpha),
                         x_prev, ref, &x1, pr, R))
            return 1;
          memcpy(ref, pr, sizeof(ref));
          double dn[5];
          for (int a = 0; a < 5; ++a) {
            dn[a] = 0.0;
            for (int b = 0; b < 5; ++b) dn[a] += R[a * 5 + b] * d[b];
          }
          memcpy(d, dn, sizeof(d));
          transport_cov(R, C);
          x_prev = x1;
        }
        if (propagate_m(c->bz, c->s_max, x_prev, xk, ref, F, margin)) return 1;
        double dn[5];
        for (int a = 0; a < 5; ++a) {
          dn[a] = 0.0;
          for (int b = 0; b < 5; ++b) dn[a] += F[a * 5 + b] * d[b];
        }
        memcpy(d, dn, sizeof(d));
        transport_cov(F, C);
      }
      double s = sigma_at(g, c, z[i]);
      chi2 += orc_kf_update(d, C, y[i] - ref[0], z[i] - ref[1], s * s, s * s);
      x_prev = xk;
    }
    for (int q = 0; q < 5; ++q) est[q] = ref[q] + d[q];
    x_cur = X[row[L[0].id]];
  }
  memcpy(p_out, est, sizeof(est));
  int mm = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) cov_out[mm++] = C[i * 5 + j];
  *chi2_out = chi2;
  *x_out = x_cur;
  return 0;
}

#define MPUSH(res, w, val) do { __typeof__(val) v_ = (val); if (vec_push(&(res)->a[w], &v_)) goto oom; } while (0)

orc_merge_result* orc_merge(const orc_geometry* g, const orc_cuts* c, const orc_merge_cuts* mc,
                            const orc_result* tr, int64_t n_inst, const int32_t* inst_sector,
                            const int32_t* inst_event, const double* y, const double* z, const int32_t* row) {
  if (!g || !c || !mc || !tr || !inst_sector || !inst_event || !y || !z || !row || n_inst < 0) return NULL;
  const int64_t K = tr->a[ORC_TR_INST].n;
  const int32_t* tinst = (const int32_t*)tr->a[ORC_TR_INST].p;
  const int32_t* tncl = (const int32_t*)tr->a[ORC_TR_NCL].p;
  const int32_t* toff = (const int32_t*)tr->a[ORC_TR_OFFSET].p;
  const int32_t* tst = (const int32_t*)tr->a[ORC_TR_STATUS].p;
  const int32_t* tids = (const int32_t*)tr->a[ORC_TR_IDS].p;
  const double* txr = (const double*)tr->a[ORC_TR_XREF].p;
  const double* tpar = (const double*)tr->a[ORC_TR_PARAM].p;
  const double* tcov = (const double*)tr->a[ORC_TR_COV].p;
  orc_merge_result* res = (orc_merge_result*)calloc(1, sizeof(orc_merge_result));
  if (!res) return NULL;
  for (int i = 0; i < ORM_N_ARRAYS; ++i) vec_init(&res->a[i], orm_elem[i]);
  res->k = K;
  mtrack* T = (mtrack*)calloc((size_t)(K > 0 ? K : 1), sizeof(mtrack));
  int64_t* first = (int64_t*)calloc((size_t)(n_inst + 1), sizeof(int64_t));
  int32_t* best_out = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
  int32_t* best_in = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
  double* chi_out = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* chi_in = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* chi2_out2 = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* chi2_in2 = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* marg = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  int32_t* inst_of = NULL;
  mcl* L = NULL;
  if (!T || !first || !best_out || !best_in || !chi_out || !chi_in || !chi2_out2 || !chi2_in2 || !marg) goto oom;
  /* per track */
  for (int64_t k = 0; k < K; ++k) {
    mtrack* t = &T[k];
    t->inst = tinst[k];
    t->sector = inst_sector[t->inst];
    t->alpha = mc->alpha0 + (double)(t->sector % 18) * mc->dalpha;
    t->n = tncl[k];
    t->status = tst[k];
    t->ids = tids + toff[k];
    t->x_ref = txr[k];
    memcpy(t->p, tpar + 5 * k, sizeof(t->p));
    int mm = 0;
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j <= i; ++j) { t->C[i * 5 + j] = t->C[j * 5 + i] = tcov[15 * k + mm]; ++mm; }
    t->r_ref = sqrt(t->x_ref * t->x_ref + t->p[0] * t->p[0]);
    int32_t a = t->ids[0], b = t->ids[t->n - 1];
    double ca = cos(t->alpha), sa = sin(t->alpha);
    double xa = g->row_x[row[a]], xb = g->row_x[row[b]];
    t->in_x = xa * ca - y[a] * sa; t->in_y = xa * sa + y[a] * ca;
    t->out_x = xb * ca - y[b] * sa; t->out_y = xb * sa + y[b] * ca;
    t->x_out = xb;
    best_out[k] = best_in[k] = -1;
    chi_out[k] = chi_in[k] = chi2_out2[k] = chi2_in2[k] = INFINITY;
    marg[k] = INFINITY;
    first[t->inst + 1]++;
  }
  for (int64_t i = 0; i < n_inst; ++i) first[i + 1] += first[i];
  /* instance of (collision, sector) */
  int32_t n_ev = 0;
  for (int64_t i = 0; i < n_inst; ++i) if (inst_event[i] + 1 > n_ev) n_ev = inst_event[i] + 1;
  inst_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_ev > 0 ? n_ev : 1) * 36);
  if (!inst_of) goto oom;
  for (int64_t i = 0; i < (int64_t)n_ev * 36; ++i) inst_of[i] = -1;
  for (int64_t i = 0; i < n_inst; ++i)
    if (inst_sector[i] >= 0 && inst_sector[i] < 36) inst_of[(int64_t)inst_event[i] * 36 + inst_sector[i]] = (int32_t)i;
  /* pairs over every boundary k | k+1 of each side */
  for (int32_t e = 0; e < n_ev; ++e)
    for (int side = 0; side < 2; ++side)
      for (int kk = 0; kk < 18; ++kk) {
        int32_t ia = inst_of[(int64_t)e * 36 + side * 18 + kk];
        int32_t ib = inst_of[(int64_t)e * 36 + side * 18 + (kk + 1) % 18];
        if (ia < 0 || ib < 0) continue;
        for (int64_t a = first[ia]; a < first[ia + 1]; ++a)
          for (int64_t b = first[ib]; b < first[ib + 1]; ++b) {
            if (T[a].status || T[b].status) continue;
            int64_t I = a, O = b;
            if (T[b].r_ref < T[a].r_ref || (T[b].r_ref == T[a].r_ref && b < a)) { I = b; O = a; }
            double dt = fabs(T[I].p[3] - T[O].p[3]);
            double gx = T[I].out_x - T[O].in_x, gy = T[I].out_y - T[O].in_y;
            double gap = sqrt(gx * gx + gy * gy);
            double m = dmin(rel_margin(dt, mc->max_dtanl), rel_margin(gap, mc->max_gap));
            if (dt <= mc->max_dtanl * EXT && gap <= mc->max_gap * EXT) {
              marg[I] = dmin(marg[I], m);
              marg[O] = dmin(marg[O], m);
            }
            if (!(dt <= mc->max_dtanl && gap <= mc->max_gap)) continue;
            double chi2;
            if (pair_chi2(c, &T[I], &T[O], &chi2)) continue;
            double pr[3] = {(double)I, (double)O, chi2};
            for (int q = 0; q < 3; ++q) MPUSH(res, ORM_PAIRS, pr[q]);
            double mc2 = rel_margin(chi2, mc->chi2_max);
            marg[I] = dmin(marg[I], mc2);
            marg[O] = dmin(marg[O], mc2);
            if (!(chi2 <= mc->chi2_max)) continue;
            /* best outer partner of I, best inner partner of O (ties to the smaller index) */
            if (chi2 < chi_out[I] || (chi2 == chi_out[I] && O < best_out[I])) {
              chi2_out2[I] = chi_out[I]; chi_out[I] = chi2; best_out[I] = (int32_t)O;
            } else if (chi2 < chi2_out2[I]) {
              chi2_out2[I] = chi2;
            }
            if (chi2 < chi_in[O] || (chi2 == chi_in[O] && I < best_in[O])) {
              chi2_in2[O] = chi_in[O]; chi_in[O] = chi2; best_in[O] = (int32_t)I;
            } else if (chi2 < chi2_in2[O]) {
              chi2_in2[O] = chi2;
            }
          }
      }
  /* links: mutual best */
  for (int64_t k = 0; k < K; ++k) {
    if (chi2_out2[k] < INFINITY) marg[k] = dmin(marg[k], (chi2_out2[k] - chi_out[k]) / chi2_out2[k]);
    if (chi2_in2[k] < INFINITY) marg[k] = dmin(marg[k], (chi2_in2[k] - chi_in[k]) / chi2_in2[k]);
  }
  for (int64_t k = 0; k < K; ++k) {
    int32_t o = best_out[k];
    int32_t lo = (o >= 0 && best_in[o] == k) ? o : -1;
    MPUSH(res, ORM_LINK_OUT, lo);
  }
  for (int64_t k = 0; k < K; ++k) {
    int32_t i = best_in[k];
    int32_t li = (i >= 0 && best_out[i] == k) ? i : -1;
    MPUSH(res, ORM_LINK_IN, li);
    MPUSH(res, ORM_MARGIN, marg[k]);
  }
  /* chains and their global refit, in order of the head track */
  const int32_t* lout = (const int32_t*)res->a[ORM_LINK_OUT].p;
  const int32_t* lin = (const int32_t*)res->a[ORM_LINK_IN].p;
  int32_t segs[64];
  for (int64_t k = 0; k < K; ++k) {
    if (lin[k] >= 0 || lout[k] < 0) continue;
    int m = 0, n = 0;
    for (int64_t s2 = k; s2 >= 0 && m < 64; s2 = lout[s2]) { segs[m++] = (int32_t)s2; n += T[s2].n; }
    free(L);
    L = (mcl*)malloc(sizeof(mcl) * (size_t)n);
    if (!L) goto oom;
    int q = 0;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < T[segs[j]].n; ++i) { L[q].id = T[segs[j]].ids[i]; L[q].seg = j; ++q; }
    double pout[5], cov[15], chi2 = 0.0, xout = 0.0, margin = INFINITY;
    int status = chain_refit(g, c, T, segs, m, y, z, row, L, n, pout, cov, &chi2, &xout, &margin);
    if (status) {
      memcpy(pout, T[k].p, sizeof(pout));
      for (int i = 0; i < 15; ++i) cov[i] = 0.0;
      xout = T[k].x_ref;
      chi2 = 0.0;
    }
    MPUSH(res, ORM_CH_HEAD, (int32_t)k);
    MPUSH(res, ORM_CH_NSEG, (int32_t)m);
    MPUSH(res, ORM_CH_NCL, (int32_t)n);
    MPUSH(res, ORM_CH_OFFSET, (int32_t)res->a[ORM_CH_IDS].n);
    MPUSH(res, ORM_CH_NDF, (int32_t)(2 * n - 5));
    MPUSH(res, ORM_CH_STATUS, (int32_t)status);
    MPUSH(res, ORM_CH_INST, T[k].inst);
    MPUSH(res, ORM_CH_XREF, xout);
    MPUSH(res, ORM_CH_CHI2, chi2);
    MPUSH(res, ORM_CH_MARGIN, margin);
    for (int i = 0; i < 5; ++i) MPUSH(res, ORM_CH_PARAM, pout[i]);
    for (int i = 0; i < 15; ++i) MPUSH(res, ORM_CH_COV, cov[i]);
    for (int j = 0; j < m; ++j) MPUSH(res, ORM_CH_SEGS, segs[j]);
    for (int i = 0; i < n; ++i) MPUSH(res, ORM_CH_IDS, L[i].id);
  }
  free(T); free(first); free(best_out); free(best_in); free(chi_out); free(chi_in);
  free(chi2_out2); free(chi2_in2); free(marg); free(inst_of); free(L);
  return res;
oom:
  free(T); free(first); free(best_out); free(best_in); free(chi_out); free(chi_in);
  free(chi2_out2); free(chi2_in2); free(marg); free(inst_of); free(L);
  orm_free(res);
  return NULL;
}
