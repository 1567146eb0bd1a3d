/*
 * cluster_oracle.c -- plain, single-threaded CPU oracle of TPC cluster
 * finding.  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library and
 * is never called by it; it shares no code, header or table with it.
 *
 * Cluster finding is the other named part of the paper's "TPC Processing
 * (Tracking, Clustering, Compression)" (Table 1, 99.37 % of synchronous
 * reconstruction).  The paper does not describe the algorithm; the steps
 * below are stated readings, each parameter passed in through orc_cf_params:
 *
 *   CF0 readout: row r has n_pad(r) = 2 ceil(x_r tan_half / pitch(r) - 1e-9)
 *       pads (pitch: inner rows / outer rows) and n_time time bins; a digit
 *       is one (pad, time) cell of one row with its ADC value; cells are
 *       unique within a row, any order; ADC values below 32768.
 *   CF1 peak: a digit of charge q at (p, t) is a peak iff q >= q_peak_min and,
 *       for each of its 8 neighbours n, q > Q(n) when n comes before (p, t)
 *       in (time, pad) order and q >= Q(n) otherwise (Q = 0 off the row's
 *       cells): the first cell of a plateau in that order is its peak.
 *   CF2 suppression: a peak P (charge q) is dropped iff some other peak P'
 *       (charge q') at Chebyshev distance exactly 2 is higher (q' > q, or
 *       q' == q and P' before P) and the cell M one step from P towards P'
 *       (on each axis where the offset is 2; 0 where it is 1 or 0) holds
 *       Q(M) >= q - valley_delta: no valley between the two.
 *   CF3 cluster: the 3 x 3 cells around a kept peak, plus every cell O at
 *       Chebyshev distance 2 with 0 < Q(O) <= Q(M_O), M_O the cell one step
 *       from the peak towards O as in CF2; charge-weighted mean and variance
 *       of the pad and time offsets from the peak; q_tot = the sum, q_max =
 *       the peak charge; flags bit 0 = peak on the first or last pad, bit 1 =
 *       on the first or last time bin.  Position: y = (pad + 0.5 - n_pad / 2)
 *       * pitch, drift length (time + 0.5) * time_bin, z = +-(z_max - drift)
 *       on side A / C (sector < 18 / >= 18), x = row radius.
 *   Order: clusters of a row in (time, pad) order of their peaks; rows in
 *       (instance, row) order.
 *
 * Everything is integer except the final means, variances and positions,
 * which are FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int n_rows;
  const double* row_x;        /* [n_rows] */
  double tan_half;
  double z_max;
  double pad_pitch_inner, pad_pitch_outer;
  int n_inner_rows;
  double time_bin;
  int n_time;
  int q_peak_min;
  int valley_delta;
} orc_cf_params;

enum { OCF_X, OCF_Y, OCF_Z, OCF_PAD, OCF_TIME, OCF_SPAD, OCF_STIME, OCF_QTOT, OCF_QMAX, OCF_ROW, OCF_FLAGS,
       OCF_INST, OCF_PEAK, OCF_N };

typedef struct { char* p; int64_t n, cap; size_t es; } cvec;

struct orc_cf_result {
  cvec a[OCF_N];
};
typedef struct orc_cf_result orc_cf_result;

static const size_t ocf_elem[OCF_N] = {8, 8, 8, 8, 8, 8, 8, 4, 2, 1, 1, 4, 8};

static int cpush(cvec* v, const void* e) {
  if (v->n == v->cap) {
    int64_t c = v->cap ? 2 * v->cap : 1024;
    char* q = (char*)realloc(v->p, (size_t)c * v->es);
    if (!q) return 1;
    v->p = q;
    v->cap = c;
  }
  memcpy(v->p + (size_t)v->n * v->es, e, v->es);
  v->n++;
  return 0;
}

void orc_cf_free(orc_cf_result* r) {
  if (!r) return;
  for (int i = 0; i < OCF_N; ++i) free(r->a[i].p);
  free(r);
}
int64_t orc_cf_count(const orc_cf_result* r) { return r ? r->a[OCF_INST].n : -1; }
const void* orc_cf_array(const orc_cf_result* r, int w) { return (r && w >= 0 && w < OCF_N) ? r->a[w].p : NULL; }

/* CF0 */
static double row_pitch(const orc_cf_params* P, int r) {
  return r < P->n_inner_rows ? P->pad_pitch_inner : P->pad_pitch_outer;
}
static int row_pads(const orc_cf_params* P, int r) {
  return 2 * (int)ceil(P->row_x[r] * P->tan_half / row_pitch(P, r) - 1e-9);
}

/* charge of cell (p, t) of the current row's map, 0 off the row */
static int Q(const int* map, int np, int nt, int p, int t) {
  if (p < 0 || p >= np || t < 0 || t >= nt) return 0;
  return map[p * nt + t];
}

/* (t1, p1) before (t0, p0) in (time, pad) order */
static int before(int p1, int t1, int p0, int t0) { return t1 < t0 || (t1 == t0 && p1 < p0); }

/* one step from 0 towards an offset d in {-2..2}: +-1 where |d| == 2, else 0 */
static int half_step(int d) { return d == 2 ? 1 : (d == -2 ? -1 : 0); }

/* (time, pad) order of two digits (qsort over digit indices) */
static const uint16_t *g_pad, *g_time;
static int cmp_time_pad(const void* a, const void* b) {
  const int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  if (g_time[i] != g_time[j]) return g_time[i] < g_time[j] ? -1 : 1;
  return (g_pad[i] > g_pad[j]) - (g_pad[i] < g_pad[j]);
}

/* CF1 */
static int is_peak(const int* map, int np, int nt, int p, int t, int qmin) {
  int q = Q(map, np, nt, p, t);
  if (q < qmin) return 0;
  for (int dt = -1; dt <= 1; ++dt)
    for (int dp = -1; dp <= 1; ++dp) {
      if (dp == 0 && dt == 0) continue;
      int qn = Q(map, np, nt, p + dp, t + dt);
      if (before(p + dp, t + dt, p, t)) {
        if (!(q > qn)) return 0;
      } else {
        if (!(q >= qn)) return 0;
      }
    }
  return 1;
}

/* CF2 */
static int suppressed(const int* map, const unsigned char* pk, int np, int nt, int p, int t, int delta) {
  int q = Q(map, np, nt, p, t);
  for (int dt = -2; dt <= 2; ++dt)
    for (int dp = -2; dp <= 2; ++dp) {
      if (abs(dp) != 2 && abs(dt) != 2) continue;           /* Chebyshev distance 2 only */
      int p2 = p + dp, t2 = t + dt;
      if (p2 < 0 || p2 >= np || t2 < 0 || t2 >= nt || !pk[p2 * nt + t2]) continue;
      int q2 = map[p2 * nt + t2];
      if (!(q2 > q || (q2 == q && before(p2, t2, p, t)))) continue;
      int qm = Q(map, np, nt, p + half_step(dp), t + half_step(dt));
      if (qm >= q - delta) return 1;
    }
  return 0;
}

orc_cf_result* orc_find_clusters(const orc_cf_params* P, int64_t n_inst, const int32_t* inst_sector,
                                 const int64_t* row_offsets, const uint16_t* pad, const uint16_t* time,
                                 const uint16_t* adc, int* err) {
  *err = 0;
  if (!P || !row_offsets || n_inst < 0 || P->n_rows <= 0 || P->n_time <= 0) { *err = 1; return NULL; }
  orc_cf_result* res = (orc_cf_result*)calloc(1, sizeof(orc_cf_result));
  if (!res) { *err = 4; return NULL; }
  for (int i = 0; i < OCF_N; ++i) res->a[i].es = ocf_elem[i];
  int np_max = 0;
  for (int r = 0; r < P->n_rows; ++r)
    if (row_pads(P, r) > np_max) np_max = row_pads(P, r);
  const int nt = P->n_time;
  int* map = (int*)calloc((size_t)np_max * nt, sizeof(int));
  unsigned char* pk = (unsigned char*)calloc((size_t)np_max * nt, 1);
  int64_t max_row = 1;
  for (int64_t k = 0; k < n_inst * P->n_rows; ++k)
    if (row_offsets[k + 1] - row_offsets[k] > max_row) max_row = row_offsets[k + 1] - row_offsets[k];
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)max_row);
  if (!map || !pk || !order) { free(map); free(pk); free(order); orc_cf_free(res); *err = 4; return NULL; }
  for (int64_t inst = 0; inst < n_inst; ++inst) {
    const int side_c = inst_sector[inst] >= 18;
    for (int r = 0; r < P->n_rows; ++r) {
      const int64_t b = row_offsets[inst * P->n_rows + r], e = row_offsets[inst * P->n_rows + r + 1];
      const int np = row_pads(P, r);
      const double pitch = row_pitch(P, r);
      /* the row's map */
      for (int64_t i = b; i < e; ++i) {
        if (pad[i] >= np || time[i] >= nt || adc[i] >= 32768) { *err = 3; goto fail; }
        if (map[pad[i] * nt + time[i]] != 0) { *err = 2; goto fail; }
        map[pad[i] * nt + time[i]] = adc[i];
      }
      for (int64_t i = b; i < e; ++i)
        pk[pad[i] * nt + time[i]] = (unsigned char)is_peak(map, np, nt, pad[i], time[i], P->q_peak_min);
      /* kept peaks of the row, in (time, pad) order */
      int64_t nk = 0;
      for (int64_t i = b; i < e; ++i) {
        const int p = pad[i], t = time[i];
        if (pk[p * nt + t] && !suppressed(map, pk, np, nt, p, t, P->valley_delta)) order[nk++] = i;
      }
      g_pad = pad; g_time = time;
      qsort(order, (size_t)nk, sizeof(int64_t), cmp_time_pad);
      for (int64_t kq = 0; kq < nk; ++kq) {
        const int64_t i = order[kq];
        const int p = pad[i], t = time[i];
        /* CF3 */
        int64_t s0 = 0, sp = 0, st = 0, spp = 0, stt = 0;
        for (int dt = -2; dt <= 2; ++dt)
          for (int dp = -2; dp <= 2; ++dp) {
            const int qc = Q(map, np, nt, p + dp, t + dt);
            if (qc <= 0) continue;
            if (abs(dp) == 2 || abs(dt) == 2) {
              const int qm = Q(map, np, nt, p + half_step(dp), t + half_step(dt));
              if (!(qc <= qm)) continue;
            }
            s0 += qc; sp += (int64_t)qc * dp; st += (int64_t)qc * dt;
            spp += (int64_t)qc * dp * dp; stt += (int64_t)qc * dt * dt;
          }
        const double mp = (double)sp / (double)s0, mt = (double)st / (double)s0;
        double vp = (double)spp / (double)s0 - mp * mp, vt = (double)stt / (double)s0 - mt * mt;
        if (vp < 0.0) vp = 0.0;
        if (vt < 0.0) vt = 0.0;
        const double cpad = (double)p + mp, ctime = (double)t + mt;
        const double y = (cpad + 0.5 - 0.5 * (double)np) * pitch;
        const double drift = (ctime + 0.5) * P->time_bin;
        const double z = side_c ? -(P->z_max - drift) : (P->z_max - drift);
        const double x = P->row_x[r];
        const double sgp = sqrt(vp), sgt = sqrt(vt);
        const uint32_t qtot = (uint32_t)s0;
        const uint16_t qmax = (uint16_t)map[p * nt + t];
        const uint8_t rowv = (uint8_t)r;
        const uint8_t flags = (uint8_t)((p == 0 || p == np - 1 ? 1 : 0) | (t == 0 || t == nt - 1 ? 2 : 0));
        const int32_t instv = (int32_t)inst;
        const int64_t peak = i;
        if (cpush(&res->a[OCF_X], &x) || cpush(&res->a[OCF_Y], &y) || cpush(&res->a[OCF_Z], &z) ||
            cpush(&res->a[OCF_PAD], &cpad) || cpush(&res->a[OCF_TIME], &ctime) ||
            cpush(&res->a[OCF_SPAD], &sgp) || cpush(&res->a[OCF_STIME], &sgt) ||
            cpush(&res->a[OCF_QTOT], &qtot) || cpush(&res->a[OCF_QMAX], &qmax) ||
            cpush(&res->a[OCF_ROW], &rowv) || cpush(&res->a[OCF_FLAGS], &flags) ||
            cpush(&res->a[OCF_INST], &instv) || cpush(&res->a[OCF_PEAK], &peak)) {
          *err = 4;
          goto fail;
        }
      }
      /* clear the row's cells */
      for (int64_t i = b; i < e; ++i) { map[pad[i] * nt + time[i]] = 0; pk[pad[i] * nt + time[i]] = 0; }
    }
  }
  free(map);
  free(pk);
  free(order);
  return res;
fail:
  free(map);
  free(pk);
  free(order);
  orc_cf_free(res);
  return NULL;
}
