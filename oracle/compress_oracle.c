/*
 * compress_oracle.c -- plain, single-threaded CPU oracle of track-model
 * compression of TPC clusters and of its decoding.  TEST INFRASTRUCTURE
 * ONLY: it exists to check the CUDA library and is never called by it; it
 * shares no code, header or table with it.
 *
 * The paper counts TPC compression inside "TPC Processing (Tracking,
 * Clustering, Compression)" (Table 1), calls it critical for storage
 * (Section 1) and reports that porting the track-model decoding to GPUs sped
 * up the offline reconstruction by 1.2-3 % (Section 2).  It does not give the
 * format; the readings below are stated here and in the C ABI:
 *
 *   TM1 quantisation: y and z of a cluster become integers Y = rint(200 y),
 *       Z = rint(200 z) (a 50 um grid, 1/4 of the smallest cluster sigma /
 *       sqrt(12) below it); row radii are multiples of 0.05 cm, so a row's
 *       X = rint(200 x_r) is exact.
 *   TM2 tracks: a track's clusters (row-ascending) are coded as: the cluster
 *       count, the first row, Y0, Z0, charge0; then for every further cluster
 *       the number of rows skipped since the previous one, the residuals
 *       Y - P_y, Z - P_z against a prediction from the already decoded
 *       clusters of the same track, and the charge.  Prediction of cluster k
 *       at X_k: k = 1: the previous value; k = 2: the line through clusters
 *       0, 1; k >= 3: the parabola through clusters k-3, k-2, k-1 (Lagrange
 *       form in exact integer arithmetic, the quotient rounded half away from
 *       zero).  Everything is integer, so the decoder repeats it bit for bit.
 *   TM3 clusters in no track: per (instance, row), sorted by (Y, Z, charge):
 *       the count, then Y as a difference to the previous one (the first
 *       absolute), Z and the charge.
 *   TM4 bytes: every value is a LEB128 varint (7 bits per byte, low first);
 *       signed values are zigzag-mapped first (v >= 0 -> 2v, v < 0 -> -2v-1).
 *       Tracks come first in output order, then the rows; per track and per
 *       row the byte offset of its block.
 *   Decoding returns x, y = Y / 200, z = Z / 200 (float), charge, row, in the
 *   order tracks (their clusters row-ascending), then rows (sorted as TM3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int n_rows;
  const double* row_x;   /* [n_rows] */
} orc_tm_geometry;

static int64_t qpos(float v) { return (int64_t)rint((double)v * 200.0); }
static int64_t row_X(const orc_tm_geometry* g, int r) { return (int64_t)rint(g->row_x[r] * 200.0); }

/* round half away from zero of n / d, d > 0 */
static int64_t div_round(int64_t n, int64_t d) {
  if (d < 0) { n = -n; d = -d; }
  return n >= 0 ? (2 * n + d) / (2 * d) : -((-2 * n + d) / (2 * d));
}

/* Prediction of the value at x from the previous k points (k = 1, 2 or 3),
 * oldest first.  k = 3: Newton's form of the parabola through the three,
 * v2 + (x - a2) f[a2, a1] + (x - a2)(x - a1) f[a2, a1, a0], with the divided
 * differences over the common denominator h1 h2 (a2 - a0) (h1 = a1 - a0,
 * h2 = a2 - a1) so that a single rounded division remains. */
static int64_t predict(const int64_t* xs, const int64_t* vs, int k, int64_t x) {
  if (k == 1) return vs[0];
  if (k == 2) return vs[1] + div_round((vs[1] - vs[0]) * (x - xs[1]), xs[1] - xs[0]);
  const int64_t h1 = xs[1] - xs[0], h2 = xs[2] - xs[1], h02 = xs[2] - xs[0];
  const int64_t first = (vs[2] - vs[1]) * h1 * h02;                    /* f[a2, a1] * den */
  const int64_t second = (vs[2] - vs[1]) * h1 - (vs[1] - vs[0]) * h2;  /* f[a2, a1, a0] * den */
  return vs[2] + div_round((x - xs[2]) * (first + (x - xs[1]) * second), h1 * h2 * h02);
}

/* ---------------------------------------------------------------- byte stream */
typedef struct { uint8_t* p; int64_t n, cap; } bytes;

static int put_u(bytes* b, uint64_t v) {
  for (;;) {
    if (b->n == b->cap) {
      int64_t c = b->cap ? 2 * b->cap : 4096;
      uint8_t* q = (uint8_t*)realloc(b->p, (size_t)c);
      if (!q) return 1;
      b->p = q;
      b->cap = c;
    }
    uint8_t byte = (uint8_t)(v & 127u);
    v >>= 7;
    if (v) byte |= 128u;
    b->p[b->n++] = byte;
    if (!v) return 0;
  }
}
static uint64_t zig(int64_t v) { return v >= 0 ? (uint64_t)v << 1 : (((uint64_t)(-v)) << 1) - 1; }
static int put_s(bytes* b, int64_t v) { return put_u(b, zig(v)); }

static uint64_t get_u(const uint8_t* p, int64_t* pos) {
  uint64_t v = 0;
  int sh = 0;
  for (;;) {
    const uint8_t byte = p[(*pos)++];
    v |= (uint64_t)(byte & 127u) << sh;
    if (!(byte & 128u)) return v;
    sh += 7;
  }
}
static int64_t unzig(uint64_t u) { return (u & 1u) ? -(int64_t)((u + 1) >> 1) : (int64_t)(u >> 1); }
static int64_t get_s(const uint8_t* p, int64_t* pos) { return unzig(get_u(p, pos)); }

typedef struct {
  bytes data;
  int64_t* track_off;   /* [n_tracks + 1] */
  int64_t* row_off;     /* [n_inst * n_rows + 1] */
  int64_t n_tracks, n_blocks;
} orc_tm_stream;

void orc_tm_free(orc_tm_stream* s) {
  if (!s) return;
  free(s->data.p);
  free(s->track_off);
  free(s->row_off);
  free(s);
}
int64_t orc_tm_bytes(const orc_tm_stream* s) { return s ? s->data.n : -1; }
const uint8_t* orc_tm_data(const orc_tm_stream* s) { return s ? s->data.p : NULL; }
const int64_t* orc_tm_track_offsets(const orc_tm_stream* s) { return s ? s->track_off : NULL; }
const int64_t* orc_tm_row_offsets(const orc_tm_stream* s) { return s ? s->row_off : NULL; }

typedef struct { int64_t y, z; int32_t q; } ucl;
static int cmp_ucl(const void* a, const void* b) {
  const ucl *u = (const ucl*)a, *v = (const ucl*)b;
  if (u->y != v->y) return u->y < v->y ? -1 : 1;
  if (u->z != v->z) return u->z < v->z ? -1 : 1;
  return (u->q > v->q) - (u->q < v->q);
}

/* Encode.  Clusters: n, grouped by instance (inst_off[n_inst + 1]), y, z,
 * charge, row.  Tracks: n_tracks with their clusters in ids[off[k] ..
 * off[k] + ncl[k]) (ids are cluster positions, rows ascending). */
orc_tm_stream* orc_tm_encode(const orc_tm_geometry* g, int64_t n, int64_t n_inst, const int64_t* inst_off,
                             const float* y, const float* z, const uint16_t* charge, const uint8_t* row,
                             int64_t n_tracks, const int32_t* off, const int32_t* ncl, const int32_t* ids) {
  orc_tm_stream* s = (orc_tm_stream*)calloc(1, sizeof(orc_tm_stream));
  unsigned char* used = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
  ucl* tmp = NULL;
  if (!s || !used) goto fail;
  s->n_tracks = n_tracks;
  s->n_blocks = n_inst * g->n_rows;
  s->track_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_tracks + 1));
  s->row_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n_blocks + 1));
  if (!s->track_off || !s->row_off) goto fail;
  for (int64_t k = 0; k < n_tracks; ++k) {
    s->track_off[k] = s->data.n;
    const int32_t* c = ids + off[k];
    const int m = ncl[k];
    int64_t xs[3], ys[3], zs[3];
    if (put_u(&s->data, (uint64_t)m)) goto fail;
    for (int j = 0; j < m; ++j) {
      const int32_t i = c[j];
      used[i] = 1;
      const int64_t X = row_X(g, row[i]), Y = qpos(y[i]), Z = qpos(z[i]);
      if (j == 0) {
        if (put_u(&s->data, row[i]) || put_s(&s->data, Y) || put_s(&s->data, Z)) goto fail;
      } else {
        const int kk = j < 3 ? j : 3;
        if (put_u(&s->data, (uint64_t)(row[i] - row[c[j - 1]] - 1)) ||
            put_s(&s->data, Y - predict(xs + 3 - kk, ys + 3 - kk, kk, X)) ||
            put_s(&s->data, Z - predict(xs + 3 - kk, zs + 3 - kk, kk, X)))
          goto fail;
      }
      if (put_u(&s->data, charge ? charge[i] : 0)) goto fail;
      /* history: the last three points, oldest first */
      xs[0] = xs[1]; ys[0] = ys[1]; zs[0] = zs[1];
      xs[1] = xs[2]; ys[1] = ys[2]; zs[1] = zs[2];
      xs[2] = X; ys[2] = Y; zs[2] = Z;
    }
  }
  s->track_off[n_tracks] = s->data.n;
  tmp = (ucl*)malloc(sizeof(ucl) * (size_t)(n > 0 ? n : 1));
  if (!tmp) goto fail;
  for (int64_t inst = 0; inst < n_inst; ++inst) {
    for (int r = 0; r < g->n_rows; ++r) {
      s->row_off[inst * g->n_rows + r] = s->data.n;
      int64_t m = 0;
      for (int64_t i = inst_off[inst]; i < inst_off[inst + 1]; ++i)
        if (!used[i] && row[i] == r) {
          tmp[m].y = qpos(y[i]); tmp[m].z = qpos(z[i]); tmp[m].q = charge ? charge[i] : 0;
          ++m;
        }
      qsort(tmp, (size_t)m, sizeof(ucl), cmp_ucl);
      if (put_u(&s->data, (uint64_t)m)) goto fail;
      int64_t prev = 0;
      for (int64_t j = 0; j < m; ++j) {
        if ((j == 0 ? put_s(&s->data, tmp[j].y) : put_u(&s->data, (uint64_t)(tmp[j].y - prev))) ||
            put_s(&s->data, tmp[j].z) || put_u(&s->data, (uint64_t)tmp[j].q))
          goto fail;
        prev = tmp[j].y;
      }
    }
  }
  s->row_off[s->n_blocks] = s->data.n;
  free(used);
  free(tmp);
  return s;
fail:
  free(used);
  free(tmp);
  orc_tm_free(s);
  return NULL;
}

/* Decode into caller arrays of capacity n_max; returns the clusters written
 * or -1 (more than n_max). */
int64_t orc_tm_decode(const orc_tm_geometry* g, const uint8_t* data, int64_t n_tracks, const int64_t* track_off,
                      int64_t n_blocks, const int64_t* row_off, int64_t n_max, float* x, float* y, float* z,
                      uint16_t* charge, uint8_t* row) {
  int64_t o = 0;
  for (int64_t k = 0; k < n_tracks; ++k) {
    int64_t pos = track_off[k];
    const int m = (int)get_u(data, &pos);
    int64_t xs[3], ys[3], zs[3];
    int r = 0;
    for (int j = 0; j < m; ++j) {
      int64_t Y, Z;
      if (j == 0) {
        r = (int)get_u(data, &pos);
        Y = get_s(data, &pos);
        Z = get_s(data, &pos);
      } else {
        r = r + 1 + (int)get_u(data, &pos);
        const int64_t X = row_X(g, r);
        const int kk = j < 3 ? j : 3;
        Y = get_s(data, &pos) + predict(xs + 3 - kk, ys + 3 - kk, kk, X);
        Z = get_s(data, &pos) + predict(xs + 3 - kk, zs + 3 - kk, kk, X);
      }
      const uint64_t q = get_u(data, &pos);
      if (o >= n_max) return -1;
      x[o] = (float)g->row_x[r]; y[o] = (float)((double)Y / 200.0); z[o] = (float)((double)Z / 200.0);
      charge[o] = (uint16_t)q; row[o] = (uint8_t)r;
      ++o;
      xs[0] = xs[1]; ys[0] = ys[1]; zs[0] = zs[1];
      xs[1] = xs[2]; ys[1] = ys[2]; zs[1] = zs[2];
      xs[2] = row_X(g, r); ys[2] = Y; zs[2] = Z;
    }
  }
  for (int64_t b = 0; b < n_blocks; ++b) {
    int64_t pos = row_off[b];
    const int r = (int)(b % g->n_rows);
    const int64_t m = (int64_t)get_u(data, &pos);
    int64_t Y = 0;
    for (int64_t j = 0; j < m; ++j) {
      Y = j == 0 ? get_s(data, &pos) : Y + (int64_t)get_u(data, &pos);
      const int64_t Z = get_s(data, &pos);
      const uint64_t q = get_u(data, &pos);
      if (o >= n_max) return -1;
      x[o] = (float)g->row_x[r]; y[o] = (float)((double)Y / 200.0); z[o] = (float)((double)Z / 200.0);
      charge[o] = (uint16_t)q; row[o] = (uint8_t)r;
      ++o;
    }
  }
  return o;
}
