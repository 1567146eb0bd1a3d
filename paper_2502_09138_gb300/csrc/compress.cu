// Track-model compression of TPC clusters and its decoding (the paper:
// compression is part of "TPC Processing (Tracking, Clustering,
// Compression)", Table 1; GPU track-model decoding sped up the offline
// reconstruction by 1.2-3 %, Section 2).  Format (readings):
//   positions on a 50 um grid: Y = rint(200 y), Z = rint(200 z); row X =
//   rint(200 x_r), exact for the geometry's radii;
//   a track (clusters row-ascending): count, first row, Y0, Z0, charge0, then
//   per cluster the rows skipped, the residuals against the value predicted
//   from the previous decoded clusters of the track (previous value; line
//   through two; parabola through three, in exact integer arithmetic, the
//   quotient rounded half away from zero) and the charge;
//   clusters in no track: per (instance, row), sorted by (Y, Z, charge): the
//   count, Y (first absolute, then differences), Z, charge;
//   every value a LEB128 varint, signed values zigzag-mapped; tracks first,
//   then the rows; byte offsets per track and per row.
// GPU mapping: one thread per track or per row block; a length pass, a
// device scan of the lengths, a write pass (encoding); a count pass, a scan,
// a decode pass (decoding).  Integer arithmetic only, so the GPU and any
// other decoder agree to the bit.
#include "tpct_internal.cuh"

namespace tpct {
namespace {

constexpr int kBlockT = 256;

struct TmDev {
  int n_rows, n_inst;
  int32_t n_cap;                 // track capacity (scan length of the track part)
  int64_t n;                     // clusters
  int64_t X[kMaxRows];           // 200 x_r
  float xf[kMaxRows];
  // clusters
  const float *y, *z;
  const uint16_t* charge;
  const uint8_t* row;
  const int64_t* inst_off;
  // tracks
  const int32_t *n_tracks, *tr_off, *tr_ncl, *tr_ids;
  // workspace
  uint8_t* used;                 // [n]
  int32_t *blk_count, *blk_base, *blk_cursor;   // [n_inst * n_rows + 1]
  int32_t* blk_ids;              // [n] clusters in no track, grouped by block
  uint64_t* len;                 // [n_cap + n_blocks + 1] byte lengths, then their exclusive scan
  uint64_t* off;
  // output stream
  tpct_tm_stream out;
};

__device__ __forceinline__ int64_t qpos(float v) { return (int64_t)rint((double)v * 200.0); }

__device__ __forceinline__ int64_t div_round(int64_t n, int64_t d) {
  if (d < 0) { n = -n; d = -d; }
  return n >= 0 ? (2 * n + d) / (2 * d) : -((-2 * n + d) / (2 * d));
}

// value at x predicted from the previous k (1..3) points, oldest first
__device__ __forceinline__ int64_t predict(const int64_t* xs, const int64_t* vs, int k, int64_t x) {
  if (k == 1) return vs[2];
  if (k == 2) return vs[2] + div_round((vs[2] - vs[1]) * (x - xs[2]), xs[2] - xs[1]);
  const int64_t h1 = xs[1] - xs[0], h2 = xs[2] - xs[1], h02 = xs[2] - xs[0];
  const int64_t first = (vs[2] - vs[1]) * h1 * h02;
  const int64_t second = (vs[2] - vs[1]) * h1 - (vs[1] - vs[0]) * h2;
  return vs[2] + div_round((x - xs[2]) * (first + (x - xs[1]) * second), h1 * h2 * h02);
}

__device__ __forceinline__ uint64_t zig(int64_t v) { return v >= 0 ? (uint64_t)v << 1 : ((uint64_t)(-v) << 1) - 1; }
__device__ __forceinline__ int64_t unzig(uint64_t u) { return (u & 1u) ? -(int64_t)((u + 1) >> 1) : (int64_t)(u >> 1); }
__device__ __forceinline__ int vlen(uint64_t v) {
  int n = 1;
  while (v >= 128u) { v >>= 7; ++n; }
  return n;
}

// Writes (or, with dst == nullptr, only counts) a varint.
struct Sink {
  uint8_t* dst;
  int64_t pos;
  __device__ void u(uint64_t v) {
    if (!dst) { pos += vlen(v); return; }
    do {
      uint8_t b = (uint8_t)(v & 127u);
      v >>= 7;
      if (v) b |= 128u;
      dst[pos++] = b;
    } while (v);
  }
  __device__ void s(int64_t v) { u(zig(v)); }
};

struct Source {
  const uint8_t* p;
  int64_t pos;
  __device__ uint64_t u() {
    uint64_t v = 0;
    int sh = 0;
    while (true) {
      const uint8_t b = p[pos++];
      v |= (uint64_t)(b & 127u) << sh;
      if (!(b & 128u)) return v;
      sh += 7;
    }
  }
  __device__ int64_t s() { return unzig(u()); }
};

__device__ __forceinline__ int track_count(const TmDev& T) { return min(*T.n_tracks, T.n_cap); }

// one track's block (history shifts in from the right: xs[2] is the latest)
__device__ void code_track(const TmDev& T, int k, Sink& o) {
  const int32_t* c = T.tr_ids + T.tr_off[k];
  const int m = T.tr_ncl[k];
  int64_t xs[3] = {0, 0, 0}, ys[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
  o.u((uint64_t)m);
  for (int j = 0; j < m; ++j) {
    const int32_t i = c[j];
    const int r = T.row[i];
    const int64_t X = T.X[r], Y = qpos(T.y[i]), Z = qpos(T.z[i]);
    if (j == 0) {
      o.u((uint64_t)r); o.s(Y); o.s(Z);
    } else {
      const int kk = j < 3 ? j : 3;
      o.u((uint64_t)(r - (int)T.row[c[j - 1]] - 1));
      o.s(Y - predict(xs, ys, kk, X));
      o.s(Z - predict(xs, zs, kk, X));
    }
    o.u(T.charge ? T.charge[i] : 0u);
    xs[0] = xs[1]; xs[1] = xs[2]; xs[2] = X;
    ys[0] = ys[1]; ys[1] = ys[2]; ys[2] = Y;
    zs[0] = zs[1]; zs[1] = zs[2]; zs[2] = Z;
  }
}

__device__ __forceinline__ bool ucl_less(int64_t y1, int64_t z1, int q1, int64_t y2, int64_t z2, int q2) {
  return y1 < y2 || (y1 == y2 && (z1 < z2 || (z1 == z2 && q1 < q2)));
}

__device__ void code_block(const TmDev& T, int b, Sink& o) {
  const int32_t* ids = T.blk_ids + T.blk_base[b];
  const int m = T.blk_count[b];
  o.u((uint64_t)m);
  int64_t prev = 0;
  for (int j = 0; j < m; ++j) {
    const int32_t i = ids[j];
    const int64_t Y = qpos(T.y[i]);
    if (j == 0) o.s(Y); else o.u((uint64_t)(Y - prev));
    o.s(qpos(T.z[i]));
    o.u(T.charge ? T.charge[i] : 0u);
    prev = Y;
  }
}

__global__ void k_tm_mark(const __grid_constant__ TmDev T) {
  const int nt = track_count(T);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += gridDim.x * blockDim.x) {
    const int32_t* c = T.tr_ids + T.tr_off[k];
    for (int j = 0; j < T.tr_ncl[k]; ++j) T.used[c[j]] = 1;
  }
}

__global__ void k_tm_count(const __grid_constant__ TmDev T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (T.used[i]) continue;
    // instance of cluster i: binary search in the instance offsets
    int lo = 0, hi = T.n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (T.inst_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    atomicAdd(&T.blk_count[lo * T.n_rows + T.row[i]], 1);
  }
}

__global__ void k_tm_fill(const __grid_constant__ TmDev T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (T.used[i]) continue;
    int lo = 0, hi = T.n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (T.inst_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int b = lo * T.n_rows + T.row[i];
    T.blk_ids[T.blk_base[b] + atomicAdd(&T.blk_cursor[b], 1)] = (int32_t)i;
  }
}

// sort every block's clusters by (Y, Z, charge) (insertion sort: blocks hold
// a few dozen clusters), then its encoded length
__global__ void k_tm_block_len(const __grid_constant__ TmDev T) {
  const int nb = T.n_inst * T.n_rows;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    int32_t* ids = T.blk_ids + T.blk_base[b];
    const int m = T.blk_count[b];
    for (int j = 1; j < m; ++j) {
      const int32_t v = ids[j];
      const int64_t yv = qpos(T.y[v]), zv = qpos(T.z[v]);
      const int qv = T.charge ? T.charge[v] : 0;
      int a = j - 1;
      while (a >= 0) {
        const int32_t w = ids[a];
        if (!ucl_less(yv, zv, qv, qpos(T.y[w]), qpos(T.z[w]), T.charge ? T.charge[w] : 0)) break;
        ids[a + 1] = w;
        --a;
      }
      ids[a + 1] = v;
    }
    Sink o{nullptr, 0};
    code_block(T, b, o);
    T.len[T.n_cap + b] = (uint64_t)o.pos;
  }
}

__global__ void k_tm_track_len(const __grid_constant__ TmDev T) {
  const int nt = track_count(T);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < T.n_cap; k += gridDim.x * blockDim.x) {
    uint64_t l = 0;
    if (k < nt) {
      Sink o{nullptr, 0};
      code_track(T, k, o);
      l = (uint64_t)o.pos;
    }
    T.len[k] = l;
  }
}

__global__ void k_tm_write(const __grid_constant__ TmDev T) {
  const int nt = track_count(T);
  const int nb = T.n_inst * T.n_rows;
  const int64_t total = (int64_t)T.off[T.n_cap + nb];
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < T.n_cap + nb; w += gridDim.x * blockDim.x) {
    const int64_t at = (int64_t)T.off[w];
    if (w < T.n_cap) {
      if (w <= nt && T.out.track_offsets) T.out.track_offsets[w] = at;
      if (w >= nt) continue;
    } else {
      if (T.out.row_offsets) T.out.row_offsets[w - T.n_cap] = at;
    }
    if (at + (int64_t)T.len[w] > T.out.capacity) continue;
    Sink o{T.out.data, at};
    if (w < T.n_cap) code_track(T, w, o); else code_block(T, w - T.n_cap, o);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *T.out.n_bytes = total;
    if (nt == T.n_cap && T.out.track_offsets) T.out.track_offsets[nt] = (int64_t)T.off[T.n_cap];
    if (T.out.row_offsets) T.out.row_offsets[nb] = total;
  }
}

// ---------------------------------------------------------------- decoding
struct TdDev {
  int n_rows;
  int32_t n_tracks, n_blocks;
  int64_t X[kMaxRows];
  float xf[kMaxRows];
  const uint8_t* data;
  const int64_t *track_off, *row_off;
  uint64_t *cnt, *base;          // [n_tracks + n_blocks + 1]
  tpct_tm_decoded out;
};

__global__ void k_td_count(const __grid_constant__ TdDev D) {
  const int nw = D.n_tracks + D.n_blocks;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    Source s{D.data, w < D.n_tracks ? D.track_off[w] : D.row_off[w - D.n_tracks]};
    D.cnt[w] = s.u();
  }
}

__device__ __forceinline__ void put_cluster(const TdDev& D, int64_t o, int r, int64_t Y, int64_t Z, uint64_t q) {
  if (o >= D.out.capacity) return;
  D.out.x[o] = D.xf[r];
  D.out.y[o] = (float)((double)Y / 200.0);
  D.out.z[o] = (float)((double)Z / 200.0);
  D.out.charge[o] = (uint16_t)q;
  D.out.row[o] = (uint8_t)r;
}

__global__ void k_td_decode(const __grid_constant__ TdDev D) {
  const int nw = D.n_tracks + D.n_blocks;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    int64_t o = (int64_t)D.base[w];
    if (w < D.n_tracks) {
      Source s{D.data, D.track_off[w]};
      const int m = (int)s.u();
      int64_t xs[3] = {0, 0, 0}, ys[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
      int r = 0;
      for (int j = 0; j < m; ++j) {
        int64_t Y, Z;
        if (j == 0) {
          r = (int)s.u();
          Y = s.s();
          Z = s.s();
        } else {
          r = r + 1 + (int)s.u();
          const int kk = j < 3 ? j : 3;
          const int64_t X = D.X[r];
          Y = s.s() + predict(xs, ys, kk, X);
          Z = s.s() + predict(xs, zs, kk, X);
        }
        put_cluster(D, o++, r, Y, Z, s.u());
        xs[0] = xs[1]; xs[1] = xs[2]; xs[2] = D.X[r];
        ys[0] = ys[1]; ys[1] = ys[2]; ys[2] = Y;
        zs[0] = zs[1]; zs[1] = zs[2]; zs[2] = Z;
      }
    } else {
      const int b = w - D.n_tracks;
      const int r = b % D.n_rows;
      Source s{D.data, D.row_off[b]};
      const int64_t m = (int64_t)s.u();
      int64_t Y = 0;
      for (int64_t j = 0; j < m; ++j) {
        Y = j == 0 ? s.s() : Y + (int64_t)s.u();
        const int64_t Z = s.s();
        put_cluster(D, o++, r, Y, Z, s.u());
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *D.out.n = (int64_t)D.base[nw];
}

int blocks_for_t(int64_t work) {
  int64_t b = (work + kBlockT - 1) / kBlockT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

size_t tm_carve(char* base, int64_t n, int32_t cap, int32_t n_blocks, TmDev* T) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* { char* p = base ? base + off : nullptr; off += (b + 255) / 256 * 256 + 256; return p; };
  const size_t nw = (size_t)cap + n_blocks + 1;
  uint8_t* used = (uint8_t*)take((size_t)std::max<int64_t>(n, 1));
  int32_t* cnt = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* bas = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* cur = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* ids = (int32_t*)take(4 * (size_t)std::max<int64_t>(n, 1));
  uint64_t* len = (uint64_t*)take(8 * nw);
  uint64_t* off2 = (uint64_t*)take(8 * nw);
  uint64_t* tmp = (uint64_t*)take(8 * ((size_t)scan_tmp_elems((int64_t)nw) + 32));
  if (T) {
    T->used = used; T->blk_count = cnt; T->blk_base = bas; T->blk_cursor = cur; T->blk_ids = ids;
    T->len = len; T->off = off2;
  }
  (void)tmp;
  return off;
}

}  // namespace

size_t tm_encode_workspace_bytes(int64_t n, int32_t cap_tracks, int32_t n_blocks) {
  return tm_carve(nullptr, n, cap_tracks, n_blocks, nullptr);
}

size_t tm_decode_workspace_bytes(int32_t n_tracks, int32_t n_blocks) {
  const size_t nw = (size_t)n_tracks + n_blocks + 1;
  return 2 * ((8 * nw + 255) / 256 * 256 + 256) + (8 * ((size_t)scan_tmp_elems((int64_t)nw) + 32) + 511);
}

int enqueue_tm_encode(const double* row_x, int n_rows, const tpct_clusters& cl, int64_t n, const tpct_tracks_out& tr,
                      void* ws, size_t ws_bytes, const tpct_tm_stream& out, cudaStream_t s) {
  const int32_t nb = cl.n_instances * n_rows;
  const int32_t cap = tr.capacity_tracks;
  if (tm_carve(nullptr, n, cap, nb, nullptr) > ws_bytes) return -2;
  TmDev T{};
  tm_carve((char*)ws, n, cap, nb, &T);
  T.n_rows = n_rows; T.n_inst = cl.n_instances; T.n_cap = cap; T.n = n;
  for (int r = 0; r < n_rows; ++r) { T.X[r] = (int64_t)std::llrint(row_x[r] * 200.0); T.xf[r] = (float)row_x[r]; }
  T.y = cl.y; T.z = cl.z; T.charge = cl.charge; T.row = cl.row; T.inst_off = cl.sector_offsets;
  T.n_tracks = tr.n_tracks; T.tr_off = tr.offset; T.tr_ncl = tr.n_cl; T.tr_ids = tr.cluster_ids;
  T.out = out;
  // the scan's block sums follow the offsets array in the workspace layout
  uint64_t* tmp = (uint64_t*)((char*)T.off + ((8 * ((size_t)cap + nb + 1) + 255) / 256 * 256 + 256));
  int k = 0;
  cudaMemsetAsync(T.used, 0, (size_t)std::max<int64_t>(n, 1), s);
  cudaMemsetAsync(T.blk_count, 0, 4 * ((size_t)nb + 1), s);
  cudaMemsetAsync(T.blk_cursor, 0, 4 * ((size_t)nb + 1), s);
  k_tm_mark<<<blocks_for_t(cap), kBlockT, 0, s>>>(T); ++k;
  k_tm_count<<<blocks_for_t(n), kBlockT, 0, s>>>(T); ++k;
  launch_scan_i32(T.blk_count, T.blk_base, nb, tmp, s); k += 3;
  k_tm_fill<<<blocks_for_t(n), kBlockT, 0, s>>>(T); ++k;
  k_tm_block_len<<<blocks_for_t(nb), kBlockT, 0, s>>>(T); ++k;
  k_tm_track_len<<<blocks_for_t(cap), kBlockT, 0, s>>>(T); ++k;
  launch_scan_u64(T.len, T.off, (int64_t)cap + nb, tmp, s); k += 3;
  k_tm_write<<<blocks_for_t((int64_t)cap + nb), kBlockT, 0, s>>>(T); ++k;
  return k;
}

int enqueue_tm_decode(const double* row_x, int n_rows, const uint8_t* data, const int64_t* track_off, int32_t n_tracks,
                      const int64_t* row_off, int32_t n_blocks, void* ws, size_t ws_bytes, const tpct_tm_decoded& out,
                      cudaStream_t s) {
  if (tm_decode_workspace_bytes(n_tracks, n_blocks) > ws_bytes) return -2;
  TdDev D{};
  const size_t nw = (size_t)n_tracks + n_blocks + 1;
  char* p = (char*)ws;
  D.cnt = (uint64_t*)p;
  D.base = (uint64_t*)(p + (8 * nw + 255) / 256 * 256 + 256);
  uint64_t* tmp = (uint64_t*)(p + 2 * ((8 * nw + 255) / 256 * 256 + 256));
  tmp = (uint64_t*)(((uintptr_t)tmp + 255) / 256 * 256);
  D.n_rows = n_rows; D.n_tracks = n_tracks; D.n_blocks = n_blocks;
  for (int r = 0; r < n_rows; ++r) { D.X[r] = (int64_t)std::llrint(row_x[r] * 200.0); D.xf[r] = (float)row_x[r]; }
  D.data = data; D.track_off = track_off; D.row_off = row_off; D.out = out;
  int k = 0;
  k_td_count<<<blocks_for_t((int64_t)n_tracks + n_blocks), kBlockT, 0, s>>>(D); ++k;
  launch_scan_u64(D.cnt, D.base, (int64_t)n_tracks + n_blocks, tmp, s); k += 3;
  k_td_decode<<<blocks_for_t((int64_t)n_tracks + n_blocks), kBlockT, 0, s>>>(D); ++k;
  return k;
}

}  // namespace tpct
