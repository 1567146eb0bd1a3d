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
// GPU mapping (encoding): one warp per track or row block, one lane per
// cluster -- a cluster's residuals depend only on the quantised input, so no
// lane waits for another; a length pass (which also sorts each block in the
// warp), a device scan of the lengths, a write pass in which a warp scan of
// the clusters' lengths places every lane's bytes (coalesced stores).
// Decoding: one thread per track or block (the predictor chains every
// cluster to the decoded previous ones); a count pass, a scan, a decode pass.
// Integer arithmetic only, so the GPU and any other decoder agree to the bit.
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
  uint32_t* used;                // [n] number of tracks listing each cluster
  uint4* code;                   // [n] a cluster's bytes, coded once by the length pass (<= 16)
  uint8_t* clen;                 // [n] their count; 0: not staged (coded again by the write pass)
  int32_t *blk_count, *blk_base, *blk_cursor;   // [n_inst * n_rows + 1]
  int32_t* blk_ids;              // [n] clusters in no track, grouped by block
  int32_t* blk_sorted;           // [n] the same, each block sorted by (Y, Z, charge)
  uint64_t* len;                 // [n_cap + n_blocks + 1] byte lengths, then their exclusive scan
  uint64_t* off;
  // output stream
  tpct_tm_stream out;
};

// rint(200 v) of a float v, from its IEEE-754 fields with integer
// arithmetic only (the FP64 pipe is 1/64 of the FP32 rate on this part):
// v = m 2^(E-150) with a 24-bit m, so 200 v = 25 m 2^(E-147) exactly; a right
// shift rounds half to even like rint.  Values beyond the int64 shift range
// and non-finite ones take the double expression.
__device__ __forceinline__ int64_t qpos(float v) {
  const uint32_t bits = __float_as_uint(v);
  const int E = (int)((bits >> 23) & 0xffu);
  if (E == 0) return 0;                              // |200 v| < 0.5
  const int sh = E - 147;
  if (E == 255 || sh > 34) return (int64_t)rint((double)v * 200.0);
  const uint64_t P = 25ull * ((bits & 0x7fffffu) | 0x800000u);
  uint64_t q;
  if (sh >= 0) {
    q = P << sh;
  } else {
    const int s = -sh;
    if (s >= 31) return 0;                           // P < 2^29: below one half
    q = P >> s;
    const uint64_t rem = P & ((1ull << s) - 1u), half = 1ull << (s - 1);
    if (rem > half || (rem == half && (q & 1u))) ++q;
  }
  return (bits >> 31) ? -(int64_t)q : (int64_t)q;
}

// floor(a / b): a quotient estimate from a float division, then the exact
// correction by the remainder (the estimate is within 2 of the quotient when
// the quotient is below 2^20); other operands use the 64-bit division.
// 64-bit integer <-> float conversions run on the FP64 pipe of this part, so
// the operands are converted in 32-bit halves (the estimate only has to be
// within a few units of the quotient).
__device__ __forceinline__ float u64_to_float_approx(uint64_t v) {
  return __fmaf_rn((float)(uint32_t)(v >> 32), 4294967296.f, (float)(uint32_t)v);
}

__device__ __forceinline__ uint64_t udiv(uint64_t a, uint64_t b) {
  if (a < (1ull << 62) && b < (1ull << 40)) {
    const float qf = __fdiv_rn(u64_to_float_approx(a), u64_to_float_approx(b));
    if (qf < 1048576.f) {
      int64_t q = (int64_t)(int32_t)qf;
      int64_t r = (int64_t)a - q * (int64_t)b;
      for (int k = 0; k < 4 && r < 0; ++k) { --q; r += (int64_t)b; }
      for (int k = 0; k < 4 && r >= (int64_t)b; ++k) { ++q; r -= (int64_t)b; }
      if (r >= 0 && r < (int64_t)b) return (uint64_t)q;
    }
  }
  return a / b;
}

__device__ __forceinline__ int64_t div_round(int64_t n, int64_t d) {
  if (d < 0) { n = -n; d = -d; }
  return n >= 0 ? (int64_t)udiv((uint64_t)(2 * n + d), (uint64_t)(2 * d))
                : -(int64_t)udiv((uint64_t)(-2 * n + d), (uint64_t)(2 * d));
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

// Reads the varints of one stream item: bytes [pos, end).  The encoder's own
// streams never trip a check; the decoder runs on caller data, so a read past
// the item's end or a varint longer than 10 bytes (more than 64 bits) sets
// `bad` and returns 0 instead of reading further.
struct Source {
  const uint8_t* p;
  int64_t pos, end;
  bool bad;
  __device__ uint64_t u() {
    uint64_t v = 0;
    for (int i = 0; i < 10; ++i) {
      if (pos >= end) { bad = true; return 0; }
      const uint8_t b = p[pos++];
      v |= (uint64_t)(b & 127u) << (7 * i);
      if (!(b & 128u)) return v;
    }
    bad = true;
    return 0;
  }
  __device__ int64_t s() { return unzig(u()); }
};

__device__ __forceinline__ int track_count(const TmDev& T) { return min(*T.n_tracks, T.n_cap); }

// Writes a varint at dst + pos (pos advanced).
__device__ __forceinline__ void put_u(uint8_t* dst, int64_t& pos, uint64_t v) {
  do {
    uint8_t b = (uint8_t)(v & 127u);
    v >>= 7;
    if (v) b |= 128u;
    dst[pos++] = b;
  } while (v);
}

// The values one cluster of a work item contributes to the stream.  Every
// value depends only on the quantised input (the predictor uses the exact
// quantised positions the decoder reproduces), so the clusters of an item
// are coded independently, one per lane.
struct CodedCluster {
  uint64_t v0;              // rows skipped (first cluster of a track: its row); blocks: Y or Y step
  int64_t s1, s2;           // tracks: Y and Z residuals (first: Y, Z); blocks: s2 = Z, s1 unused
  uint32_t q;
  bool block;
  __device__ int length() const {
    return block ? vlen(v0) + vlen(zig(s2)) + vlen(q) : vlen(v0) + vlen(zig(s1)) + vlen(zig(s2)) + vlen(q);
  }
  // the bytes in a 16-byte word (only for length() <= 16)
  __device__ uint4 pack() const {
    uint64_t lo = 0, hi = 0;
    int pos = 0;
    auto put = [&](uint64_t v) {
      do {
        uint64_t b = v & 127u;
        v >>= 7;
        if (v) b |= 128u;
        if (pos < 8) lo |= b << (8 * pos); else hi |= b << (8 * (pos - 8));
        ++pos;
      } while (v);
    };
    put(v0);
    if (!block) put(zig(s1));
    put(zig(s2));
    put(q);
    return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
  }
  __device__ void write(uint8_t* dst, int64_t pos) const {
    if (block) {
      put_u(dst, pos, v0);
      put_u(dst, pos, zig(s2));
      put_u(dst, pos, q);
    } else {
      put_u(dst, pos, v0);
      put_u(dst, pos, zig(s1));
      put_u(dst, pos, zig(s2));
      put_u(dst, pos, q);
    }
  }
};

// cluster j of track k (j < its count)
__device__ CodedCluster code_track_cluster(const TmDev& T, const int32_t* c, int j) {
  CodedCluster o;
  o.block = false;
  const int32_t i = c[j];
  const int r = T.row[i];
  o.q = T.charge ? T.charge[i] : 0u;
  const int64_t Y = qpos(T.y[i]), Z = qpos(T.z[i]);
  if (j == 0) {
    o.v0 = (uint64_t)r;
    o.s1 = Y;
    o.s2 = Z;
    return o;
  }
  // the previous kk points, oldest first in slots 3 - kk .. 2
  const int kk = j < 3 ? j : 3;
  int64_t xs[3] = {0, 0, 0}, ys[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
  int r_prev = 0;
#pragma unroll
  for (int d = 1; d <= 3; ++d) {
    if (d > kk) break;
    const int32_t ip = c[j - d];
    const int rp = T.row[ip];
    if (d == 1) r_prev = rp;
    xs[3 - d] = T.X[rp];
    ys[3 - d] = qpos(T.y[ip]);
    zs[3 - d] = qpos(T.z[ip]);
  }
  const int64_t X = T.X[r];
  o.v0 = (uint64_t)(r - r_prev - 1);
  o.s1 = Y - predict(xs, ys, kk, X);
  o.s2 = Z - predict(xs, zs, kk, X);
  return o;
}

// Keeps a cluster's bytes for the write pass when they fit 16 bytes and the
// cluster is coded in one place only (a cluster listed by two tracks is
// coded again by each).
__device__ __forceinline__ void stage_code(const TmDev& T, int32_t i, const CodedCluster& cc, int len, bool unique) {
  const bool keep = unique && len <= 16;
  if (keep) T.code[i] = cc.pack();
  T.clen[i] = keep ? (uint8_t)len : (uint8_t)0;
}

// The same coding from values already at hand: this cluster's row, Y, Z, X
// and charge, and the previous three clusters' rows, X, Y, Z (slot 2 the
// latest; slots before the track's start unused).
__device__ __forceinline__ CodedCluster code_track_values(int j, int r, int64_t X, int64_t Y, int64_t Z, uint32_t q,
                                                          int r_prev, const int64_t* xs, const int64_t* ys,
                                                          const int64_t* zs) {
  CodedCluster o;
  o.block = false;
  o.q = q;
  if (j == 0) {
    o.v0 = (uint64_t)r;
    o.s1 = Y;
    o.s2 = Z;
    return o;
  }
  const int kk = j < 3 ? j : 3;
  o.v0 = (uint64_t)(r - r_prev - 1);
  o.s1 = Y - predict(xs, ys, kk, X);
  o.s2 = Z - predict(xs, zs, kk, X);
  return o;
}

__device__ __forceinline__ int64_t shfl_up64(int64_t v, int d) {
  const uint32_t lo = __shfl_up_sync(0xffffffffu, (uint32_t)(uint64_t)v, d);
  const uint32_t hi = __shfl_up_sync(0xffffffffu, (uint32_t)((uint64_t)v >> 32), d);
  return (int64_t)(((uint64_t)hi << 32) | lo);
}
__device__ __forceinline__ int64_t shfl_idx64(int64_t v, int src) {
  const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)(uint64_t)v, src);
  const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)((uint64_t)v >> 32), src);
  return (int64_t)(((uint64_t)hi << 32) | lo);
}

// Byte length of track k, one lane per cluster; every cluster's inputs are
// loaded and quantised once, and its three predecessors come from the
// neighbouring lanes (or, at a chunk's start, from the previous chunk's last
// three lanes).  Stages the bytes like the block path.
__device__ uint64_t track_length_warp(const TmDev& T, const int32_t* c, int m, int lane) {
  uint64_t l = 0;
  int64_t cx[3] = {0, 0, 0}, cy[3] = {0, 0, 0}, cz[3] = {0, 0, 0};   // clusters j0-3 .. j0-1
  int cr = 0;                                                        // row of cluster j0-1
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int j = j0 + lane;
    const bool valid = j < m;
    const int32_t i = valid ? c[j] : 0;
    const int r = valid ? (int)T.row[i] : 0;
    const int64_t X = T.X[r];
    const int64_t Y = valid ? qpos(T.y[i]) : 0, Z = valid ? qpos(T.z[i]) : 0;
    const uint32_t q = valid && T.charge ? T.charge[i] : 0u;
    int64_t xs[3], ys[3], zs[3];
    int r_prev;
#pragma unroll
    for (int d = 1; d <= 3; ++d) {
      const int64_t xu = shfl_up64(X, d), yu = shfl_up64(Y, d), zu = shfl_up64(Z, d);
      const int k = 3 + lane - d;          // carry slot when lane < d
      const bool from_carry = lane < d;
      xs[3 - d] = from_carry ? (k == 2 ? cx[2] : k == 1 ? cx[1] : cx[0]) : xu;
      ys[3 - d] = from_carry ? (k == 2 ? cy[2] : k == 1 ? cy[1] : cy[0]) : yu;
      zs[3 - d] = from_carry ? (k == 2 ? cz[2] : k == 1 ? cz[1] : cz[0]) : zu;
    }
    {
      const int ru = __shfl_up_sync(0xffffffffu, r, 1);
      r_prev = lane == 0 ? cr : ru;
    }
    if (valid) {
      const CodedCluster cc = code_track_values(j, r, X, Y, Z, q, r_prev, xs, ys, zs);
      const int len = cc.length();
      stage_code(T, i, cc, len, T.used[i] == 1u);
      l += (uint64_t)len;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {        // the next chunk's predecessors (full chunks only continue)
      cx[k] = shfl_idx64(X, 29 + k);
      cy[k] = shfl_idx64(Y, 29 + k);
      cz[k] = shfl_idx64(Z, 29 + k);
    }
    cr = __shfl_sync(0xffffffffu, r, 31);
  }
  return l;
}

// cluster j of a sorted block
__device__ CodedCluster code_block_cluster(const TmDev& T, const int32_t* ids, int j) {
  CodedCluster o;
  o.block = true;
  o.s1 = 0;
  const int32_t i = ids[j];
  const int64_t Y = qpos(T.y[i]);
  o.v0 = j == 0 ? zig(Y) : (uint64_t)(Y - qpos(T.y[ids[j - 1]]));
  o.s2 = qpos(T.z[i]);
  o.q = T.charge ? T.charge[i] : 0u;
  return o;
}

__device__ __forceinline__ bool ucl_less(int64_t y1, int64_t z1, int q1, int64_t y2, int64_t z2, int q2) {
  return y1 < y2 || (y1 == y2 && (z1 < z2 || (z1 == z2 && q1 < q2)));
}

// Warp-wide: the clusters (ids) of a block sorted by (Y, Z, charge) into
// `out`; every element's rank is counted against all others (ties: the
// earlier position), so any order of equal keys gives the same bytes.
__device__ void warp_sort_block(const TmDev& T, const int32_t* ids, int m, int32_t* out, int lane) {
  for (int a = lane; a - lane < m; a += 32) {
    const bool mine = a < m;
    const int32_t ia = mine ? ids[a] : 0;
    const int64_t ya = mine ? qpos(T.y[ia]) : 0, za = mine ? qpos(T.z[ia]) : 0;
    const int qa = mine && T.charge ? T.charge[ia] : 0;
    int rank = 0;
    for (int c0 = 0; c0 < m; c0 += 32) {
      const int cj = c0 + lane;
      const bool has = cj < m;
      const int32_t ic = has ? ids[cj] : 0;
      const int64_t yc = has ? qpos(T.y[ic]) : 0, zc = has ? qpos(T.z[ic]) : 0;
      const int qc = has && T.charge ? T.charge[ic] : 0;
      const int lim = min(32, m - c0);
      for (int t = 0; t < lim; ++t) {
        const int64_t yo = __shfl_sync(0xffffffffu, yc, t), zo = __shfl_sync(0xffffffffu, zc, t);
        const int qo = __shfl_sync(0xffffffffu, qc, t);
        const int jo = c0 + t;
        rank += (ucl_less(yo, zo, qo, ya, za, qa) || (yo == ya && zo == za && qo == qa && jo < a)) ? 1 : 0;
      }
    }
    if (mine) out[rank] = ia;
  }
}

// Byte length of work item w (tracks first, then blocks); blocks are sorted
// into blk_sorted here.  One warp per item.
__global__ void __launch_bounds__(kBlockT) k_tm_len(const __grid_constant__ TmDev T) {
  const int lane = threadIdx.x & 31;
  const int nt = track_count(T);
  const int nw = T.n_cap + T.n_inst * T.n_rows;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += warps) {
    uint64_t l = 0;
    if (w < T.n_cap) {
      if (w < nt) {
        const int32_t* c = T.tr_ids + T.tr_off[w];
        const int m = T.tr_ncl[w];
        l = track_length_warp(T, c, m, lane);
        if (lane == 0) l += (uint64_t)vlen((uint64_t)m);
      }
    } else {
      const int b = w - T.n_cap;
      const int m = T.blk_count[b];
      int32_t* sorted = T.blk_sorted + T.blk_base[b];
      warp_sort_block(T, T.blk_ids + T.blk_base[b], m, sorted, lane);
      __syncwarp();
      for (int j = lane; j < m; j += 32) {
        const CodedCluster cc = code_block_cluster(T, sorted, j);
        const int len = cc.length();
        stage_code(T, sorted[j], cc, len, true);
        l += (uint64_t)len;
      }
      if (lane == 0) l += (uint64_t)vlen((uint64_t)m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) T.len[w] = l;
  }
}

// Writes every item at its offset: the count, then each lane's cluster at
// the position a warp scan of the cluster lengths gives.
__global__ void __launch_bounds__(kBlockT) k_tm_write(const __grid_constant__ TmDev T) {
  const int lane = threadIdx.x & 31;
  const int nt = track_count(T);
  const int nb = T.n_inst * T.n_rows;
  const int nw = T.n_cap + nb;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += warps) {
    const int64_t at = (int64_t)T.off[w];
    bool track = w < T.n_cap;
    if (lane == 0) {
      if (track && w <= nt && T.out.track_offsets) T.out.track_offsets[w] = at;
      if (!track && T.out.row_offsets) T.out.row_offsets[w - T.n_cap] = at;
    }
    if (track && w >= nt) continue;
    if (at + (int64_t)T.len[w] > T.out.capacity) continue;
    int m;
    const int32_t* ids;
    if (track) {
      m = T.tr_ncl[w];
      ids = T.tr_ids + T.tr_off[w];
    } else {
      m = T.blk_count[w - T.n_cap];
      ids = T.blk_sorted + T.blk_base[w - T.n_cap];
    }
    int64_t pos = at + vlen((uint64_t)m);
    if (lane == 0) {
      int64_t p0 = at;
      put_u(T.out.data, p0, (uint64_t)m);
    }
    for (int j0 = 0; j0 < m; j0 += 32) {
      const int j = j0 + lane;
      CodedCluster cc;
      int len = 0;
      uint4 staged = make_uint4(0u, 0u, 0u, 0u);
      bool have = false;
      if (j < m) {
        const int32_t i = ids[j];
        len = T.clen[i];
        have = len > 0 && (!track || T.used[i] == 1u);
        if (have) {
          staged = T.code[i];
        } else {
          cc = track ? code_track_cluster(T, ids, j) : code_block_cluster(T, ids, j);
          len = cc.length();
        }
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (j < m) {
        if (have) {
          const uint64_t lo = (uint64_t)staged.x | ((uint64_t)staged.y << 32);
          const uint64_t hi = (uint64_t)staged.z | ((uint64_t)staged.w << 32);
          uint8_t* dst = T.out.data + pos + incl - len;
          for (int b = 0; b < len; ++b) dst[b] = (uint8_t)(b < 8 ? lo >> (8 * b) : hi >> (8 * (b - 8)));
        } else {
          cc.write(T.out.data, pos + incl - len);
        }
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *T.out.n_bytes = (int64_t)T.off[nw];
    if (nt == T.n_cap && T.out.track_offsets) T.out.track_offsets[nt] = (int64_t)T.off[T.n_cap];
    if (T.out.row_offsets) T.out.row_offsets[nb] = (int64_t)T.off[nw];
  }
}

__global__ void k_tm_mark(const __grid_constant__ TmDev T) {
  const int nt = track_count(T);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += gridDim.x * blockDim.x) {
    const int32_t* c = T.tr_ids + T.tr_off[k];
    for (int j = 0; j < T.tr_ncl[k]; ++j) atomicAdd(&T.used[c[j]], 1u);
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

// ---------------------------------------------------------------- decoding
struct TdDev {
  int n_rows;
  int32_t n_tracks, n_blocks;
  int64_t n_bytes;
  int64_t X[kMaxRows];
  float xf[kMaxRows];
  const uint8_t* data;
  const int64_t *track_off, *row_off;   // [n_tracks + 1], [n_blocks + 1]
  uint64_t *cnt, *base;          // [n_tracks + n_blocks + 1]
  tpct_tm_decoded out;
};

// The bytes of work item w (a track, then the (instance, row) blocks) and its
// cluster count.  An item whose offsets leave [0, n_bytes] or run backwards,
// whose count varint is unreadable, or whose count needs more bytes than the
// item holds (every track cluster takes at least 4 varints, every block
// cluster 3) is bad: count 0, status bit set.
__device__ Source td_item(const TdDev& D, int w, int64_t* m) {
  const bool trk = w < D.n_tracks;
  const int64_t a = trk ? D.track_off[w] : D.row_off[w - D.n_tracks];
  const int64_t b = trk ? D.track_off[w + 1] : D.row_off[w - D.n_tracks + 1];
  Source s{D.data, a, b, false};
  if (!(a >= 0 && a <= b && b <= D.n_bytes)) {
    s.bad = true;
    s.end = s.pos = 0;
  }
  const uint64_t c = s.bad ? 0u : s.u();
  if (!s.bad && c > (uint64_t)(s.end - s.pos) / (trk ? 4u : 3u)) s.bad = true;
  *m = s.bad ? 0 : (int64_t)c;
  return s;
}

__global__ void k_td_count(const __grid_constant__ TdDev D) {
  const int nw = D.n_tracks + D.n_blocks;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    int64_t m;
    const Source s = td_item(D, w, &m);
    D.cnt[w] = (uint64_t)m;
    if (s.bad) atomicOr(D.out.status, (uint32_t)TPCT_TD_BAD_STREAM);
  }
}

// (float)(V / 200.0): for |V| < 2^24 the float V is exact and one correctly
// rounded float division gives the same float (V / 200 is a dyadic rational
// or has a binary expansion of period 20, so no double-rounding case exists).
__device__ __forceinline__ float grid_to_cm(int64_t V) {
  if (V > -(1 << 24) && V < (1 << 24)) return __fdiv_rn((float)(int32_t)V, 200.f);
  return (float)((double)V / 200.0);
}

__device__ __forceinline__ void put_cluster(const TdDev& D, int64_t o, int r, int64_t Y, int64_t Z, uint64_t q) {
  if (o >= D.out.capacity) return;
  D.out.x[o] = D.xf[r];
  D.out.y[o] = grid_to_cm(Y);
  D.out.z[o] = grid_to_cm(Z);
  D.out.charge[o] = (uint16_t)q;
  D.out.row[o] = (uint8_t)r;
}

// Decodes every item again from its start.  A row outside the geometry, a
// charge above 65535 or an unreadable varint ends the item (status bit set;
// its remaining output slots are left unwritten).
__global__ void k_td_decode(const __grid_constant__ TdDev D) {
  const int nw = D.n_tracks + D.n_blocks;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    int64_t o = (int64_t)D.base[w];
    int64_t m;
    Source s = td_item(D, w, &m);
    if (w < D.n_tracks) {
      int64_t xs[3] = {0, 0, 0}, ys[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
      int r = 0;
      for (int64_t j = 0; j < m; ++j) {
        int64_t Y, Z;
        if (j == 0) {
          const uint64_t r0 = s.u();
          if (r0 >= (uint64_t)D.n_rows) s.bad = true;
          else r = (int)r0;
          Y = s.s();
          Z = s.s();
        } else {
          const uint64_t skip = s.u();
          if (skip >= (uint64_t)(D.n_rows - 1 - r)) {
            s.bad = true;
          } else {
            r = r + 1 + (int)skip;
          }
          const int kk = j < 3 ? (int)j : 3;
          const int64_t X = D.X[r];
          Y = s.s() + predict(xs, ys, kk, X);
          Z = s.s() + predict(xs, zs, kk, X);
        }
        const uint64_t q = s.u();
        if (q > 65535u) s.bad = true;
        if (s.bad) break;
        put_cluster(D, o++, r, Y, Z, q);
        xs[0] = xs[1]; xs[1] = xs[2]; xs[2] = D.X[r];
        ys[0] = ys[1]; ys[1] = ys[2]; ys[2] = Y;
        zs[0] = zs[1]; zs[1] = zs[2]; zs[2] = Z;
      }
    } else {
      const int b = w - D.n_tracks;
      const int r = b % D.n_rows;
      int64_t Y = 0;
      for (int64_t j = 0; j < m; ++j) {
        Y = j == 0 ? s.s() : Y + (int64_t)s.u();
        const int64_t Z = s.s();
        const uint64_t q = s.u();
        if (q > 65535u) s.bad = true;
        if (s.bad) break;
        put_cluster(D, o++, r, Y, Z, q);
      }
    }
    if (s.bad) atomicOr(D.out.status, (uint32_t)TPCT_TD_BAD_STREAM);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t n = (int64_t)D.base[nw];
    *D.out.n = n;
    if (n > D.out.capacity) atomicOr(D.out.status, (uint32_t)TPCT_TD_CAPACITY);
  }
}

int blocks_for_t(int64_t work) {
  int64_t b = (work + kBlockT - 1) / kBlockT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

size_t tm_carve(char* base, int64_t n, int32_t cap, int32_t n_blocks, TmDev* T) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* { char* p = base ? base + off : nullptr; off += (b + 255) / 256 * 256 + 256; return p; };
  const size_t nw = (size_t)cap + n_blocks + 1;
  uint32_t* used = (uint32_t*)take(4 * (size_t)std::max<int64_t>(n, 1));
  uint4* code = (uint4*)take(16 * (size_t)std::max<int64_t>(n, 1));
  uint8_t* clen = (uint8_t*)take((size_t)std::max<int64_t>(n, 1));
  int32_t* cnt = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* bas = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* cur = (int32_t*)take(4 * ((size_t)n_blocks + 1));
  int32_t* ids = (int32_t*)take(4 * (size_t)std::max<int64_t>(n, 1));
  int32_t* srt = (int32_t*)take(4 * (size_t)std::max<int64_t>(n, 1));
  uint64_t* len = (uint64_t*)take(8 * nw);
  uint64_t* off2 = (uint64_t*)take(8 * nw);
  uint64_t* tmp = (uint64_t*)take(8 * ((size_t)scan_tmp_elems((int64_t)nw) + 32));
  if (T) {
    T->used = used; T->code = code; T->clen = clen; T->blk_count = cnt; T->blk_base = bas; T->blk_cursor = cur; T->blk_ids = ids;
    T->blk_sorted = srt;
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
  cudaMemsetAsync(T.used, 0, 4 * (size_t)std::max<int64_t>(n, 1), s);
  cudaMemsetAsync(T.blk_count, 0, 4 * ((size_t)nb + 1), s);
  cudaMemsetAsync(T.blk_cursor, 0, 4 * ((size_t)nb + 1), s);
  k_tm_mark<<<blocks_for_t(cap), kBlockT, 0, s>>>(T); ++k;
  k_tm_count<<<blocks_for_t(n), kBlockT, 0, s>>>(T); ++k;
  launch_scan_i32(T.blk_count, T.blk_base, nb, tmp, s); k += 3;
  k_tm_fill<<<blocks_for_t(n), kBlockT, 0, s>>>(T); ++k;
  k_tm_len<<<blocks_for_t(((int64_t)cap + nb) * 32), kBlockT, 0, s>>>(T); ++k;
  launch_scan_u64(T.len, T.off, (int64_t)cap + nb, tmp, s); k += 3;
  k_tm_write<<<blocks_for_t(((int64_t)cap + nb) * 32), kBlockT, 0, s>>>(T); ++k;
  return k;
}

int enqueue_tm_decode(const double* row_x, int n_rows, const uint8_t* data, int64_t n_bytes, const int64_t* track_off,
                      int32_t n_tracks, const int64_t* row_off, int32_t n_blocks, void* ws, size_t ws_bytes,
                      const tpct_tm_decoded& out, cudaStream_t s) {
  if (tm_decode_workspace_bytes(n_tracks, n_blocks) > ws_bytes) return -2;
  TdDev D{};
  const size_t nw = (size_t)n_tracks + n_blocks + 1;
  char* p = (char*)ws;
  D.cnt = (uint64_t*)p;
  D.base = (uint64_t*)(p + (8 * nw + 255) / 256 * 256 + 256);
  uint64_t* tmp = (uint64_t*)(p + 2 * ((8 * nw + 255) / 256 * 256 + 256));
  tmp = (uint64_t*)(((uintptr_t)tmp + 255) / 256 * 256);
  D.n_rows = n_rows; D.n_tracks = n_tracks; D.n_blocks = n_blocks; D.n_bytes = n_bytes;
  for (int r = 0; r < n_rows; ++r) { D.X[r] = (int64_t)std::llrint(row_x[r] * 200.0); D.xf[r] = (float)row_x[r]; }
  D.data = data; D.track_off = track_off; D.row_off = row_off; D.out = out;
  int k = 0;
  cudaMemsetAsync(out.status, 0, sizeof(uint32_t), s);
  k_td_count<<<blocks_for_t((int64_t)n_tracks + n_blocks), kBlockT, 0, s>>>(D); ++k;
  launch_scan_u64(D.cnt, D.base, (int64_t)n_tracks + n_blocks, tmp, s); k += 3;
  k_td_decode<<<blocks_for_t((int64_t)n_tracks + n_blocks), kBlockT, 0, s>>>(D); ++k;
  return k;
}

}  // namespace tpct
