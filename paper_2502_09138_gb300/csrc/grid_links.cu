// Steps 1-4 of sector track finding: row binning into y/z grids, neighbour
// finding by the straight-line criterion, reciprocal cleaning, start hits.
// (The paper's "TPC Processing (Tracking)" row, Tables 1-3.)
#include <mutex>

#include "tpct_internal.cuh"

namespace tpct {

namespace {

constexpr int kBlock = 256;
constexpr int kGridThreads = 512;
constexpr int kNbDown = 8;                     // down candidates of a hit listed in shared memory
constexpr int kGridSmemWords = 24576;          // 96 KB of bin counters per CTA (two CTAs per SM)


// ------------------------------------------------------------------ step 1: rows and grids
__global__ void k_init_rows(const __grid_constant__ Params P) {
  int nr = P.n_inst * P.n_rows;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nr; i += gridDim.x * blockDim.x) {
    P.row_count[i] = 0;
    P.row_tl_count[i] = 0;
  }
}

// row whose x is nearest to xc (ties to the lower row)
__device__ __forceinline__ int nearest_row(const Params& P, float xc) {
  double x = (double)xc;
  int lo = 0, hi = P.n_rows - 1;
  while (lo < hi) {            // first row with rx >= x (or the last row)
    int mid = (lo + hi) >> 1;
    if (P.rx[mid] < x) lo = mid + 1; else hi = mid;
  }
  if (lo > 0 && fabs(x - P.rx[lo - 1]) <= fabs(x - P.rx[lo])) lo = lo - 1;
  return lo;
}

// The whole of step 1 for one instance per CTA (rows, extents, grid
// dimensions, bin counts, bin starts, the sorted copy): an instance's
// clusters fill the sorted positions [inst_off[i], inst_off[i+1]) and its
// bins the entries [ib(i), ib(i+1)) of bin_start, ib(i) = inst_off[i] / k +
// 2 n_rows i, so no step needs a device-wide scan and the counters live in
// shared memory: two 16-bit counters per 32-bit word when the instance's
// clusters fit 16-bit offsets (49,152 bins), else one 32-bit counter per word
// (24,576 bins), else global memory.
// row_start and bin_start hold what device-wide exclusive scans of the row
// and bin counts would give; the bin grid of a row holds about k clusters
// per bin with bins roughly square in cm, and its bin_start entries start at
// row_start / k + 2 ir, which leaves room for max(1, n / k) bins plus the
// end entry.
__global__ void __launch_bounds__(kGridThreads) k_grid_build(const __grid_constant__ Params P) {
  extern __shared__ int g_bins[];               // [kGridSmemWords]
  __shared__ int r_cnt[kMaxRows], r_start[kMaxRows + 1];
  __shared__ uint32_t r_ext[4][kMaxRows];
  __shared__ RowGrid r_grid[kMaxRows];
  __shared__ int s_wsum[kGridThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_inst;
  const int k = P.clusters_per_bin;
  // instances from a work counter (their sizes differ by two orders of magnitude)
  if (tid == 0) s_inst = (int)atomicAdd(&P.work[0], 1u);
  __syncthreads();
  for (int inst = s_inst; inst < P.n_inst; inst = s_inst) {
    const int c0 = (int)P.inst_off[inst], c1 = (int)P.inst_off[inst + 1];
    for (int r = tid; r < P.n_rows; r += kGridThreads) {
      r_cnt[r] = 0;
      r_ext[0][r] = 0xffffffffu; r_ext[1][r] = 0u; r_ext[2][r] = 0xffffffffu; r_ext[3][r] = 0u;
    }
    __syncthreads();
    // pass A: rows, counts, extents
    for (int c = c0 + tid; c < c1; c += kGridThreads) {
      int r = P.row ? (int)P.row[c] : nearest_row(P, P.x[c]);
      if (r >= P.n_rows) {
        atomicOr(P.status, kDevBadRow);
        r = P.n_rows - 1;
      }
      P.c_ir[c] = inst * P.n_rows + r;
      atomicAdd(&r_cnt[r], 1);
      const uint32_t ky = float_order_key(P.y[c]), kz = float_order_key(P.z[c]);
      atomicMin(&r_ext[0][r], ky); atomicMax(&r_ext[1][r], ky);
      atomicMin(&r_ext[2][r], kz); atomicMax(&r_ext[3][r], kz);
    }
    __syncthreads();
    if (warp == 0) {   // exclusive scan of the row counts
      int run = 0;
      for (int r0 = 0; r0 < P.n_rows; r0 += 32) {
        const int r = r0 + lane;
        const int v = r < P.n_rows ? r_cnt[r] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int x = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += x;
        }
        if (r < P.n_rows) r_start[r] = run + incl - v;
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) r_start[P.n_rows] = run;
    }
    __syncthreads();
    // grid dimensions of every row (the same arithmetic as k_grid_dims)
    for (int r = tid; r < P.n_rows; r += kGridThreads) {
      const int ir = inst * P.n_rows + r;
      const int n = r_cnt[r];
      const int start = c0 + r_start[r];
      const int nb = max(1, n / k);
      float ymin = 0.f, ymax = 0.f, zmin = 0.f, zmax = 0.f;
      if (n > 0) {
        ymin = float_from_order_key(r_ext[0][r]);
        ymax = float_from_order_key(r_ext[1][r]);
        zmin = float_from_order_key(r_ext[2][r]);
        zmax = float_from_order_key(r_ext[3][r]);
      }
      const float ly = fmaxf(ymax - ymin, 1e-3f), lz = fmaxf(zmax - zmin, 1e-3f);
      int ny = (int)rintf(sqrtf((float)nb * ly / lz));
      ny = min(max(ny, 1), min(nb, 32767));
      const int nz = min(max(nb / ny, 1), 32767);
      RowGrid g;
      g.y0 = ymin;
      g.z0 = zmin;
      g.idy = (float)ny / ly;
      g.idz = (float)nz / lz;
      g.bin_base = start / k + 2 * ir;
      g.ny = (int16_t)ny;
      g.nz = (int16_t)nz;
      r_grid[r] = g;
      P.grid[ir] = g;
      P.row_count[ir] = n;
      P.row_start[ir] = start;
    }
    if (tid == 0) {
      P.row_start[(inst + 1) * P.n_rows] = c1;   // also the next instance's first row (same value)
      if (inst == P.n_inst - 1) P.row_count[P.n_inst * P.n_rows] = 0;
    }
    // this instance's bin entries [ib0, ib1]
    const int ib0 = c0 / k + 2 * inst * P.n_rows, ib1 = c1 / k + 2 * (inst + 1) * P.n_rows;
    const int span = ib1 - ib0;
    // counters: packed halves of shared words (every running offset of the
    // instance, its final value included, stays below 2^16, so a half never
    // carries into its neighbour), whole shared words, or global memory
    const bool packed = c1 - c0 < 65536 && span <= 2 * kGridSmemWords;
    int* cnt = packed || span <= kGridSmemWords ? g_bins : P.bin_count + ib0;
    unsigned* wcnt = reinterpret_cast<unsigned*>(g_bins);
    const int n_words = packed ? (span + 1) >> 1 : span;
    for (int b = tid; b < n_words; b += kGridThreads) cnt[b] = 0;
    __syncthreads();
    auto bump = [&](int b) -> int {   // add one to counter b, return its old value
      if (packed) {
        const int sh = (b & 1) << 4;
        return (int)((atomicAdd(&wcnt[b >> 1], 1u << sh) >> sh) & 0xffffu);
      }
      return atomicAdd(&cnt[b], 1);
    };
    auto get = [&](int b) -> int { return packed ? (int)((wcnt[b >> 1] >> ((b & 1) << 4)) & 0xffffu) : cnt[b]; };
    // pass B: bin counts
    for (int c = c0 + tid; c < c1; c += kGridThreads) {
      const RowGrid g = r_grid[P.c_ir[c] - inst * P.n_rows];
      const int b = g.bin_base - ib0 + bin_z(g, P.z[c]) * g.ny + bin_y(g, P.y[c]);
      bump(b);
    }
    __syncthreads();
    // exclusive scan of the counts in place (a contiguous chunk per thread;
    // chunks of whole words when packed, so no two threads write one word)
    const int per = ((span + kGridThreads - 1) / kGridThreads + 1) & ~1;
    const int b_lo = min(tid * per, span), b_hi = min(b_lo + per, span);
    int sum = 0;
    for (int b = b_lo; b < b_hi; ++b) sum += get(b);
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int run = incl - sum;
    for (int q = 0; q < warp; ++q) run += s_wsum[q];
    for (int b = b_lo; b < b_hi; ++b) {
      const int v = get(b);
      if (packed) {
        const int sh = (b & 1) << 4;
        wcnt[b >> 1] = (wcnt[b >> 1] & ~(0xffffu << sh)) | ((unsigned)run << sh);
      } else {
        cnt[b] = run;
      }
      P.bin_start[ib0 + b] = c0 + run;
      run += v;
    }
    if (tid == 0) P.bin_start[ib1] = c1;   // also the next instance's first entry (same value)
    __syncthreads();
    // pass C: the sorted copy (the order inside a bin is that of the atomics)
    for (int c = c0 + tid; c < c1; c += kGridThreads) {
      const int r = P.c_ir[c] - inst * P.n_rows;
      const RowGrid g = r_grid[r];
      const int b = g.bin_base - ib0 + bin_z(g, P.z[c]) * g.ny + bin_y(g, P.y[c]);
      const int pos = c0 + bump(b);
      P.sy[pos] = P.y[c];
      P.sz[pos] = P.z[c];
      P.sid[pos] = c;
      P.srow[pos] = (uint8_t)r;
      P.W[pos] = 0u;
    }
    if (tid == 0) s_inst = (int)atomicAdd(&P.work[0], 1u);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ scans
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// exclusive block scan of one value per thread; *total receives the block sum
template <class T>
__device__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_sums[32];
  __shared__ T block_total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    const T s = lane < nw ? warp_sums[lane] : (T)0;
    const T si = warp_incl_scan(s);
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == 31) block_total = si;
  }
  __syncthreads();
  const T res = inc - v + warp_sums[w];
  if (total) *total = block_total;
  __syncthreads();
  return res;
}

template <class Tin, class T>
__global__ void k_scan_reduce(const Tin* in, int64_t m, T* tmp) {
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < m) s += (T)in[i];
  }
  T total;
  block_excl_scan<T>(s, &total);
  if (threadIdx.x == 0) tmp[blockIdx.x] = total;
}

template <class T>
__global__ void k_scan_top(T* tmp, int64_t nb) {
  T carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    T v = i < nb ? tmp[i] : (T)0;
    T total;
    T e = block_excl_scan<T>(v, &total);
    if (i < nb) tmp[i] = e + carry;
    carry += total;
    __syncthreads();
  }
}

template <class Tin, class Tout, class T>
__global__ void k_scan_down(const Tin* in, Tout* out, int64_t m, const T* tmp) {
  int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < m ? (T)in[i] : (T)0;
    s += v[k];
  }
  T total;
  T e = block_excl_scan<T>(s, &total) + tmp[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < m) out[i] = (Tout)e;
    if (i == m - 1) out[m] = (Tout)(e + v[k]);
    e += v[k];
  }
}

__global__ void k_zero_total_i32(int32_t* out) { out[0] = 0; }
__global__ void k_zero_total_u64(uint64_t* out) { out[0] = 0; }

// ------------------------------------------------------------------ step 2: neighbours
// Straight-line criterion: for hit h in row r and candidates u (row r+1),
// d (row r-1) inside |dy| <= wy dx, |dz| <= wz dx, the pair minimising
// D = (yhat - y_h)^2 + (zhat - z_h)^2, yhat = y_d + f (y_u - y_d),
// f = (x_r - x_d) / (x_u - x_d), ties to the smaller (id_u, id_d); the pair
// is kept iff D <= D_max.  Evaluated relative to the hit (differences
// first) so that the FP32 variant keeps ~1e-7 relative accuracy in D.
template <class E>
struct NfRowSide {
  RowGrid g;
  E w_y, w_z;
  int32_t bin0;   // absolute index of the row's first bin
};

template <class E>
__device__ __forceinline__ void bin_range(const RowGrid& g, float c, float w, int& i0, int& i1, bool is_y) {
  float lo = c - w * 1.00001f - 1e-5f, hi = c + w * 1.00001f + 1e-5f;
  if (is_y) { i0 = bin_y(g, lo); i1 = bin_y(g, hi); }
  else { i0 = bin_z(g, lo); i1 = bin_z(g, hi); }
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) k_neighbours(const __grid_constant__ Params P) {
  using E = typename Prec<MODE>::E;
  __shared__ float dn_y[kNbDown][kBlock], dn_z[kNbDown][kBlock];
  __shared__ int dn_i[kNbDown][kBlock];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int nr = P.n_inst * P.n_rows;
  for (int ir = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ir < nr; ir += warps) {
    const int r = ir % P.n_rows;
    const int beg = P.row_start[ir], end = P.row_start[ir + 1];
    if (r == 0 || r == P.n_rows - 1) {
      for (int p = beg + lane; p < end; p += 32) { P.up[p] = -1; P.down[p] = -1; }
      continue;
    }
    E f, wyu, wzu, wyd, wzd;
    if constexpr (std::is_same<E, float>::value) {
      // the row's constants from the table (formed in double once per step)
      f = P.nf_tab[5 * r]; wyu = P.nf_tab[5 * r + 1]; wzu = P.nf_tab[5 * r + 2];
      wyd = P.nf_tab[5 * r + 3]; wzd = P.nf_tab[5 * r + 4];
    } else {
      const double xr = P.rx[r], xu = P.rx[r + 1], xd = P.rx[r - 1];
      f = (E)((xr - xd) / (xu - xd));
      wyu = (E)(P.nf_wy * (xu - xr)); wzu = (E)(P.nf_wz * (xu - xr));
      wyd = (E)(P.nf_wy * (xr - xd)); wzd = (E)(P.nf_wz * (xr - xd));
    }
    const E dmax = (E)P.nf_dmax;
    const RowGrid gu = P.grid[ir + 1], gd = P.grid[ir - 1];
    for (int p = beg + lane; p < end; p += 32) {
      const float yh = P.sy[p], zh = P.sz[p];
      int uy0, uy1, uz0, uz1, dy0, dy1, dz0, dz1;
      bin_range<E>(gu, yh, (float)wyu, uy0, uy1, true);
      bin_range<E>(gu, zh, (float)wzu, uz0, uz1, false);
      bin_range<E>(gd, yh, (float)wyd, dy0, dy1, true);
      bin_range<E>(gd, zh, (float)wzd, dz0, dz1, false);
      E best = (E)0;
      int bu = -1, bd = -1, idu = -1, idd = -1;
      // the pair (u, d) minimising D, ties to the smaller (id_u, id_d): the
      // minimum of a strict total order, so the visiting order is free
      auto consider = [&](E ayu, E azu, int q, E ayd, E azd, int s) {
        const E ry = ayd + f * (ayu - ayd);
        const E rz = azd + f * (azu - azd);
        const E D = ry * ry + rz * rz;
        bool better;
        if (bu < 0 || D < best) {
          better = true;
        } else if (D == best) {
          if (idu < 0) { idu = P.sid[bu]; idd = P.sid[bd]; }
          const int iu = P.sid[q], id = P.sid[s];
          better = iu < idu || (iu == idu && id < idd);
        } else {
          better = false;
        }
        if (better) { best = D; bu = q; bd = s; idu = -1; idd = -1; }
      };
      // the down candidates inside the window, gathered once per hit (up to
      // kNbDown of them; more take the nested loop)
      int nd = 0;
      for (int jz = dz0; jz <= dz1 && nd <= kNbDown; ++jz) {
        const int s0 = P.bin_start[gd.bin_base + jz * gd.ny + dy0];
        const int s1 = P.bin_start[gd.bin_base + jz * gd.ny + dy1 + 1];
        for (int s = s0; s < s1; ++s) {
          const E ayd = (E)P.sy[s] - (E)yh, azd = (E)P.sz[s] - (E)zh;
          if (!(fabs(ayd) <= wyd && fabs(azd) <= wzd)) continue;
          if (nd < kNbDown) {
            dn_y[nd][threadIdx.x] = (float)ayd;
            dn_z[nd][threadIdx.x] = (float)azd;
            dn_i[nd][threadIdx.x] = s;
          }
          if (++nd > kNbDown) break;
        }
      }
      const bool listed = nd <= kNbDown;
      if (nd > 0) {
        for (int iz = uz0; iz <= uz1; ++iz) {
          const int q0 = P.bin_start[gu.bin_base + iz * gu.ny + uy0];
          const int q1 = P.bin_start[gu.bin_base + iz * gu.ny + uy1 + 1];
          for (int q = q0; q < q1; ++q) {
            const E ayu = (E)P.sy[q] - (E)yh, azu = (E)P.sz[q] - (E)zh;
            if (!(fabs(ayu) <= wyu && fabs(azu) <= wzu)) continue;
            if (listed) {
              for (int i = 0; i < nd; ++i)
                consider(ayu, azu, q, (E)dn_y[i][threadIdx.x], (E)dn_z[i][threadIdx.x], dn_i[i][threadIdx.x]);
            } else {
              for (int jz = dz0; jz <= dz1; ++jz) {
                const int s0 = P.bin_start[gd.bin_base + jz * gd.ny + dy0];
                const int s1 = P.bin_start[gd.bin_base + jz * gd.ny + dy1 + 1];
                for (int s = s0; s < s1; ++s) {
                  const E ayd = (E)P.sy[s] - (E)yh, azd = (E)P.sz[s] - (E)zh;
                  if (!(fabs(ayd) <= wyd && fabs(azd) <= wzd)) continue;
                  consider(ayu, azu, q, ayd, azd, s);
                }
              }
            }
          }
        }
      }
      const bool ok = bu >= 0 && best <= dmax;
      P.up[p] = ok ? bu : -1;
      P.down[p] = ok ? bd : -1;
    }
  }
}

// ------------------------------------------------------------------ steps 3-4
// upc[p] = up[p] if down[up[p]] == p; start iff no reciprocal down link and
// a reciprocal chain p -> u -> uu.  Per row: count of start hits.
__global__ void k_clean_start(const __grid_constant__ Params P) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int nr = P.n_inst * P.n_rows;
  for (int ir = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ir < nr; ir += warps) {
    const int beg = P.row_start[ir], end = P.row_start[ir + 1];
    int count = 0;
    for (int base = beg; base < end; base += 32) {
      const int p = base + lane;
      bool start = false;
      if (p < end) {
        const int u = P.up[p], d = P.down[p];
        const int uc = (u >= 0 && P.down[u] == p) ? u : -1;
        const bool dc = d >= 0 && P.up[d] == p;
        bool chain = false;
        if (uc >= 0) {
          const int uu = P.up[uc];
          chain = uu >= 0 && P.down[uu] == uc;
        }
        start = !dc && chain;
        P.upc[p] = uc;
        P.sflag[p] = start ? 1 : 0;
      }
      count += __popc(__ballot_sync(0xffffffffu, start));
    }
    if (lane == 0) P.row_tl_count[ir] = count;
  }
}

// Tracklet index of a start hit: row base + number of start hits of the same
// row with a smaller input id (start-hit order is (instance, row, id)).
__global__ void k_start_fill(const __grid_constant__ Params P) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int nr = P.n_inst * P.n_rows;
  for (int ir = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ir < nr; ir += warps) {
    if (P.row_tl_count[ir] == 0) continue;
    const int beg = P.row_start[ir], end = P.row_start[ir + 1];
    const int tbase = P.row_tl_base[ir];
    for (int base = beg; base < end; base += 32) {
      const int p = base + lane;
      const bool mine = p < end && P.sflag[p];
      const int my_id = mine ? P.sid[p] : 0;
      if (__ballot_sync(0xffffffffu, mine) == 0u) continue;
      int rank = 0;
      for (int b2 = beg; b2 < end; b2 += 32) {
        const int q = b2 + lane;
        const bool st = q < end && P.sflag[q];
        const int qid = st ? P.sid[q] : 0x7fffffff;
        uint32_t m = __ballot_sync(0xffffffffu, st);
        while (m) {
          const int k = __ffs(m) - 1;
          m &= m - 1;
          const int other = __shfl_sync(0xffffffffu, qid, k);
          rank += (mine && other < my_id) ? 1 : 0;
        }
      }
      if (mine) {
        const int t = tbase + rank;
        if (t < P.tcap) {
          P.tl_start[t] = p;
          P.tl_ir[t] = ir;
        } else {
          atomicOr(P.status, kDevTrackletCap);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ debug export of links
__global__ void k_export_links(const __grid_constant__ Params P, tpct_debug_out D) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += gridDim.x * blockDim.x) {
    const int id = P.sid[p];
    const int u = P.up[p], d = P.down[p];
    if (D.up) D.up[id] = u >= 0 ? P.sid[u] : -1;
    if (D.down) D.down[id] = d >= 0 ? P.sid[d] : -1;
    if (D.upc) { const int uc = P.upc[p]; D.upc[id] = uc >= 0 ? P.sid[uc] : -1; }
    if (D.downc) D.downc[id] = (d >= 0 && P.up[d] == p) ? P.sid[d] : -1;
    if (D.weight) D.weight[id] = P.W[p];
  }
}

int blocks_for(int64_t work, int block) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

}  // namespace

int64_t scan_tmp_elems(int64_t m) { return (m + kScanChunk - 1) / kScanChunk + 1; }

void launch_init_rows(const Params& P, cudaStream_t s) {
  k_init_rows<<<blocks_for(P.n_inst * P.n_rows + 1, kBlock), kBlock, 0, s>>>(P);
}

void launch_grid_build(const Params& P, cudaStream_t s) {
  static std::once_flag attr;   // the serving runtime enqueues from several threads
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_grid_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kGridSmemWords);
  });
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(P.n_inst, n_sm * 2));
  k_grid_build<<<grid, kGridThreads, 4 * kGridSmemWords, s>>>(P);
}

template <class Tin, class T>
static void scan_impl(const Tin* in, Tin* out, int64_t m, T* tmp, cudaStream_t s) {
  if (m <= 0) {
    if constexpr (sizeof(Tin) == 4) k_zero_total_i32<<<1, 1, 0, s>>>((int32_t*)out);
    else k_zero_total_u64<<<1, 1, 0, s>>>((uint64_t*)out);
    return;
  }
  int64_t nb = (m + kScanChunk - 1) / kScanChunk;
  k_scan_reduce<Tin, T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, m, tmp);
  k_scan_top<T><<<1, kScanThreads, 0, s>>>(tmp, nb);
  k_scan_down<Tin, Tin, T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, m, tmp);
}

void launch_scan_i32(const int32_t* in, int32_t* out, int64_t m, uint64_t* tmp, cudaStream_t s) {
  scan_impl<int32_t, uint64_t>(in, out, m, tmp, s);
}
void launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t m, uint64_t* tmp, cudaStream_t s) {
  scan_impl<uint64_t, uint64_t>(in, out, m, tmp, s);
}

void launch_neighbours(const Params& P, int mode, cudaStream_t s) {
  const int warps = P.n_inst * P.n_rows;
  const int blocks = blocks_for((int64_t)warps * 32, kBlock);
  // the neighbour arithmetic is float in every mode but FP64
  if (mode == 0) k_neighbours<0><<<blocks, kBlock, 0, s>>>(P);
  else if (mode == 2) k_neighbours<2><<<blocks, kBlock, 0, s>>>(P);
  else k_neighbours<1><<<blocks, kBlock, 0, s>>>(P);
}

void launch_clean_start(const Params& P, cudaStream_t s) {
  k_clean_start<<<blocks_for((int64_t)P.n_inst * P.n_rows * 32, kBlock), kBlock, 0, s>>>(P);
}

void launch_start_fill(const Params& P, cudaStream_t s) {
  k_start_fill<<<blocks_for((int64_t)P.n_inst * P.n_rows * 32, kBlock), kBlock, 0, s>>>(P);
}

void launch_export_links(const Params& P, const tpct_debug_out& d, cudaStream_t s) {
  k_export_links<<<blocks_for(P.n, kBlock), kBlock, 0, s>>>(P, d);
}

}  // namespace tpct
