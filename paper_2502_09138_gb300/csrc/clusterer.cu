// TPC cluster finding: zero-suppressed digits (pad, time bin, ADC) of each
// pad row -> clusters (charge-weighted centroid and width, total and peak
// charge, local position).  The paper names clustering as part of "TPC
// Processing (Tracking, Clustering, Compression)" (Table 1); the steps are
// the stated readings:
//   peak      q >= q_peak_min, q > every 3x3 neighbour that comes before it in
//             (time, pad) order and q >= every later one;
//   valley    a peak is dropped if a higher peak (ties: the earlier one) lies
//             at Chebyshev distance 2 and the cell between them holds at least
//             q - valley_delta;
//   cluster   the 3x3 cells around a kept peak plus each outer-ring cell whose
//             inner neighbour towards the peak holds at least its charge.
// Clusters come in (instance, row) order, inside a row in (time, pad) order
// of their peaks.
//
// GB300 mapping, three kernels and a scan:
//   k_cf_sort    one CTA per pad row: a counting sort of the row's digits by
//                time bin (shared-memory histogram and scan) into packed
//                32-bit words, and the row's time-bin starts;
//   k_clusterer  persistent, 256-thread CTAs, four per SM; a work item is one
//                pad row and one tile of kTileT time bins, whose digits (plus
//                three bins on each side) are now one contiguous range.  The
//                CTA scatters them into a shared-memory charge map with a zero
//                border (no bounds tests), tests peaks and valleys there, ranks
//                the kept peaks in (time, pad) order by one scan over a kept-peak
//                bitmap and writes the clusters to a staging area at slots taken
//                with one atomic per item: CTAs never wait for one another;
//   scan, k_cf_emit  the items' counts give every item its place in the
//                output; a warp per item moves its staged clusters there and
//                derives x, y, z and the flags.
#include "tpct_internal.cuh"

namespace tpct {
namespace {

constexpr int kCfThreads = 256;
constexpr int kCfWarps = kCfThreads / 32;
constexpr int kTileT = 128;                // time bins per work item
constexpr int kHalo = 3;                   // map rows kept on each side of a tile
constexpr int kMapRows = kTileT + 2 * kHalo;
constexpr int kWordsPer = kTileT * 256 / 32 / kCfThreads;   // kept-bitmap words per thread (pads <= 252)
constexpr int kCfMaxPeaks = 2048;          // kept peaks of a tile
constexpr int kCfPerSm = 4;                // resident CTAs per SM
constexpr int kMaxTime = 512;              // time bins per row at most
constexpr int kSortThreads = 256;
constexpr int kSortU = 4;                  // digits per thread in flight in the sort passes
constexpr int kScanPer = (kMaxTime + 1 + kSortThreads - 1) / kSortThreads;
constexpr int kEmitThreads = 256;

// A staged cluster: moments and charges, peak cell packed as p | t << 8 | q << 17.
struct __align__(8) CfStage {
  float cp, ct, sp, st;
  uint32_t qtot, ptq;
};

struct CfDev {
  const uint16_t *pad, *time, *adc;
  const int64_t* row_offsets;
  const int32_t* inst_sector;
  int32_t n_inst, n_rows, n_time, n_tiles;
  int32_t wp;                               // map row width: pads + 4, a multiple of 32
  int32_t q_peak_min, valley_delta;
  float z_max, time_bin;
  uint32_t* work;                           // [2] item counter, staging counter
  uint32_t* srt;                            // [srt_cap] packed digits, sorted by time inside each row
  int64_t srt_cap;
  int32_t* tpos;                            // [rows][kMaxTime + 1] time-bin starts in the sorted row
  int32_t *item_cnt, *item_at, *item_dst;   // [n_items] clusters, staging slot, output slot (+1: total)
  CfStage* stage;                           // [out.capacity]
  int16_t n_pad[kMaxRows];
  float pitch[kMaxRows], row_x[kMaxRows];
  tpct_cf_out out;
};

// The tile map: cell (p, t) of the row, t in [t0 - 3, t0 + kTileT + 3), lives
// at (t - t0 + 3) * wp + (p + 2).  Pads -2, -1 and >= n_pad and time bins
// outside the row hold 0, so every neighbourhood read up to distance 2 of a
// cell in [t0 - 1, t0 + kTileT + 1) stays inside the map without a bounds test.
__device__ __forceinline__ bool before(int dp, int dt) { return dt < 0 || (dt == 0 && dp < 0); }
__device__ __forceinline__ int half_step(int d) { return d == 2 ? 1 : (d == -2 ? -1 : 0); }
__device__ __forceinline__ bool bit_at(const uint32_t* bits, int cell) { return (bits[cell >> 5] >> (cell & 31)) & 1u; }

__device__ __forceinline__ bool peak_test(const uint16_t* map, int W, int c, int qmin) {
  const int q = map[c];
  if (q < qmin) return false;
  bool ok = true;
#pragma unroll
  for (int dt = -1; dt <= 1; ++dt)
#pragma unroll
    for (int dp = -1; dp <= 1; ++dp) {
      if (dp == 0 && dt == 0) continue;
      const int qn = map[c + dt * W + dp];
      ok &= before(dp, dt) ? q > qn : q >= qn;
    }
  return ok;
}

__device__ __forceinline__ bool suppressed(const uint16_t* map, const uint32_t* bits, int W, int c, int delta) {
  const int q = map[c];
  bool sup = false;
#pragma unroll
  for (int dt = -2; dt <= 2; ++dt)
#pragma unroll
    for (int dp = -2; dp <= 2; ++dp) {
      if (dp > -2 && dp < 2 && dt > -2 && dt < 2) continue;   // the Chebyshev-2 ring only
      const int c2 = c + dt * W + dp;
      if (!bit_at(bits, c2)) continue;
      const int q2 = map[c2];
      if (!(q2 > q || (q2 == q && before(dp, dt)))) continue;
      sup |= (int)map[c + half_step(dt) * W + half_step(dp)] >= q - delta;
    }
  return sup;
}

struct Cluster {
  float cp, ct, sp, st;
  uint32_t qtot;
  int p, t, q;
};

__device__ __forceinline__ Cluster build_cluster(const uint16_t* map, int W, int c, int t0) {
  const int p = c % W - 2, tl = c / W;
  int s0 = 0, sp = 0, st = 0, spp = 0, stt = 0;
#pragma unroll
  for (int dt = -2; dt <= 2; ++dt)
#pragma unroll
    for (int dp = -2; dp <= 2; ++dp) {
      const int qc = map[c + dt * W + dp];
      const bool outer = dp == 2 || dp == -2 || dt == 2 || dt == -2;
      const bool take = qc > 0 && (!outer || qc <= (int)map[c + half_step(dt) * W + half_step(dp)]);
      const int q = take ? qc : 0;
      s0 += q; sp += q * dp; st += q * dt; spp += q * dp * dp; stt += q * dt * dt;
    }
  const float fs0 = (float)s0;
  const float mp = __fdiv_rn((float)sp, fs0), mt = __fdiv_rn((float)st, fs0);
  Cluster k;
  k.p = p;
  k.t = t0 + tl - kHalo;
  k.q = map[c];
  k.cp = (float)p + mp;
  k.ct = (float)k.t + mt;
  k.sp = sqrtf(fmaxf(__fdiv_rn((float)spp, fs0) - mp * mp, 0.f));
  k.st = sqrtf(fmaxf(__fdiv_rn((float)stt, fs0) - mt * mt, 0.f));
  k.qtot = (uint32_t)s0;
  return k;
}

__device__ __forceinline__ void store_cluster(const tpct_cf_out& O, long long slot, const Cluster& k, float row_x,
                                              float pitch, int np, int nt, float side, float z_max, float time_bin,
                                              int r) {
  O.pad[slot] = k.cp;
  O.time[slot] = k.ct;
  O.sigma_pad[slot] = k.sp;
  O.sigma_time[slot] = k.st;
  O.x[slot] = row_x;
  O.y[slot] = (k.cp + 0.5f - 0.5f * (float)np) * pitch;
  O.z[slot] = side * (z_max - (k.ct + 0.5f) * time_bin);
  O.q_tot[slot] = k.qtot;
  O.q_max[slot] = (uint16_t)k.q;
  O.row[slot] = (uint8_t)r;
  O.flags[slot] = (uint8_t)((k.p == 0 || k.p == np - 1 ? 1 : 0) | (k.t == 0 || k.t == nt - 1 ? 2 : 0));
}

// Pass 1, one CTA per pad row: counting sort of the row's digits by time bin
// into packed words (pad | time << 8 | ADC << 17), plus the row's time-bin
// starts (tpos[t] = first sorted digit with time >= t, row-relative).  The
// order inside a time bin is that of the atomics; nothing downstream depends
// on it (cells are unique and the peaks are ranked from a bitmap).
__global__ void __launch_bounds__(kSortThreads) k_cf_sort(const __grid_constant__ CfDev P) {
  __shared__ int hist[kMaxTime + 1];
  __shared__ int s_wsum[kSortThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = P.n_time;
  const int n_rows_total = P.n_inst * P.n_rows;
  const tpct_cf_out& O = P.out;
  for (int row = blockIdx.x; row < n_rows_total; row += gridDim.x) {
    const int64_t b = P.row_offsets[row];
    int64_t e = P.row_offsets[row + 1];
    if (e > P.srt_cap) {   // beyond the workspace: the row is left empty
      if (tid == 0) atomicOr(O.status, TPCT_CF_WORKSPACE);
      e = b;
    }
    const int np = P.n_pad[row % P.n_rows];
    for (int t = tid; t <= kMaxTime; t += kSortThreads) hist[t] = 0;
    __syncthreads();
    // both passes load kSortU digits per thread before using any
    for (int64_t base = b; base < e; base += kSortThreads * kSortU) {
      uint32_t pv[kSortU], tv[kSortU], qv[kSortU];
#pragma unroll
      for (int u = 0; u < kSortU; ++u) {
        const int64_t i = base + u * kSortThreads + tid;
        pv[u] = i < e ? P.pad[i] : 0u;
        tv[u] = i < e ? P.time[i] : 0u;
        qv[u] = i < e ? P.adc[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kSortU; ++u) {
        if (base + u * kSortThreads + tid >= e) break;
        if ((int)pv[u] < np && (int)tv[u] < nt && qv[u] < 32768u) atomicAdd(&hist[tv[u]], 1);
        else atomicOr(O.status, TPCT_CF_BAD_DIGIT);
      }
    }
    __syncthreads();
    // exclusive scan of hist[0, kMaxTime]: kScanPer bins per thread
    int v[kScanPer], sum = 0;
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
      const int t = tid * kScanPer + u;
      v[u] = t <= kMaxTime ? hist[t] : 0;
      sum += v[u];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int run = incl - sum;
#pragma unroll
    for (int q = 0; q < kSortThreads / 32; ++q) run += q < warp ? s_wsum[q] : 0;
    int32_t* tp = P.tpos + (int64_t)row * (kMaxTime + 1);
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
      const int t = tid * kScanPer + u;
      if (t <= kMaxTime) {
        hist[t] = run;     // becomes the bin's cursor
        tp[t] = run;
      }
      run += v[u];
    }
    __syncthreads();
    for (int64_t base = b; base < e; base += kSortThreads * kSortU) {
      uint32_t pv[kSortU], tv[kSortU], qv[kSortU];
#pragma unroll
      for (int u = 0; u < kSortU; ++u) {
        const int64_t i = base + u * kSortThreads + tid;
        pv[u] = i < e ? P.pad[i] : 0u;
        tv[u] = i < e ? P.time[i] : 0u;
        qv[u] = i < e ? P.adc[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kSortU; ++u) {
        if (base + u * kSortThreads + tid >= e) break;
        if ((int)pv[u] < np && (int)tv[u] < nt && qv[u] < 32768u) {
          const int at = atomicAdd(&hist[tv[u]], 1);
          P.srt[b + at] = pv[u] | (tv[u] << 8) | (qv[u] << 17);
        }
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int w_cell(uint32_t w, int t0, int W) {
  return ((int)((w >> 8) & 511u) - t0 + kHalo) * W + (int)(w & 255u) + 2;
}

// Pass 2: one (row, time tile) per work item, its digits a contiguous range
// of the sorted row.
__global__ void __launch_bounds__(kCfThreads, kCfPerSm) k_clusterer(const __grid_constant__ CfDev P) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int W = P.wp;
  const int map_words = kMapRows * W / 2, bit_words = kMapRows * W / 32;
  uint16_t* map = reinterpret_cast<uint16_t*>(smem);
  uint32_t* peak_bits = smem + map_words;
  uint32_t* kept_bits = peak_bits + bit_words;
  uint32_t* peaks = kept_bits + bit_words;        // map cells of the kept peaks, in (time, pad) order
  // an item's row start and sorted ranges: the map (tile +- 3 bins), the
  // peak tests (+- 2), the core; kept by parity like the item index
  __shared__ int s_item[2];
  __shared__ long long s_rb[2];
  __shared__ int s_rng[2][6];
  __shared__ int s_at;
  __shared__ int s_wsum[kCfWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = P.n_time;
  const int n_items = P.n_inst * P.n_rows * P.n_tiles;
  const tpct_cf_out& O = P.out;
  // tid 0 reads an item's row start and ranges (two independent loads deep)
  auto item_ranges = [&](int itm, long long& rb_o, int* rng) {
    const int rw = itm / P.n_tiles, tl = itm % P.n_tiles;
    const int a = tl * kTileT, z = min(a + kTileT, nt);
    const int32_t* tq = P.tpos + (int64_t)rw * (kMaxTime + 1);
    rb_o = P.row_offsets[rw];
    rng[0] = tq[max(a - 3, 0)]; rng[1] = tq[min(z + 3, nt)];
    rng[2] = tq[max(a - 2, 0)]; rng[3] = tq[min(z + 2, nt)];
    rng[4] = tq[a];             rng[5] = tq[z];
  };

  for (int i = tid; i < map_words + 2 * bit_words; i += kCfThreads) smem[i] = 0u;
  if (tid == 0) {
    const int it0 = (int)atomicAdd(&P.work[0], 1u);
    s_item[0] = it0;
    if (it0 < n_items) {
      long long rb0;
      int rng0[6];
      item_ranges(it0, rb0, rng0);
      s_rb[0] = rb0;
      for (int q = 0; q < 6; ++q) s_rng[0][q] = rng0[q];
    }
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    const int item = s_item[cur];
    if (item >= n_items) break;
    // the next item, taken now (no CTA waits for another, so holding it costs
    // nothing); tid 0 reads its ranges during this item and hands them over
    // at its end
    int nx = 0;
    long long nx_rb = 0;
    int nx_rng[6] = {0, 0, 0, 0, 0, 0};
    if (tid == 0) nx = (int)atomicAdd(&P.work[0], 1u);
    const int tile = item % P.n_tiles;
    const int t0 = tile * kTileT, t1 = min(t0 + kTileT, nt);
    const int core_lo = kHalo * W, core_hi = (t1 - t0 + kHalo) * W;
    const uint32_t* sd = P.srt + s_rb[cur];
    const int m_lo = s_rng[cur][0], m_hi = s_rng[cur][1];
    const int p_lo = s_rng[cur][2], p_hi = s_rng[cur][3];
    const int c_lo = s_rng[cur][4], c_hi = s_rng[cur][5];

    for (int k = m_lo + tid; k < m_hi; k += kCfThreads) {
      const uint32_t w = sd[k];
      map[w_cell(w, t0, W)] = (uint16_t)(w >> 17);
    }
    __syncthreads();
    if (tid == 0 && nx < n_items) item_ranges(nx, nx_rb, nx_rng);   // used at the end of this item
    for (int k = p_lo + tid; k < p_hi; k += kCfThreads) {
      const int c = w_cell(sd[k], t0, W);
      if (peak_test(map, W, c, P.q_peak_min)) atomicOr(&peak_bits[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    for (int k = c_lo + tid; k < c_hi; k += kCfThreads) {
      const int c = w_cell(sd[k], t0, W);
      if (bit_at(peak_bits, c) && !suppressed(map, peak_bits, W, c, P.valley_delta))
        atomicOr(&kept_bits[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    // rank the kept peaks in cell order = (time, pad) order: one scan over the
    // bitmap words of the tile's time bins (W is a multiple of 32, so a word
    // never straddles two time bins)
    const int w_lo = core_lo >> 5, w_hi = core_hi >> 5;
    int sum = 0;
#pragma unroll
    for (int u = 0; u < kWordsPer; ++u) {
      const int wi = w_lo + tid * kWordsPer + u;
      sum += wi < w_hi ? __popc(kept_bits[wi]) : 0;
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kCfWarps; ++q) {
      const int v = s_wsum[q];
      wbase += q < warp ? v : 0;
      total += v;
    }
    int rank = wbase + incl - sum;
#pragma unroll
    for (int u = 0; u < kWordsPer; ++u) {
      const int wi = w_lo + tid * kWordsPer + u;
      if (wi >= w_hi) break;
      uint32_t m = kept_bits[wi];
      while (m) {
        const int bpos = __ffs(m) - 1;
        m &= m - 1;
        if (rank < kCfMaxPeaks) peaks[rank] = (uint32_t)(wi * 32 + bpos);
        ++rank;
      }
    }
    __syncthreads();   // peaks[] complete
    // staging slots: one atomic per item, issued before the first cluster is
    // built (from shared memory, into registers) and read after it
    const int nk = min(total, kCfMaxPeaks);
    int at_mine = 0;
    if (tid == 0) {
      if (total > kCfMaxPeaks) atomicOr(O.status, TPCT_CF_ROW_OVERFLOW);
      at_mine = nk > 0 ? (int)atomicAdd(&P.work[1], (uint32_t)nk) : 0;
    }
    Cluster mine;
    if (tid < nk) mine = build_cluster(map, W, (int)peaks[tid], t0);
    if (tid == 0) {
      s_at = at_mine;
      P.item_cnt[item] = nk;
      P.item_at[item] = at_mine;
    }
    __syncthreads();
    const long long at = s_at;
    auto stage = [&](int k, const Cluster& c) {
      if (at + k >= O.capacity) return;   // the output is too small: reported by the emit pass
      CfStage g;
      g.cp = c.cp; g.ct = c.ct; g.sp = c.sp; g.st = c.st; g.qtot = c.qtot;
      g.ptq = (uint32_t)c.p | ((uint32_t)c.t << 8) | ((uint32_t)c.q << 17);
      P.stage[at + k] = g;
    };
    if (tid < nk) stage(tid, mine);
    for (int k = kCfThreads + tid; k < nk; k += kCfThreads) stage(k, build_cluster(map, W, (int)peaks[k], t0));
    __syncthreads();
    // clear what this item set: the map cells of its digits and the bitmap
    // words holding their bits
    for (int k = m_lo + tid; k < m_hi; k += kCfThreads) {
      const int c = w_cell(sd[k], t0, W);
      map[c] = 0;
      peak_bits[c >> 5] = 0u;
      kept_bits[c >> 5] = 0u;
    }
    if (tid == 0) {   // the other parity slot: read by all before this item's first barrier
      s_item[nxt] = nx;
      s_rb[nxt] = nx_rb;
      for (int q = 0; q < 6; ++q) s_rng[nxt][q] = nx_rng[q];
    }
    __syncthreads();
  }
}

// One warp per item: the staged clusters to their place in the output.
__global__ void __launch_bounds__(kEmitThreads) k_cf_emit(const __grid_constant__ CfDev P) {
  const int lane = threadIdx.x & 31;
  const int n_items = P.n_inst * P.n_rows * P.n_tiles;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const tpct_cf_out& O = P.out;
  const long long cap = O.capacity;
  for (int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < n_items; item += warps) {
    const int cnt = P.item_cnt[item];
    const long long src = P.item_at[item], dst = P.item_dst[item];
    const int row = item / P.n_tiles, tile = item % P.n_tiles;
    const int r = row % P.n_rows, inst = row / P.n_rows;
    if (lane == 0 && r == 0 && tile == 0 && O.inst_offsets) O.inst_offsets[inst] = dst;
    if (cnt == 0) continue;
    const int np = P.n_pad[r];
    const float pitch = P.pitch[r], xr = P.row_x[r];
    const float side = P.inst_sector[inst] >= 18 ? -1.f : 1.f;
    for (int k = lane; k < cnt; k += 32) {
      if (src + k >= cap || dst + k >= cap) break;
      const CfStage g = P.stage[src + k];
      Cluster c;
      c.cp = g.cp; c.ct = g.ct; c.sp = g.sp; c.st = g.st; c.qtot = g.qtot;
      c.p = (int)(g.ptq & 255u); c.t = (int)((g.ptq >> 8) & 511u); c.q = (int)(g.ptq >> 17);
      store_cluster(O, dst + k, c, xr, pitch, np, P.n_time, side, P.z_max, P.time_bin, r);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long total = P.item_dst[n_items];
    *O.n_clusters = (int32_t)total;
    if (O.inst_offsets) O.inst_offsets[P.n_inst] = total;
    if (total > cap) atomicOr(O.status, TPCT_CF_CAPACITY);
  }
}

}  // namespace

// Host side ------------------------------------------------------------------

int cf_pads(double row_x, double tan_half, double pitch) {
  return 2 * (int)std::ceil(row_x * tan_half / pitch - 1e-9);
}

size_t cf_smem_bytes(int wp) {
  return 4 * ((size_t)kMapRows * wp / 2 + 2 * (size_t)kMapRows * wp / 32 + kCfMaxPeaks);
}

namespace {
// Workspace: counters | item counts | staging slots | output slots (+ total) |
// scan temporaries | sorted digits | time-bin starts | staging area.
size_t cf_carve(char* base, int64_t n_digits, size_t n_rows_total, size_t n_items, int32_t capacity, CfDev* P,
                uint64_t** tmp) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* q = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  uint32_t* work = (uint32_t*)take(256);
  int32_t* cnt = (int32_t*)take(4 * std::max<size_t>(n_items, 1));
  int32_t* at = (int32_t*)take(4 * std::max<size_t>(n_items, 1));
  int32_t* dst = (int32_t*)take(4 * (n_items + 1));
  uint64_t* t = (uint64_t*)take(8 * ((size_t)scan_tmp_elems((int64_t)n_items) + 32));
  int32_t* tpos = (int32_t*)take(4 * (size_t)(kMaxTime + 1) * std::max<size_t>(n_rows_total, 1));
  CfStage* stage = (CfStage*)take(sizeof(CfStage) * (size_t)std::max(capacity, 1));
  uint32_t* srt = (uint32_t*)take(4 * (size_t)std::max<int64_t>(n_digits, 1));   // last: sized by the caller
  if (P) {
    P->work = work; P->item_cnt = cnt; P->item_at = at; P->item_dst = dst; P->stage = stage;
    P->srt = srt; P->tpos = tpos;
    *tmp = t;
  }
  return off;
}
}  // namespace

// Enqueue cluster finding; returns the kernels launched, or -1 (invalid
// readout), -2 (workspace too small), -3 (shared memory too large), -4 (CUDA).
int enqueue_clusters(const double* row_x, int n_rows, double tan_half, double z_max, const tpct_cf_params& prm,
                     const tpct_digits& dg, void* ws, size_t ws_bytes, const tpct_cf_out& out, cudaStream_t s,
                     cudaError_t* err) {
  if (n_rows < 1 || n_rows > kMaxRows || prm.n_time < 1 || prm.n_time > 512 || !(prm.time_bin > 0) ||
      !(prm.pad_pitch_inner > 0) || !(prm.pad_pitch_outer > 0))
    return -1;
  CfDev P{};
  int np_max = 0;
  for (int r = 0; r < n_rows; ++r) {
    const double pitch = r < prm.n_inner_rows ? prm.pad_pitch_inner : prm.pad_pitch_outer;
    const int np = cf_pads(row_x[r], tan_half, pitch);
    if (np < 1 || np > 252) return -1;
    P.n_pad[r] = (int16_t)np;
    P.pitch[r] = (float)pitch;
    P.row_x[r] = (float)row_x[r];
    np_max = np > np_max ? np : np_max;
  }
  const int wp = (np_max + 4 + 31) / 32 * 32;
  const size_t smem = cf_smem_bytes(wp);
  int dev = 0, max_optin = 0, n_sm = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return -4;
  if ((*err = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return -4;
  if ((*err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return -4;
  if (smem + 1024 > (size_t)max_optin) return -3;
  const int n_tiles = (prm.n_time + kTileT - 1) / kTileT;
  const size_t n_rows_total = (size_t)dg.n_instances * n_rows;
  const size_t n_items = n_rows_total * n_tiles;
  // the sorted digits take the rest of the workspace (rows that end beyond
  // it are skipped and reported on the device)
  uint64_t* tmp = nullptr;
  const size_t srt_at = cf_carve(nullptr, 1, n_rows_total, n_items, out.capacity, nullptr, nullptr) - 256;
  if (ws_bytes < srt_at + 256) return -2;
  cf_carve((char*)ws, 1, n_rows_total, n_items, out.capacity, &P, &tmp);
  P.srt_cap = (int64_t)((ws_bytes - srt_at) / 4);
  P.pad = dg.pad; P.time = dg.time; P.adc = dg.adc; P.row_offsets = dg.row_offsets; P.inst_sector = dg.inst_sector;
  P.n_inst = dg.n_instances; P.n_rows = n_rows; P.n_time = prm.n_time; P.n_tiles = n_tiles; P.wp = wp;
  P.q_peak_min = prm.q_peak_min; P.valley_delta = prm.valley_delta;
  P.z_max = (float)z_max; P.time_bin = (float)prm.time_bin;
  P.out = out;
  if ((*err = cudaFuncSetAttribute(k_clusterer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return -4;
  int per_sm = 0;
  if ((*err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clusterer, kCfThreads, smem)) != cudaSuccess)
    return -4;
  int k = 0;
  cudaMemsetAsync(P.work, 0, 256, s);
  cudaMemsetAsync(out.status, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(out.n_clusters, 0, sizeof(int32_t), s);
  if (n_items > 0) {
    k_cf_sort<<<(int)std::min<size_t>(n_rows_total, (size_t)n_sm * 8), kSortThreads, 0, s>>>(P); ++k;
    const int grid = (int)std::min<size_t>((size_t)n_sm * std::max(per_sm, 1), n_items);
    k_clusterer<<<grid, kCfThreads, smem, s>>>(P); ++k;
  }
  launch_scan_i32(P.item_cnt, P.item_dst, (int64_t)n_items, tmp, s); k += n_items > 0 ? 3 : 1;
  const int emit_blocks = (int)std::max<size_t>(1, std::min<size_t>((n_items * 32 + kEmitThreads - 1) / kEmitThreads,
                                                                      (size_t)n_sm * 16));
  k_cf_emit<<<emit_blocks, kEmitThreads, 0, s>>>(P); ++k;
  *err = cudaGetLastError();
  return *err == cudaSuccess ? k : -4;
}

size_t cf_workspace_bytes(int64_t n_digits, int32_t n_instances, int32_t n_rows, int32_t capacity) {
  const size_t n_rows_total = (size_t)n_instances * n_rows;
  return cf_carve(nullptr, n_digits, n_rows_total, n_rows_total * ((kMaxTime + kTileT - 1) / kTileT), capacity,
                  nullptr, nullptr);
}

}  // namespace tpct
