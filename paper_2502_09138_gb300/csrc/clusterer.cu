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
// Clusters of a row come in the input order of their peak digits; rows in
// (instance, row) order.
//
// GB300 mapping: a persistent kernel with one 1024-thread CTA per SM.  A CTA
// takes whole pad rows from a device work counter and keeps the row's charge
// map (n_pad x n_time u16, 140 KB for the outermost row) and a peak bitmap in
// shared memory: digits are scattered in once from HBM (coalesced), every
// neighbourhood test then reads shared memory only, and the map is cleared by
// re-scattering zeros at the same cells.  Output positions come from a
// single-pass decoupled look-back over the rows (each row publishes its
// cluster count, then its inclusive prefix), so clusters are written once,
// densely and in order.  Waits in the look-back are bounded; a timeout sets a
// status bit.
#include "tpct_internal.cuh"

namespace tpct {
namespace {

constexpr int kCfThreads = 1024;
constexpr int kCfMaxPeaks = 8192;          // kept peaks per row held in shared memory
constexpr int kCfPerThread = 8;            // digits per thread: rows of up to 8192 digits
constexpr int kCfMaxSpins = 1 << 22;       // look-back polls before giving up
constexpr uint64_t kLbAgg = 1ull << 62, kLbInc = 2ull << 62, kLbMask = (1ull << 62) - 1;

struct CfDev {
  const uint16_t *pad, *time, *adc;
  const int64_t* row_offsets;
  const int32_t* inst_sector;
  int32_t n_inst, n_rows, n_time, np_max;
  int32_t q_peak_min, valley_delta;
  float z_max, time_bin;
  uint32_t map_words, bit_words;            // shared-memory layout (32-bit words)
  uint64_t* lookback;                       // [n_inst * n_rows]
  uint32_t* work;                           // [1]
  int16_t n_pad[kMaxRows];
  float pitch[kMaxRows], row_x[kMaxRows];
  tpct_cf_out out;
};

// The row map has a border of two empty cells on every side: cell (p, t) of
// the row lives at (p + 2) * W + (t + 2) with W = n_time + 4, so every
// neighbourhood read up to distance 2 stays inside the map without a bounds
// test (border and unused cells hold 0; the peak bitmap has the same layout).
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
      const int qn = map[c + dp * W + dt];
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
      const int c2 = c + dp * W + dt;
      if (!bit_at(bits, c2)) continue;
      const int q2 = map[c2];
      if (!(q2 > q || (q2 == q && before(dp, dt)))) continue;
      sup |= (int)map[c + half_step(dp) * W + half_step(dt)] >= q - delta;
    }
  return sup;
}

__device__ __forceinline__ uint64_t ld_volatile(const uint64_t* a) {
  return *reinterpret_cast<const volatile unsigned long long*>(a);
}

// A digit in one register: pad (8 bits) | time (9 bits) | adc (15 bits).
constexpr uint32_t kNoDigit = 0xffffffffu;
__device__ __forceinline__ int w_pad(uint32_t w) { return (int)(w >> 24); }
__device__ __forceinline__ int w_time(uint32_t w) { return (int)((w >> 15) & 511u); }
__device__ __forceinline__ int w_adc(uint32_t w) { return (int)(w & 32767u); }

struct Cluster {
  float cp, ct, sp, st;
  uint32_t qtot;
  uint32_t packed;   // the peak digit
};

__device__ __forceinline__ Cluster build_cluster(const uint16_t* map, int W, uint32_t pw) {
  const int p = w_pad(pw), t = w_time(pw);
  const int c = (p + 2) * W + (t + 2);
  int s0 = 0, sp = 0, st = 0, spp = 0, stt = 0;
#pragma unroll
  for (int dt = -2; dt <= 2; ++dt)
#pragma unroll
    for (int dp = -2; dp <= 2; ++dp) {
      const int qc = map[c + dp * W + dt];
      const bool outer = dp == 2 || dp == -2 || dt == 2 || dt == -2;
      const bool take = qc > 0 && (!outer || qc <= (int)map[c + half_step(dp) * W + half_step(dt)]);
      const int q = take ? qc : 0;
      s0 += q; sp += q * dp; st += q * dt; spp += q * dp * dp; stt += q * dt * dt;
    }
  const float fs0 = (float)s0;
  const float mp = __fdiv_rn((float)sp, fs0), mt = __fdiv_rn((float)st, fs0);
  Cluster k;
  k.cp = (float)p + mp;
  k.ct = (float)t + mt;
  k.sp = sqrtf(fmaxf(__fdiv_rn((float)spp, fs0) - mp * mp, 0.f));
  k.st = sqrtf(fmaxf(__fdiv_rn((float)stt, fs0) - mt * mt, 0.f));
  k.qtot = (uint32_t)s0;
  k.packed = pw;
  return k;
}

__device__ __forceinline__ void store_cluster(const tpct_cf_out& O, long long slot, const Cluster& k, float row_x,
                                              float pitch, int np, int nt, float side, float z_max, float time_bin,
                                              int r) {
  const int p = w_pad(k.packed), t = w_time(k.packed);
  O.pad[slot] = k.cp;
  O.time[slot] = k.ct;
  O.sigma_pad[slot] = k.sp;
  O.sigma_time[slot] = k.st;
  O.x[slot] = row_x;
  O.y[slot] = (k.cp + 0.5f - 0.5f * (float)np) * pitch;
  O.z[slot] = side * (z_max - (k.ct + 0.5f) * time_bin);
  O.q_tot[slot] = k.qtot;
  O.q_max[slot] = (uint16_t)w_adc(k.packed);
  O.row[slot] = (uint8_t)r;
  O.flags[slot] = (uint8_t)((p == 0 || p == np - 1 ? 1 : 0) | (t == 0 || t == nt - 1 ? 2 : 0));
}

__global__ void __launch_bounds__(kCfThreads, 1) k_clusterer(const __grid_constant__ CfDev P) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint16_t* map = reinterpret_cast<uint16_t*>(smem);
  uint32_t* bits = smem + P.map_words;
  uint32_t* peaks = bits + P.bit_words;          // kept peaks of the row (packed digits), in input order
  __shared__ int s_next[2];                     // row of this / the next iteration (by parity)
  __shared__ long long s_nb[2], s_ne[2];
  __shared__ uint32_t s_ball[kCfPerThread][kCfThreads / 32];
  __shared__ int s_pref[kCfPerThread][kCfThreads / 32];
  __shared__ int s_count;
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lanes_below = (1u << lane) - 1u;
  const int nt = P.n_time, W = nt + 4;
  const int n_rows_total = P.n_inst * P.n_rows;
  const tpct_cf_out& O = P.out;

  for (uint32_t i = tid; i < P.map_words + P.bit_words; i += kCfThreads) smem[i] = 0u;
  if (tid == 0) {
    const int r0 = (int)atomicAdd(P.work, 1u);
    s_next[0] = r0;
    if (r0 < n_rows_total) { s_nb[0] = P.row_offsets[r0]; s_ne[0] = P.row_offsets[r0 + 1]; }
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    const int row = s_next[cur];
    if (row >= n_rows_total) break;
    const int64_t b = s_nb[cur], e = s_ne[cur];
    // the next row's index and range, fetched while this row is processed
    // (the other parity slot: every thread read it before the last barrier)
    if (tid == 0) {
      const int nx = (int)atomicAdd(P.work, 1u);
      s_next[nxt] = nx;
      if (nx < n_rows_total) { s_nb[nxt] = P.row_offsets[nx]; s_ne[nxt] = P.row_offsets[nx + 1]; }
    }
    const int r = row % P.n_rows, inst = row / P.n_rows;
    const int np = P.n_pad[r];
    if (tid == 0 && e - b > (int64_t)kCfPerThread * kCfThreads) atomicOr(O.status, TPCT_CF_ROW_OVERFLOW);

    // the row's digits, k-major (digit b + k * 1024 + tid), loaded once
    uint32_t w[kCfPerThread];
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k) {
      const int64_t i = b + (int64_t)k * kCfThreads + tid;
      w[k] = kNoDigit;
      if (i < e) {
        const uint32_t p = P.pad[i], t = P.time[i], q = P.adc[i];
        if ((int)p < np && (int)t < nt && q < 32768u) w[k] = (p << 24) | (t << 15) | q;
        else atomicOr(O.status, TPCT_CF_BAD_DIGIT);
      }
    }
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k)
      if (w[k] != kNoDigit) map[(w_pad(w[k]) + 2) * W + w_time(w[k]) + 2] = (uint16_t)w_adc(w[k]);
    __syncthreads();
    // peaks
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k)
      if (w[k] != kNoDigit) {
        const int c = (w_pad(w[k]) + 2) * W + w_time(w[k]) + 2;
        if (peak_test(map, W, c, P.q_peak_min)) atomicOr(&bits[c >> 5], 1u << (c & 31));
      }
    __syncthreads();
    // kept peaks: one ballot per k, then one scan over (k, warp) gives every
    // kept digit its rank in input order
    uint32_t keep = 0u;
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k) {
      bool kp = false;
      if (w[k] != kNoDigit) {
        const int c = (w_pad(w[k]) + 2) * W + w_time(w[k]) + 2;
        kp = bit_at(bits, c) && !suppressed(map, bits, W, c, P.valley_delta);
      }
      const uint32_t ball = __ballot_sync(0xffffffffu, kp);
      if (lane == 0) s_ball[k][warp] = ball;
      keep |= (kp ? 1u : 0u) << k;
    }
    __syncthreads();
    if (warp == 0) {
      // lane j owns the (k, warp) entries [kPer j, kPer (j + 1)) of the k-major list
      constexpr int kPer = kCfPerThread * (kCfThreads / 32) / 32;
      int loc[kPer], sum = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int f = lane * kPer + u;
        loc[u] = sum;
        sum += __popc(s_ball[f / (kCfThreads / 32)][f % (kCfThreads / 32)]);
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int excl = incl - sum;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int f = lane * kPer + u;
        s_pref[f / (kCfThreads / 32)][f % (kCfThreads / 32)] = excl + loc[u];
      }
      if (lane == 31) s_count = incl;
    }
    __syncthreads();
    const int count = s_count;
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k)
      if ((keep >> k) & 1u) {
        const int rank = s_pref[k][warp] + __popc(s_ball[k][warp] & lanes_below);
        if (rank < kCfMaxPeaks) peaks[rank] = w[k];
      }
    if (count > kCfMaxPeaks && tid == 0) atomicOr(O.status, TPCT_CF_ROW_OVERFLOW);
    __syncthreads();

    // The last warp runs the decoupled look-back (publish the row's count,
    // read the states of the 32 preceding rows at once; the nearest one with
    // an inclusive prefix ends the walk, all nearer ones must have published
    // their counts; else add all 32 counts and move 32 rows back; publish the
    // inclusive prefix) while the other warps build their first clusters.
    const int nk = min(count, kCfMaxPeaks);
    constexpr int kBuilders = kCfThreads - 32;
    Cluster mine;
    const bool have = warp < kCfThreads / 32 - 1 && tid < nk;
    if (have) mine = build_cluster(map, W, peaks[tid]);
    if (warp == kCfThreads / 32 - 1) {
      long long prefix = 0;
      if (lane == 0) {
        __threadfence();
        atomicExch((unsigned long long*)&P.lookback[row],
                   (unsigned long long)((row == 0 ? kLbInc : kLbAgg) | (uint64_t)count));
      }
      if (row > 0) {
        int j0 = row - 1, spins = 0;
        while (true) {
          const int j = j0 - lane;
          const uint64_t v = j >= 0 ? ld_volatile(&P.lookback[j]) : kLbInc;   // before row 0: prefix 0
          const uint32_t st = (uint32_t)(v >> 62);
          const uint32_t inc = __ballot_sync(0xffffffffu, st == 2u);
          const uint32_t unset = __ballot_sync(0xffffffffu, st == 0u);
          const int first = inc ? __ffs(inc) - 1 : 32;
          const uint32_t upto = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
          if (unset & upto) {
            if (++spins > kCfMaxSpins) {
              if (lane == 0) atomicOr(O.status, TPCT_CF_TIMEOUT);
              break;
            }
            __nanosleep(64);
            continue;
          }
          long long val = lane <= first ? (long long)(v & kLbMask) : 0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
          prefix += __shfl_sync(0xffffffffu, val, 0);
          if (first < 32) break;
          j0 -= 32;
        }
        if (lane == 0) {
          __threadfence();
          atomicExch((unsigned long long*)&P.lookback[row],
                     (unsigned long long)(kLbInc | (uint64_t)(prefix + count)));
        }
      }
      if (lane == 0) {
        s_base = prefix;
        if (r == 0 && O.inst_offsets) O.inst_offsets[inst] = prefix;
        if (row == n_rows_total - 1) {
          *O.n_clusters = (int32_t)min(prefix + count, (long long)0x7fffffff);
          if (O.inst_offsets) O.inst_offsets[P.n_inst] = prefix + count;
          if (prefix + count > O.capacity) atomicOr(O.status, TPCT_CF_CAPACITY);
        }
      }
    }
    __syncthreads();
    const long long base_out = s_base;
    const float pitch = P.pitch[r], xr = P.row_x[r];
    const float side = P.inst_sector[inst] >= 18 ? -1.f : 1.f;
    if (have && base_out + tid < O.capacity)
      store_cluster(O, base_out + tid, mine, xr, pitch, np, nt, side, P.z_max, P.time_bin, r);
    for (int k = kBuilders + tid; k < nk; k += kCfThreads) {   // rows with more clusters than builders
      if (base_out + k >= O.capacity) break;
      store_cluster(O, base_out + k, build_cluster(map, W, peaks[k]), xr, pitch, np, nt, side, P.z_max,
                    P.time_bin, r);
    }
    __syncthreads();
    // clear the row's cells and peak bits
#pragma unroll
    for (int k = 0; k < kCfPerThread; ++k)
      if (w[k] != kNoDigit) {
        const int c = (w_pad(w[k]) + 2) * W + w_time(w[k]) + 2;
        map[c] = 0;
        bits[c >> 5] = 0u;
      }
    __syncthreads();
  }
}

}  // namespace

// Host side ------------------------------------------------------------------

int cf_pads(double row_x, double tan_half, double pitch) {
  return 2 * (int)std::ceil(row_x * tan_half / pitch - 1e-9);
}

// map: (np_max + 4) x (n_time + 4) u16 with a two-cell empty border; bitmap: one bit per map cell
size_t cf_map_cells(int np_max, int n_time) { return (size_t)(np_max + 4) * (n_time + 4); }
size_t cf_smem_bytes(int np_max, int n_time) {
  const size_t cells = cf_map_cells(np_max, n_time);
  return 4 * ((cells + 1) / 2 + (cells + 31) / 32) + 4 * (size_t)kCfMaxPeaks;
}

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
    if (np < 1 || np > 256) return -1;
    P.n_pad[r] = (int16_t)np;
    P.pitch[r] = (float)pitch;
    P.row_x[r] = (float)row_x[r];
    np_max = np > np_max ? np : np_max;
  }
  const size_t smem = cf_smem_bytes(np_max, prm.n_time);
  int dev = 0, max_optin = 0, n_sm = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return -4;
  if ((*err = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return -4;
  if ((*err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return -4;
  if (smem + 2048 > (size_t)max_optin) return -3;
  const size_t n_rows_total = (size_t)dg.n_instances * n_rows;
  const size_t need = 8 * n_rows_total + 256;
  if (ws_bytes < need) return -2;
  P.pad = dg.pad; P.time = dg.time; P.adc = dg.adc; P.row_offsets = dg.row_offsets; P.inst_sector = dg.inst_sector;
  P.n_inst = dg.n_instances; P.n_rows = n_rows; P.n_time = prm.n_time; P.np_max = np_max;
  P.q_peak_min = prm.q_peak_min; P.valley_delta = prm.valley_delta;
  P.z_max = (float)z_max; P.time_bin = (float)prm.time_bin;
  P.map_words = (uint32_t)((cf_map_cells(np_max, prm.n_time) + 1) / 2);
  P.bit_words = (uint32_t)((cf_map_cells(np_max, prm.n_time) + 31) / 32);
  P.work = (uint32_t*)ws;
  P.lookback = (uint64_t*)((char*)ws + 256);
  P.out = out;
  if ((*err = cudaFuncSetAttribute(k_clusterer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return -4;
  int k = 0;
  cudaMemsetAsync(ws, 0, need, s);
  cudaMemsetAsync(out.status, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(out.n_clusters, 0, sizeof(int32_t), s);
  if (n_rows_total > 0) {
    const int grid = (int)std::min<size_t>((size_t)n_sm, n_rows_total);
    k_clusterer<<<grid, kCfThreads, smem, s>>>(P); ++k;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? k : -4;
}

size_t cf_workspace_bytes(int32_t n_instances, int32_t n_rows) {
  return 8 * (size_t)n_instances * n_rows + 256;
}

}  // namespace tpct
