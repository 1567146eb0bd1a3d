// Steps 6-7 of sector track finding: selection by owned clusters and shared
// fraction, output compaction, and the iterated refit of every selected
// track.  (The paper's "TPC Processing (Tracking)", Tables 1-3.)
#include "refit_update.cuh"

namespace tpct {
namespace {

constexpr int kBlock = 256;

// A hint to bring the line holding a (a valid address) into L1.
__device__ __forceinline__ void prefetch_l1(const void* a) { asm volatile("prefetch.global.L1 [%0];" :: "l"(a)); }

__device__ __forceinline__ int tracklet_count(const Params& P) {
  return min(P.row_tl_base[P.n_inst * P.n_rows], P.tcap);
}

// Weight of tracklet t: longer wins, then the earlier start hit of the sector.
__device__ __forceinline__ uint32_t tracklet_weight(const Params& P, int t, int nh) {
  const int ir = P.tl_ir[t];
  const int inst_row0 = ir - ir % P.n_rows;
  int rank = t - P.row_tl_base[inst_row0];
  if (rank > (int)kRankMask) rank = (int)kRankMask;
  return ((uint32_t)nh << kRankBits) | (kRankMask - (uint32_t)rank);
}

// W[c] = max weight over the tracklets that hold c (order independent).
__global__ void k_weights(const __grid_constant__ Params P) {
  const int n_tl = tracklet_count(P);
  const int R = P.n_rows;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tl; t += gridDim.x * blockDim.x) {
    const int nh = P.tl_nhits[t];
    const uint32_t w = tracklet_weight(P, t, nh);
    // slots from R-1 down (slot-major: the lanes of a warp read one slot row)
    for (int j = R - 1; j >= R - nh; --j) atomicMax(&P.W[P.tl_hits[hit_at(P, t, j)]], w);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int T = P.row_tl_base[P.n_inst * R];
    if (T > P.tcap) atomicOr(P.status, kDevTrackletCap);
  }
}

// owned = clusters whose weight is this tracklet's; accept iff owned >= n_min
// and shared <= f_shared * nhits.  tl_sel[t] = accepted << 32 | owned.
__global__ void k_own(const __grid_constant__ Params P) {
  const int n_tl = tracklet_count(P);
  const int R = P.n_rows;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.tcap; t += gridDim.x * blockDim.x) {
    uint64_t sel = 0;
    if (t < n_tl) {
      const int nh = P.tl_nhits[t];
      const uint32_t w = tracklet_weight(P, t, nh);
      int own = 0;
      for (int j = R - 1; j >= R - nh; --j) own += P.W[P.tl_hits[hit_at(P, t, j)]] == w;
      const bool acc = own >= P.n_min && (double)(nh - own) <= P.f_shared * (double)nh;
      if (acc) sel = (1ull << 32) | (uint64_t)own;
    }
    P.tl_sel[t] = sel;
  }
}

__global__ void k_emit(const __grid_constant__ Params P) {
  const int n_tl = tracklet_count(P);
  const int R = P.n_rows;
  const uint64_t total = P.tl_sel_scan[P.tcap];
  const int n_trk = (int)(total >> 32), n_ids = (int)(total & 0xffffffffu);
  const tpct_tracks_out& O = P.out;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *O.n_tracks = n_trk;
    *O.n_ids = n_ids;
    if (n_trk > O.capacity_tracks || n_ids > O.capacity_ids) atomicOr(P.status, kDevCapacity);
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tl; t += gridDim.x * blockDim.x) {
    const uint64_t sel = P.tl_sel[t];
    if (!sel) continue;
    const uint64_t sc = P.tl_sel_scan[t];
    const int k = (int)(sc >> 32), off = (int)(sc & 0xffffffffu);
    const int own = (int)(sel & 0xffffffffu);
    if (k >= O.capacity_tracks) continue;
    const int nh = P.tl_nhits[t];
    const uint32_t w = tracklet_weight(P, t, nh);
    O.instance[k] = P.tl_ir[t] / R;
    O.n_cl[k] = own;
    O.offset[k] = off;
    O.ndf[k] = 2 * own - 5;
    P.trk_tl[k] = t;
    if (off + own > O.capacity_ids) continue;   // ids overflow: sizes reported, refit skips it
    // owned clusters row-ascending: walk the slots from the top row down and
    // fill the track's id range from its end
    int m = own;
    for (int j = R - 1; j >= R - nh; --j) {
      const int p = P.tl_hits[hit_at(P, t, j)];
      if (P.W[p] == w) {
        --m;
        O.cluster_ids[off + m] = P.sid[p];
        P.trk_pos[off + m] = p;
      }
    }
  }
}

// Iterated refit: each pass transports the previous estimate (exact helix) to
// the outermost owned cluster and along all owned clusters inward (the
// reference trajectory), and filters the deviation from it with a diffuse
// prior; reference + deviation at the innermost cluster is the next estimate.
//
// Persistent: every lane runs one track as a state machine, one cluster per
// loop iteration, and takes the next track from a device work queue when it
// finishes, so the covariance arithmetic runs with full warps.
template <int MODE, int STAGE> struct RefitTypes {
  using S = typename Prec<MODE>::RS; using E = typename Prec<MODE>::RE; using C = typename Prec<MODE>::RC;
};
template <int MODE> struct RefitTypes<MODE, 1> {
  using S = typename Prec<MODE>::PS; using E = typename Prec<MODE>::PE; using C = typename Prec<MODE>::PC;
};
// STAGE 3: the last pass after its first kRefitHead clusters (double-float)
template <int MODE> struct RefitTypes<MODE, 3> {
  using S = typename Prec<MODE>::PS; using E = typename Prec<MODE>::PE; using C = typename Prec<MODE>::PC;
};

template <int MODE, int STAGE>
__global__ void __launch_bounds__(kMaxBlock) k_refit(const __grid_constant__ Params P) {
  using S = typename RefitTypes<MODE, STAGE>::S;
  using E = typename RefitTypes<MODE, STAGE>::E;
  using C = typename RefitTypes<MODE, STAGE>::C;
  // STAGE 0: all passes; 1: the leading passes; 2: the last pass, handing a
  // track over after its first kRefitHead clusters; 3: the rest of the last pass
  const int pass_begin = STAGE >= 2 ? P.n_refit - 1 : 0;
  const int pass_end = STAGE == 1 ? P.n_refit - 1 : P.n_refit;
  const tpct_tracks_out& O = P.out;
  const uint64_t total = P.tl_sel_scan[P.tcap];
  const int n_trk = min((int)(total >> 32), O.capacity_tracks);
  const E kb = (E)P.kb, smax = (E)P.s_max;
  const int lane = threadIdx.x & 31;
  const uint32_t lanes_below = (1u << lane) - 1u;

  int k = -1, n = 0, t = 0, pass = 0, j = 0, status = 0;
  bool exhausted = false;
  const int* pos = P.trk_pos;
  double x_cur = 0.0, x_prev = 0.0;
  S est[5], ref[5], d[5];
  C m[15], chi2 = (C)0;

  while (true) {
    const bool need = k < 0 && !exhausted;
    const uint32_t want = __ballot_sync(0xffffffffu, need);
    if (want) {
      const int leader = __ffs(want) - 1;
      int base = 0;
      if (lane == leader) base = (int)atomicAdd(P.work + (STAGE >= 2 ? STAGE : 1), (uint32_t)__popc(want));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const int slot = base + __popc(want & lanes_below);
        if (slot >= n_trk) {
          exhausted = true;
        } else {
          const int mine = P.trk_order[slot];
          const int nn = O.n_cl[mine], off = O.offset[mine];
          // ids of overflowing tracks were not written; the tail takes only
          // the tracks the head handed over
          if (nn >= 1 && off >= 0 && off + nn <= O.capacity_ids && (STAGE != 3 || P.rf_j[mine] >= 0)) {
            k = mine;
            n = nn;
            pos = P.trk_pos + off;
            t = P.trk_tl[k];
            if (STAGE == 3) {
#pragma unroll
              for (int i = 0; i < 5; ++i) {
                ref[i] = conv<S>(P.rf_state[(int64_t)i * P.tcap + k]);
                d[i] = conv<S>(P.rf_state[(int64_t)(5 + i) * P.tcap + k]);
              }
#pragma unroll
              for (int i = 0; i < 15; ++i) m[i] = conv<C>(P.rf_state[(int64_t)(10 + i) * P.tcap + k]);
              chi2 = conv<C>(P.rf_state[(int64_t)25 * P.tcap + k]);
              x_prev = P.rf_state[(int64_t)26 * P.tcap + k];
              status = 0;
              j = P.rf_j[k];
            } else if (STAGE == 2) {
#pragma unroll
              for (int i = 0; i < 5; ++i) est[i] = (S)P.trk_est[(int64_t)i * P.tcap + k];
              x_cur = P.trk_x[k];
              status = P.trk_st[k];
            } else {
#pragma unroll
              for (int i = 0; i < 5; ++i) est[i] = (S)P.tl_par[(int64_t)i * P.tcap + t];
              x_cur = P.rx[P.tl_rowref[t]];
              status = 0;
            }
            pass = pass_begin;
            if (STAGE != 3) j = n - 1;
          }
        }
      }
    }
    // a lane whose refill found an unusable track (not exhausted) refills again
    if (__ballot_sync(0xffffffffu, k >= 0 || !exhausted) == 0u) break;
    if (k < 0) continue;

    const int pj = pos[j];
    const int pj_next = j > 0 ? pos[j - 1] : -1;   // the next cluster of this pass, prefetched below
    const double xj = P.rx[P.srow[pj]];
    // One transport per iteration for every lane: at a pass start the
    // reference restarts from the previous estimate at x_cur, otherwise it
    // continues from the previous cluster.  Keeping both cases in one code
    // path issues the FP64 transport once per warp.
    const bool start = j == n - 1;
    if (start) {
#pragma unroll
      for (int i = 0; i < 5; ++i) { ref[i] = est[i]; d[i] = (S)0; }
    }
    Step<E> st;
    if (!helix_step<E>(to_e<E>(ref[2]), to_e<E>(ref[3]), to_e<E>(ref[4]), conv<E>(xj - (start ? x_cur : x_prev)),
                       kb, smax, st)) {
      status = 1;
    } else {
      ref[0] += conv<S>(st.dy); ref[1] += conv<S>(st.dz); ref[2] += conv<S>(st.ds);
      if (start) {
        cov_diag<C>(m, (C)P.c_yz_refit, (C)P.c_yz_refit, (C)P.c_s, (C)P.c_t, (C)P.c_qpt_refit);
        chi2 = (C)0;
      } else {
        d[0] += st.j_ys * d[2] + st.j_yq * d[4];
        d[1] += st.j_zs * d[2] + st.j_zt * d[3] + st.j_zq * d[4];
        d[2] += st.j_sq * d[4];
        cov_transport<C, E>(m, st);
      }
    }
    // the next cluster's position, row and row radius into L1 while this
    // one is filtered (each iteration otherwise waits on two dependent loads)
    if (pj_next >= 0) {
      prefetch_l1(&P.sy[pj_next]);
      prefetch_l1(&P.sz[pj_next]);
      prefetch_l1(&P.srow[pj_next]);
    }
    bool done = status != 0 || pass >= pass_end;
    if (!done) {
      x_prev = xj;
      const C sg = sigma_of<C>(P, conv<C>(P.sz[pj]));
      const C r0 = (conv<C>(P.sy[pj]) - ref[0]) - d[0], r1 = (conv<C>(P.sz[pj]) - ref[1]) - d[1];
      // (the leading passes only move the reference: their chi2 is never read)
      chi2 += refit_update<C, S>(d, m, r0, r1, sg * sg);
      if (STAGE == 2 && j >= 1 && n - j >= kRefitHead) {
        // hand the track over to the double-float tail at cluster j - 1
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          P.rf_state[(int64_t)i * P.tcap + k] = to_double(ref[i]);
          P.rf_state[(int64_t)(5 + i) * P.tcap + k] = to_double(d[i]);
        }
#pragma unroll
        for (int i = 0; i < 15; ++i) P.rf_state[(int64_t)(10 + i) * P.tcap + k] = to_double(m[i]);
        P.rf_state[(int64_t)25 * P.tcap + k] = to_double(chi2);
        P.rf_state[(int64_t)26 * P.tcap + k] = x_prev;
        P.rf_j[k] = j - 1;
        k = -1;
        continue;
      }
      if (--j < 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) est[i] = ref[i] + d[i];
        x_cur = P.rx[P.srow[pos[0]]];
        if (++pass < pass_end) j = n - 1; else done = true;
      }
    }
    if (done && STAGE == 1) {
#pragma unroll
      for (int i = 0; i < 5; ++i) P.trk_est[(int64_t)i * P.tcap + k] = to_double(est[i]);
      P.trk_x[k] = x_cur;
      P.trk_st[k] = status;
      k = -1;
    } else if (done) {
      if (STAGE == 2) P.rf_j[k] = -1;   // finished in the head
      O.status[k] = status;
      O.chi2[k] = status ? 0.0 : to_double(chi2);
      O.x_ref[k] = status ? P.rx[P.tl_rowref[t]] : x_cur;
#pragma unroll
      for (int i = 0; i < 5; ++i)
        O.param[(int64_t)k * 5 + i] = status ? P.tl_par[(int64_t)i * P.tcap + t] : to_double(est[i]);
#pragma unroll
      for (int i = 0; i < 15; ++i) O.cov[(int64_t)k * 15 + i] = status ? 0.0 : to_double(m[i]);
      k = -1;
    }
  }
}

// Refit work order: output tracks by cluster count, longest first (a
// counting sort over kLenClasses classes).  Every track's refit is
// independent, so the order changes no result; longest-first keeps the
// lanes of the persistent refit busy until the queue's end (the last tracks
// taken are the short ones).
__device__ __forceinline__ int refit_track_count(const Params& P) {
  return min((int)(P.tl_sel_scan[P.tcap] >> 32), P.out.capacity_tracks);
}

__global__ void k_order_count(const __grid_constant__ Params P) {
  const int n = refit_track_count(P);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    atomicAdd(&P.len_cnt[min(max(P.out.n_cl[k], 0), kLenClasses - 1)], 1);
}

// one block of kLenClasses threads: cursor[L] = tracks in longer classes
__global__ void __launch_bounds__(kLenClasses) k_order_scan(const __grid_constant__ Params P) {
  __shared__ int sh[kLenClasses];
  const int L = threadIdx.x;
  const int cnt = P.len_cnt[L];
  sh[L] = cnt;
  __syncthreads();
  for (int off = 1; off < kLenClasses; off <<= 1) {
    const int v = L + off < kLenClasses ? sh[L + off] : 0;
    __syncthreads();
    sh[L] += v;
    __syncthreads();
  }
  P.len_cnt[L] = sh[L] - cnt;
}

__global__ void k_order_fill(const __grid_constant__ Params P) {
  const int n = refit_track_count(P);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    P.trk_order[atomicAdd(&P.len_cnt[min(max(P.out.n_cl[k], 0), kLenClasses - 1)], 1)] = k;
}

__global__ void k_export_tracklets(const __grid_constant__ Params P, tpct_debug_out D) {
  const int n_tl = tracklet_count(P);
  const int R = P.n_rows;
  const int lim = min(n_tl, D.capacity_tracklets);
  if (blockIdx.x == 0 && threadIdx.x == 0 && D.n_tracklets) *D.n_tracklets = n_tl;
  if (D.tr_tracklet) {
    const int n_trk = min(min((int)(P.tl_sel_scan[P.tcap] >> 32), P.out.capacity_tracks), D.capacity_tracklets);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_trk; k += gridDim.x * blockDim.x)
      D.tr_tracklet[k] = P.trk_tl[k];
  }
  if (D.counters) {
    long long c0 = 0, c1 = 0, c2 = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tl; t += gridDim.x * blockDim.x) {
      c0 += P.tl_cnt[t];
      c1 += P.tl_cnt[(int64_t)P.tcap + t];
      c2 += P.tl_cnt[2 * (int64_t)P.tcap + t];
    }
    atomicAdd((unsigned long long*)&D.counters[0], (unsigned long long)c0);
    atomicAdd((unsigned long long*)&D.counters[1], (unsigned long long)c1);
    atomicAdd((unsigned long long*)&D.counters[2], (unsigned long long)c2);
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < lim; t += gridDim.x * blockDim.x) {
    const int nh = P.tl_nhits[t];
    if (D.tl_start) D.tl_start[t] = P.sid[P.tl_start[t]];
    if (D.tl_nhits) D.tl_nhits[t] = nh;
    if (D.tl_row_ref) D.tl_row_ref[t] = P.tl_rowref[t];
    if (D.tl_param)
      for (int i = 0; i < 5; ++i) D.tl_param[(int64_t)t * 5 + i] = P.tl_par[(int64_t)i * P.tcap + t];
    if (D.tl_hits) {
      int32_t* h = D.tl_hits + (int64_t)t * R;
      for (int r = 0; r < R; ++r) h[r] = -1;
      for (int j = R - nh; j < R; ++j) {
        const int p = P.tl_hits[hit_at(P, t, j)];
        h[P.srow[p]] = P.sid[p];
      }
    }
  }
}

int blocks_for(int64_t work, int block) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

}  // namespace

void launch_weights(const Params& P, cudaStream_t s) {
  k_weights<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P);
}
void launch_own(const Params& P, cudaStream_t s) {
  k_own<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P);
}
void launch_emit(const Params& P, cudaStream_t s) {
  k_emit<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P);
}
void launch_refit_order(const Params& P, cudaStream_t s) {
  k_order_count<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P);
  k_order_scan<<<1, kLenClasses, 0, s>>>(P);
  k_order_fill<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P);
}
void launch_refit(const Params& P, int mode, int stage, int block, int blocks, cudaStream_t s) {
  if (block <= 0 || block > kMaxBlock) block = 128;
  if (blocks < 1) blocks = 1;
  switch (mode * 4 + stage) {
    case 0: k_refit<0, 0><<<blocks, block, 0, s>>>(P); break;
    case 4: k_refit<1, 0><<<blocks, block, 0, s>>>(P); break;
    case 5: k_refit<1, 1><<<blocks, block, 0, s>>>(P); break;
    case 6: k_refit<1, 2><<<blocks, block, 0, s>>>(P); break;
    case 7: k_refit<1, 3><<<blocks, block, 0, s>>>(P); break;
    case 8: k_refit<2, 0><<<blocks, block, 0, s>>>(P); break;
    case 12: k_refit<3, 0><<<blocks, block, 0, s>>>(P); break;
    case 13: k_refit<3, 1><<<blocks, block, 0, s>>>(P); break;
    case 14: k_refit<3, 2><<<blocks, block, 0, s>>>(P); break;
    case 15: k_refit<3, 3><<<blocks, block, 0, s>>>(P); break;
    default: break;
  }
}

int refit_blocks_per_sm(int mode, int block) {
  int nb = 0;
  cudaError_t e;
  switch (mode) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refit<0, 0>, block, 0); break;
    case 1: {
      int nb1 = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refit<1, 2>, block, 0);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_refit<1, 1>, block, 0);
      if (nb1 < nb) nb = nb1;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_refit<1, 3>, block, 0);
      if (nb1 < nb) nb = nb1;
      break;
    }
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refit<2, 0>, block, 0); break;
    default: {
      int nb1 = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refit<3, 2>, block, 0);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_refit<3, 1>, block, 0);
      if (nb1 < nb) nb = nb1;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_refit<3, 3>, block, 0);
      if (nb1 < nb) nb = nb1;
      break;
    }
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

void launch_export_tracklets(const Params& P, const tpct_debug_out& d, cudaStream_t s) {
  k_export_tracklets<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P, d);
}

}  // namespace tpct
