// Steps 6-7 of sector track finding: selection by owned clusters and shared
// fraction, output compaction, and the iterated refit of every selected
// track.  (The paper's "TPC Processing (Tracking)", Tables 1-3.)
#include "track_math.cuh"

namespace tpct {
namespace {

constexpr int kBlock = 256;

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
    for (int j = R - nh; j < R; ++j) atomicMax(&P.W[P.tl_hits[(int64_t)j * P.tcap + t]], w);
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
      for (int j = R - nh; j < R; ++j) own += P.W[P.tl_hits[(int64_t)j * P.tcap + t]] == w;
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
    int m = 0;
    for (int j = R - nh; j < R; ++j) {
      const int p = P.tl_hits[(int64_t)j * P.tcap + t];
      if (P.W[p] == w) {
        O.cluster_ids[off + m] = P.sid[p];
        P.trk_pos[off + m] = p;
        ++m;
      }
    }
  }
}

// Iterated refit: each pass transports the previous estimate (exact helix) to
// the outermost owned cluster and along all owned clusters inward (the
// reference trajectory), and filters the deviation from it with a diffuse
// prior; reference + deviation at the innermost cluster is the next estimate.
template <int MODE>
__global__ void __launch_bounds__(kMaxBlock) k_refit(const __grid_constant__ Params P) {
  using R = typename Prec<MODE>::R;
  const tpct_tracks_out& O = P.out;
  const uint64_t total = P.tl_sel_scan[P.tcap];
  const int n_trk = min((int)(total >> 32), O.capacity_tracks);
  const R kb = (R)P.kb, smax = (R)P.s_max;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_trk; k += gridDim.x * blockDim.x) {
    const int n = O.n_cl[k], off = O.offset[k];
    if (n < 1 || off < 0 || off + n > O.capacity_ids) continue;
    const int t = P.trk_tl[k];
    const int* pos = P.trk_pos + off;
    R est[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) est[i] = (R)P.tl_par[(int64_t)i * P.tcap + t];
    double x_cur = P.rx[P.tl_rowref[t]];
    R m[15], d[5], ref[5], chi2 = (R)0;
    int status = 0;
    for (int pass = 0; pass < P.n_refit && !status; ++pass) {
#pragma unroll
      for (int i = 0; i < 5; ++i) { ref[i] = est[i]; d[i] = (R)0; }
      int p_prev = pos[n - 1];
      double x_prev = P.rx[P.srow[p_prev]];
      Step<R> st;
      if (!helix_step<R>(ref[2], ref[3], ref[4], (R)(x_prev - x_cur), kb, smax, st)) { status = 1; break; }
      ref[0] += st.dy; ref[1] += st.dz; ref[2] += st.ds;
      cov_diag<R>(m, (R)P.c_yz_refit, (R)P.c_yz_refit, (R)P.c_s, (R)P.c_t, (R)P.c_qpt_refit);
      chi2 = (R)0;
      for (int j = n - 1; j >= 0; --j) {
        const int pj = pos[j];
        const double xj = P.rx[P.srow[pj]];
        if (j < n - 1) {
          if (!helix_step<R>(ref[2], ref[3], ref[4], (R)(xj - x_prev), kb, smax, st)) { status = 1; break; }
          ref[0] += st.dy; ref[1] += st.dz; ref[2] += st.ds;
          d[0] += st.j_ys * d[2] + st.j_yq * d[4];
          d[1] += st.j_zs * d[2] + st.j_zt * d[3] + st.j_zq * d[4];
          d[2] += st.j_sq * d[4];
          cov_transport<R, R>(m, st);
        }
        x_prev = xj;
        const R sg = sigma_of<R>(P, (R)P.sz[pj]);
        const R v = sg * sg;
        const R r0 = ((R)P.sy[pj] - ref[0]) - d[0], r1 = ((R)P.sz[pj] - ref[1]) - d[1];
        chi2 += kf_chi2_update<R, R>(d, m, r0, r1, v);
      }
      if (status) break;
#pragma unroll
      for (int i = 0; i < 5; ++i) est[i] = ref[i] + d[i];
      x_cur = P.rx[P.srow[pos[0]]];
    }
    O.status[k] = status;
    O.chi2[k] = status ? 0.0 : (double)chi2;
    O.x_ref[k] = status ? P.rx[P.tl_rowref[t]] : x_cur;
#pragma unroll
    for (int i = 0; i < 5; ++i) O.param[(int64_t)k * 5 + i] = status ? P.tl_par[(int64_t)i * P.tcap + t] : (double)est[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) O.cov[(int64_t)k * 15 + i] = status ? 0.0 : (double)m[i];
  }
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
        const int p = P.tl_hits[(int64_t)j * P.tcap + t];
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
void launch_refit(const Params& P, int mode, int block, cudaStream_t s) {
  if (block <= 0 || block > kMaxBlock) block = 128;
  // tracks <= tracklets <= tcap; the kernel reads the count on the device
  const int blocks = blocks_for(P.tcap / 4 + 1, block);
  if (mode == 0) k_refit<0><<<blocks, block, 0, s>>>(P);
  else if (mode == 1) k_refit<1><<<blocks, block, 0, s>>>(P);
  else k_refit<2><<<blocks, block, 0, s>>>(P);
}
void launch_export_tracklets(const Params& P, const tpct_debug_out& d, cudaStream_t s) {
  k_export_tracklets<<<blocks_for(P.tcap, kBlock), kBlock, 0, s>>>(P, d);
}

}  // namespace tpct
