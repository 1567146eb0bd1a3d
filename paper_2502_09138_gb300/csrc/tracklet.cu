// Step 5 of sector track finding: tracklet growth with a Kalman filter.
// One thread per tracklet (start hit).  Upward pass: follow reciprocal links
// while the previous accepted cluster is in the row below and has one, else
// search the row's grid around the prediction; accept a cluster iff its chi2
// passes; stop on a failed transport, the sector edge, too many consecutive
// misses, or |sin phi| at its limit.  Downward pass: from the outermost
// accepted cluster, covariance reset, to row 0, reusing the upward clusters
// at their rows and searching elsewhere.  (The paper's "TPC Processing
// (Tracking)", Tables 1-3.)
#include "track_math.cuh"

namespace tpct {
namespace {

// Best cluster of row key ir around (py, pz): inside |dy|^2 <= k^2 (Cyy + s_c^2)
// and |dz|^2 <= k^2 (Czz + s_c^2) with s_c the cluster's sigma; minimal
// dy^2/(Cyy+s_c^2) + dz^2/(Czz+s_c^2), ties to the smaller input id.
template <class E, class S, class C>
__device__ int search_row(const Params& P, int ir, S py, S pz, C cyy, C czz) {
  const RowGrid g = P.grid[ir];
  const E k = (E)P.search_k, k2 = k * k;
  const E sig_hi = (E)fmax(P.sig_readout, P.sig_cathode);
  const E wy = k * sqrt((E)cyy + sig_hi * sig_hi), wz = k * sqrt((E)czz + sig_hi * sig_hi);
  const float fy = (float)py, fz = (float)pz;
  const float wyf = (float)wy * 1.0001f + 1e-4f, wzf = (float)wz * 1.0001f + 1e-4f;
  const int iy0 = bin_y(g, fy - wyf), iy1 = bin_y(g, fy + wyf);
  const int iz0 = bin_z(g, fz - wzf), iz1 = bin_z(g, fz + wzf);
  int best = -1, best_id = 0;
  E best_d = (E)0;
  for (int iz = iz0; iz <= iz1; ++iz) {
    const int q0 = P.bin_start[g.bin_base + iz * g.ny + iy0];
    const int q1 = P.bin_start[g.bin_base + iz * g.ny + iy1 + 1];
    for (int q = q0; q < q1; ++q) {
      const float cz = P.sz[q];
      const E dy = (E)((S)P.sy[q] - py), dz = (E)((S)cz - pz);
      const E sg = sigma_of<E>(P, (E)cz);
      const E vy = (E)cyy + sg * sg, vz = (E)czz + sg * sg;
      if (!(dy * dy <= k2 * vy && dz * dz <= k2 * vz)) continue;
      const E d = dy * dy / vy + dz * dz / vz;
      if (best < 0 || d <= best_d) {
        const int id = P.sid[q];
        if (best < 0 || d < best_d || id < best_id) { best = q; best_d = d; best_id = id; }
      }
    }
  }
  return best;
}

template <int MODE>
__global__ void __launch_bounds__(kMaxBlock) k_tracklets(const __grid_constant__ Params P) {
  using S = typename Prec<MODE>::S;
  using E = typename Prec<MODE>::E;
  using C = typename Prec<MODE>::C;
  const int R = P.n_rows;
  const int n_tl = min(P.row_tl_base[P.n_inst * R], P.tcap);
  const E kb = (E)P.kb, smax = (E)P.s_max;
  const C chi2_max = (C)P.chi2_max;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tl; t += gridDim.x * blockDim.x) {
    const int p0 = P.tl_start[t], ir0 = P.tl_ir[t];
    const int r0 = ir0 % R, row0 = ir0 - r0;
    const int h1 = P.upc[p0];
    int* hits = P.tl_hits + t;
    const int64_t ts = P.tcap;

    // init from the first link of the chain: y, z of the start hit, direction of the link
    S p[5];
    C m[15];
    {
      const S dx = (S)(P.rx[r0 + 1] - P.rx[r0]);
      const S dy = (S)P.sy[h1] - (S)P.sy[p0], dz = (S)P.sz[h1] - (S)P.sz[p0];
      const S len = sqrt(dx * dx + dy * dy);
      p[0] = (S)P.sy[p0]; p[1] = (S)P.sz[p0]; p[2] = dy / len; p[3] = dz / len; p[4] = (S)0;
      const C sg = sigma_of<C>(P, (C)P.sz[p0]);
      cov_diag<C>(m, sg * sg, sg * sg, (C)P.c_s, (C)P.c_t, (C)P.c_qpt);
    }
    hits[0] = p0;
    int n_up = 1;
    int n_step = 0, n_upd = 0, n_test = 0;

    // ---- upward
    int prev = p0, prev_row = r0, miss = 0, top_row = r0, top_hit = p0;
    S top[5] = {p[0], p[1], p[2], p[3], p[4]};
    for (int r = r0 + 1; r < R; ++r) {
      Step<E> st;
      if (!helix_step<E>((E)p[2], (E)p[3], (E)p[4], (E)(P.rx[r] - P.rx[r - 1]), kb, smax, st)) break;
      ++n_step;
      p[0] += (S)st.dy; p[1] += (S)st.dz; p[2] += (S)st.ds;
      cov_transport<C, E>(m, st);
      if (fabs(p[0]) > (S)(P.rx[r] * P.tan_half + P.edge_margin)) break;
      int cand = prev_row == r - 1 ? P.upc[prev] : -1;
      if (cand < 0) cand = search_row<E, S, C>(P, row0 + r, p[0], p[1], m[0], m[2]);
      bool ok = false;
      if (cand >= 0) {
        const C sg = sigma_of<C>(P, (C)P.sz[cand]);
        const C v = sg * sg;
        const C ry = (C)((S)P.sy[cand] - p[0]), rz = (C)((S)P.sz[cand] - p[1]);
        ++n_test;
        if (kf_test_update<C, S>(p, m, ry, rz, v, chi2_max)) {
          ++n_upd;
          ok = true;
        }
      }
      if (ok) {
        hits[(int64_t)n_up * ts] = cand;
        ++n_up;
        prev = cand; prev_row = r; miss = 0;
        top_row = r; top_hit = cand;
#pragma unroll
        for (int i = 0; i < 5; ++i) top[i] = p[i];
        if (!(fabs(p[2]) < (S)P.s_max)) break;
      } else if (++miss > P.max_miss) {
        break;
      }
    }

    // ---- downward from the outermost accepted cluster, covariance reset.
    // Final clusters go to slots R-1, R-2, ... (never over an unread upward entry).
#pragma unroll
    for (int i = 0; i < 5; ++i) p[i] = top[i];
    {
      const C sg = sigma_of<C>(P, (C)P.sz[top_hit]);
      cov_diag<C>(m, sg * sg, sg * sg, (C)P.c_s, (C)P.c_t, (C)P.c_qpt);
    }
    int j_up = n_up - 2;
    int n_f = 1;
    hits[(int64_t)(R - 1) * ts] = top_hit;
    int in_row = top_row;
    S in_p[5] = {p[0], p[1], p[2], p[3], p[4]};
    miss = 0;
    for (int r = top_row - 1; r >= 0; --r) {
      Step<E> st;
      if (!helix_step<E>((E)p[2], (E)p[3], (E)p[4], (E)(P.rx[r] - P.rx[r + 1]), kb, smax, st)) break;
      ++n_step;
      p[0] += (S)st.dy; p[1] += (S)st.dz; p[2] += (S)st.ds;
      cov_transport<C, E>(m, st);
      if (fabs(p[0]) > (S)(P.rx[r] * P.tan_half + P.edge_margin)) break;
      int cand = -1;
      if (j_up >= 0) {
        const int h = hits[(int64_t)j_up * ts];
        if ((int)P.srow[h] == r) { cand = h; --j_up; }
      }
      if (cand < 0) cand = search_row<E, S, C>(P, row0 + r, p[0], p[1], m[0], m[2]);
      bool ok = false;
      if (cand >= 0) {
        const C sg = sigma_of<C>(P, (C)P.sz[cand]);
        const C v = sg * sg;
        const C ry = (C)((S)P.sy[cand] - p[0]), rz = (C)((S)P.sz[cand] - p[1]);
        ++n_test;
        if (kf_test_update<C, S>(p, m, ry, rz, v, chi2_max)) {
          ++n_upd;
          ok = true;
        }
      }
      if (ok) {
        hits[(int64_t)(R - 1 - n_f) * ts] = cand;
        ++n_f;
        in_row = r;
        miss = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) in_p[i] = p[i];
        if (!(fabs(p[2]) < (S)P.s_max)) break;
      } else if (++miss > P.max_miss) {
        break;
      }
    }
    P.tl_nhits[t] = n_f;
    P.tl_rowref[t] = in_row;
    P.tl_cnt[t] = n_step;
    P.tl_cnt[ts + t] = n_upd;
    P.tl_cnt[2 * ts + t] = n_test;
#pragma unroll
    for (int i = 0; i < 5; ++i) P.tl_par[(int64_t)i * ts + t] = (double)in_p[i];
  }
}

}  // namespace

void launch_tracklets(const Params& P, int mode, int block, cudaStream_t s) {
  if (block <= 0 || block > kMaxBlock) block = 128;
  int64_t blocks = ((int64_t)P.tcap + block - 1) / block;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (mode == 0) k_tracklets<0><<<(unsigned)blocks, block, 0, s>>>(P);
  else if (mode == 1) k_tracklets<1><<<(unsigned)blocks, block, 0, s>>>(P);
  else k_tracklets<2><<<(unsigned)blocks, block, 0, s>>>(P);
}

}  // namespace tpct
