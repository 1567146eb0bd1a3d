// Step 5 of sector track finding: tracklet growth with a Kalman filter.
//
// Upward pass: follow reciprocal links while the previous accepted cluster is
// in the row below and has one, else search the row's grid around the
// prediction; accept a cluster iff its chi2 passes; stop on a failed
// transport, the sector edge (plus margin), too many consecutive misses, or
// |sin phi| at its limit.  Downward pass: from the outermost accepted cluster,
// covariance reset, to row 0, reusing the upward clusters at their rows and
// searching elsewhere.  (The paper's "TPC Processing (Tracking)", Tables 1-3.)
//
// GB300 mapping: a persistent kernel in which every lane runs one tracklet as
// a state machine advancing one pad row per loop iteration.  A lane whose
// tracklet ends takes the next one from a device work queue (warp-aggregated
// atomic), so the FP64 (or double-float) covariance arithmetic of each
// iteration runs with full warps instead of idling lanes of finished
// tracklets.  The grid search of the lanes that need one is done by the whole
// warp together (candidates tested one per lane), since per lane its loop
// length varies and left most lanes idle; lanes whose queue ran dry stay in
// the loop as idle lanes, so that every warp stays whole for that search.
// Results do not depend on which lane or order runs a tracklet.
#include "track_math.cuh"

namespace tpct {
namespace {

// Search window of row key ir around (py, pz): inside |dy|^2 <= k^2 (Cyy + s_c^2)
// and |dz|^2 <= k^2 (Czz + s_c^2) with s_c the cluster's sigma, over the grid
// bins [iy0, iy1] x [iz0, iz1] that cover it.
template <class E>
struct SearchWin {
  RowGrid g;
  E ey, ez, cyy, czz, k2;
  int iy0, iy1, iz0, iz1;
};

template <class E, class S>
__device__ __forceinline__ SearchWin<E> search_window(const Params& P, int ir, S py, S pz, E cyy, E czz) {
  SearchWin<E> w;
  w.g = P.grid[ir];
  constexpr bool kF = std::is_same<E, float>::value;
  const E k = kF ? (E)P.search_k_f : (E)P.search_k;
  w.k2 = k * k;
  const E sig_hi = kF ? (E)P.sig_hi_f : (E)fmax(P.sig_readout, P.sig_cathode);
  E wy, wz;
  if constexpr (kF) {
    // the window only selects bins (1e-4 margin below): a root within a few ulp is enough
    const float a = cyy + sig_hi * sig_hi, b = czz + sig_hi * sig_hi;
    wy = k * (a * rsqrtf(a)); wz = k * (b * rsqrtf(b));
  } else {
    wy = k * sqrt(cyy + sig_hi * sig_hi); wz = k * sqrt(czz + sig_hi * sig_hi);
  }
  w.ey = to_e<E>(py);
  w.ez = to_e<E>(pz);
  w.cyy = cyy;
  w.czz = czz;
  const float fy = (float)w.ey, fz = (float)w.ez;
  const float wyf = (float)wy * 1.0001f + 1e-4f, wzf = (float)wz * 1.0001f + 1e-4f;
  w.iy0 = bin_y(w.g, fy - wyf);
  w.iy1 = bin_y(w.g, fy + wyf);
  w.iz0 = bin_z(w.g, fz - wzf);
  w.iz1 = bin_z(w.g, fz + wzf);
  return w;
}

// Cluster q against a window centred at (ey, ez): inside the box, and if so
// its distance d = dy^2/(Cyy+s_c^2) + dz^2/(Czz+s_c^2).
template <class E>
__device__ __forceinline__ bool search_test(const Params& P, int q, E ey, E ez, E cyy, E czz, E k2, E& d) {
  const float cz = P.sz[q];
  const E dy = (E)P.sy[q] - ey, dz = (E)cz - ez;
  const E sg = sigma_of<E>(P, (E)cz);
  const E vy = cyy + sg * sg, vz = czz + sg * sg;
  if (!(dy * dy <= k2 * vy && dz * dz <= k2 * vz)) return false;
  // float d: quotients within 2 ulp (the choice is exact up to that; closer
  // calls are inside the near-cut band of the search's top-2 gap)
  if constexpr (std::is_same<E, float>::value) d = __fdividef(dy * dy, vy) + __fdividef(dz * dz, vz);
  else d = dy * dy / vy + dz * dz / vz;
  return true;
}

// Best cluster of row key ir around (py, pz): minimal d inside the window,
// ties to the smaller input id.  One lane alone.
template <class E, class S>
__device__ int search_row(const Params& P, int ir, S py, S pz, E cyy, E czz) {
  const SearchWin<E> w = search_window<E, S>(P, ir, py, pz, cyy, czz);
  int best = -1, best_id = 0;
  E best_d = (E)0;
  for (int iz = w.iz0; iz <= w.iz1; ++iz) {
    const int q0 = P.bin_start[w.g.bin_base + iz * w.g.ny + w.iy0];
    const int q1 = P.bin_start[w.g.bin_base + iz * w.g.ny + w.iy1 + 1];
    for (int q = q0; q < q1; ++q) {
      E d;
      if (!search_test<E>(P, q, w.ey, w.ez, w.cyy, w.czz, w.k2, d)) continue;
      if (best < 0 || d <= best_d) {
        const int id = P.sid[q];
        if (best < 0 || d < best_d || id < best_id) { best = q; best_d = d; best_id = id; }
      }
    }
  }
  return best;
}

// The same search for all 32 lanes of a warp together (float window
// arithmetic; lanes that do not search take part with no candidates).  A lane's candidates are the clusters of its window's z bins,
// one contiguous range of the sorted copy per z bin; each searching lane
// lists its ranges (up to kSegLane of them) in shared memory, the warp
// concatenates all lanes' candidates by a prefix sum and tests them 32 at a
// time, one per lane, and every searching lane's best is the minimum of the
// key (bits of d, input id) over its candidates, kept with a shared-memory
// atomicMin.  d >= 0, so its bit pattern orders like its value: the key's
// minimum is the per-lane loop's choice (minimal d, ties to the smaller id),
// with the same test and the same arithmetic.  A lane whose window spans more
// z bins searches alone afterwards.
constexpr int kSegLane = 4;
struct SearchShared {
  unsigned long long key[32];   // per searching lane: minimal (d bits, id)
  int best[32];                 // per searching lane: its sorted position
  int start[32];                // first concatenated candidate of each lane
  int q0[32][kSegLane];         // per lane and z bin: first sorted position
  int cum[32][kSegLane];        // per lane and z bin: candidates up to its end
};

__device__ __forceinline__ int search_row_warp(const Params& P, bool need, int ir, float py, float pz, float cyy,
                                               float czz, SearchShared& sh) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  SearchWin<float> w;
  w.ey = py; w.ez = pz; w.cyy = cyy; w.czz = czz; w.k2 = 0.f;
  w.iy0 = w.iy1 = w.iz0 = 0; w.iz1 = -1;
  if (need) w = search_window<float, float>(P, ir, py, pz, cyy, czz);
  const int nseg = w.iz1 - w.iz0 + 1;
  const bool coop = need && nseg <= kSegLane;
  int n_lane = 0;
  if (coop) {
#pragma unroll
    for (int j = 0; j < kSegLane; ++j) {
      if (j < nseg) {
        const int b = w.g.bin_base + (w.iz0 + j) * w.g.ny;
        const int q0 = P.bin_start[b + w.iy0], q1 = P.bin_start[b + w.iy1 + 1];
        sh.q0[lane][j] = q0;
        n_lane += q1 - q0;
      }
      sh.cum[lane][j] = n_lane;
    }
  }
  int incl = n_lane;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(full, incl, d);
    if (lane >= d) incl += v;
  }
  const int total = __shfl_sync(full, incl, 31);
  sh.start[lane] = incl - n_lane;
  sh.key[lane] = ~0ull;
  sh.best[lane] = -1;
  const float k2 = P.search_k_f * P.search_k_f;
  __syncwarp();
  for (int base = 0; base < total; base += 32) {
    const int f = base + lane;
    // owner: the last lane whose first candidate is at or before f
    int owner = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1)
      if (sh.start[owner + s] <= f) owner += s;
    const float oey = __shfl_sync(full, w.ey, owner), oez = __shfl_sync(full, w.ez, owner);
    const float ocyy = __shfl_sync(full, w.cyy, owner), oczz = __shfl_sync(full, w.czz, owner);
    bool hit = false;
    unsigned long long key = 0ull;
    int q = 0;
    if (f < total) {
      const int k = f - sh.start[owner];
      int j = 0, prev = 0;
#pragma unroll
      for (int jj = 0; jj + 1 < kSegLane; ++jj) {
        const int c = sh.cum[owner][jj];
        if (j == jj && k >= c) { j = jj + 1; prev = c; }
      }
      q = sh.q0[owner][j] + (k - prev);
      const unsigned id = (unsigned)P.sid[q];
      float d;
      if (search_test<float>(P, q, oey, oez, ocyy, oczz, k2, d)) {
        key = ((unsigned long long)__float_as_uint(d) << 32) | id;
        atomicMin(&sh.key[owner], key);
        hit = true;
      }
    }
    __syncwarp();
    if (hit && sh.key[owner] == key) sh.best[owner] = q;
    __syncwarp();
  }
  int cand = coop ? sh.best[lane] : -1;
  if (need && !coop) cand = search_row<float, float>(P, ir, py, pz, cyy, czz);
  return cand;
}

// A residual (state type) in the covariance type; a double-float residual
// becomes a double by widening both halves and one addition.
template <class C, class T> __device__ __forceinline__ C to_c(T v) { return (C)v; }
template <> __device__ __forceinline__ double to_c<double, df64>(df64 v) { return to_double(v); }
template <> __device__ __forceinline__ float to_c<float, df64>(df64 v) { return to_float(v); }
template <int MODE>
__global__ void __launch_bounds__(kMaxBlock) k_tracklets(const __grid_constant__ Params P) {
  using S = typename Prec<MODE>::S;
  using E = typename Prec<MODE>::E;
  using C = typename Prec<MODE>::C;
  // float transport with a double covariance: the mixed filter (float chi2
  // decision and state increment, double gain and covariance update)
  constexpr bool kMixed = std::is_same<E, float>::value && std::is_same<C, double>::value;
  const int R = P.n_rows;
  const int n_tl = min(P.row_tl_base[P.n_inst * R], P.tcap);
  const E kb = (E)P.kb, smax = (E)P.s_max;
  const C chi2_max = (C)P.chi2_max;
  const int64_t ts = P.tcap;
  const int lane = threadIdx.x & 31;
  const uint32_t lanes_below = (1u << lane) - 1u;

  // lane state
  int t = -1;                   // current tracklet (-1: none)
  bool exhausted = false;       // the queue had nothing left for this lane
  bool up = true;               // pass
  int r = 0, row0 = 0;          // next row; row key of row 0 of the instance
  int prev = 0, prev_row = 0, miss = 0, top_row = 0, top_hit = 0, n_up = 0, j_up = 0, n_f = 0, in_row = 0;
  int n_step = 0, n_upd = 0, n_test = 0;
  S p[5];
  C m[15];
  // saved states: the outermost accepted state of the upward pass (top) and
  // the innermost of the downward pass (in_p); written at accepted clusters,
  // read at the pass switch and the end.  The mixed filter keeps them in
  // shared memory (one column per thread), which frees registers of its
  // FP64-bound loop; the other modes keep them in registers.
  constexpr bool kSmemState = kMixed;
  S top_r[kSmemState ? 1 : 5], inp_r[kSmemState ? 1 : 5];
  __shared__ S s_top[kSmemState ? 5 : 1][kSmemState ? kMaxBlock : 1], s_inp[kSmemState ? 5 : 1][kSmemState ? kMaxBlock : 1];
  auto top = [&](int i) -> S& {
    if constexpr (kSmemState) return s_top[i][threadIdx.x]; else return top_r[i];
  };
  auto in_p = [&](int i) -> S& {
    if constexpr (kSmemState) return s_inp[i][threadIdx.x]; else return inp_r[i];
  };
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = top(i) = in_p(i) = conv<S>(0.0f);
#pragma unroll
  for (int i = 0; i < 15; ++i) m[i] = conv<C>(0.0f);
  // the tracklet's hit slots: consecutive, or stride tcap (hit_at)
  constexpr bool kByTracklet = hits_by_tracklet_for(MODE);
  const int64_t hs = kByTracklet ? 1 : ts;
  if (P.hits_by_tracklet != (kByTracklet ? 1 : 0)) {   // the host set another layout: refuse
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(P.status, kDevBounds);
    return;
  }
  auto hits = P.tl_hits;
  __shared__ SearchShared s_search[kMaxBlock / 32];

  while (true) {
    // ---- refill lanes without a tracklet from the work queue
    const bool need = t < 0 && !exhausted;
    const uint32_t want = __ballot_sync(0xffffffffu, need);
    if (want) {
      const int leader = __ffs(want) - 1;
      int base = 0;
      if (lane == leader) base = (int)atomicAdd(P.work, (uint32_t)__popc(want));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const int mine = base + __popc(want & lanes_below);
        if (mine < n_tl) {
          t = mine;
          // init from the first link of the chain
          const int p0 = P.tl_start[t], ir0 = P.tl_ir[t];
          const int r0 = ir0 % R;
          row0 = ir0 - r0;
          const int h1 = P.upc[p0];
          // direction of the first link in float (like all transport arithmetic)
          const float dx = P.rdxf[r0 + 1];
          const float dy = P.sy[h1] - P.sy[p0], dz = P.sz[h1] - P.sz[p0];
          const float il = rsqrtf(dx * dx + dy * dy);
          p[0] = conv<S>(P.sy[p0]); p[1] = conv<S>(P.sz[p0]); p[2] = conv<S>(dy * il); p[3] = conv<S>(dz * il);
          p[4] = conv<S>(0.0f);
          const C v0 = conv<C>(cluster_var(P, P.sz[p0]));
          cov_diag<C>(m, v0, v0, (C)P.c_s, (C)P.c_t, (C)P.c_qpt);
          hits = P.tl_hits + (kByTracklet ? (int64_t)t * R : (int64_t)t);
          hits[0] = p0;
          n_up = 1;
          prev = p0; prev_row = r0; miss = 0; top_row = r0; top_hit = p0;
#pragma unroll
          for (int i = 0; i < 5; ++i) top(i) = p[i];
          n_step = n_upd = n_test = 0;
          up = true;
          r = r0 + 1;
        } else {
          exhausted = true;
        }
      }
    }
    const uint32_t active = __ballot_sync(0xffffffffu, t >= 0);
    if (active == 0u) break;
    const bool live = t >= 0;   // lanes whose queue ran dry stay in the loop, idle, so that warps stay full
    __syncwarp();

    // ---- one row of the current pass.  Every lane with a tracklet runs the
    // same straight-line sequence (transport, candidate, test/update); the
    // __syncwarp calls rejoin the lanes after the divergent candidate search so
    // that the covariance arithmetic issues once per warp.
    bool go = true;   // pass continues after this row
    Step<E> st;
    const E dx = !live ? (E)0 : up ? row_dx<E>(P, r) : -row_dx<E>(P, r + 1);
    const bool stepped = live && helix_step<E>(to_e<E>(p[2]), to_e<E>(p[3]), to_e<E>(p[4]), dx, kb, smax, st);
    if (stepped) {
      ++n_step;
      p[0] += conv<S>(st.dy); p[1] += conv<S>(st.dz); p[2] += conv<S>(st.ds);
      cov_transport<C, E>(m, st);
    }
    // the edge and sin(phi) limits are compared in the transport precision
    const bool inside = stepped && !abs_exceeds(to_e<E>(p[0]), EdgeOf<E>::get(P, r));
    go = inside;
    int cand = -1;
    bool srch = false;   // this lane searches the row's grid
    if (inside) {
      if (up) {
        if (prev_row == r - 1) cand = P.upc[prev];
      } else if (j_up >= 0) {
        const int h = hits[(int64_t)j_up * hs];
        if ((int)P.srow[h] == r) { cand = h; --j_up; }
      }
      srch = cand < 0;
    }
    if constexpr (std::is_same<E, float>::value) {
      // every lane of the warp is here (idle lanes included): the whole warp searches
      const int c = search_row_warp(P, srch, row0 + r, to_e<E>(p[0]), to_e<E>(p[1]), to_e<E>(m[0]),
                                    to_e<E>(m[2]), s_search[threadIdx.x >> 5]);
      if (srch) cand = c;
      srch = false;
    }
    if (srch) cand = search_row<E, S>(P, row0 + r, p[0], p[1], to_e<E>(m[0]), to_e<E>(m[2]));
    __syncwarp();
    bool ok = false;
    if (cand >= 0) {
      ++n_test;
      bool pass;
      if constexpr (kMixed) {
        // the mixed filter uses the residuals only in float (chi2 decision,
        // state increment): rounded once from the state's difference
        const float fry = to_float(conv<S>(P.sy[cand]) - p[0]), frz = to_float(conv<S>(P.sz[cand]) - p[1]);
        pass = kf_test_update_mixed(p, m, fry, frz, cluster_var(P, P.sz[cand]), P.chi2_max_f);
      } else {
        const C ry = to_c<C>(conv<S>(P.sy[cand]) - p[0]), rz = to_c<C>(conv<S>(P.sz[cand]) - p[1]);
        pass = kf_test_update<C, S>(p, m, ry, rz, conv<C>(cluster_var(P, P.sz[cand])), chi2_max);
      }
      if (pass) { ++n_upd; ok = true; }
    }
    __syncwarp();
    if (inside) {
      {
        if (ok) {
          miss = 0;
          if (up) {
            hits[(int64_t)n_up * hs] = cand;
            ++n_up;
            prev = cand; prev_row = r; top_row = r; top_hit = cand;
#pragma unroll
            for (int i = 0; i < 5; ++i) top(i) = p[i];
          } else {
            hits[(int64_t)(R - 1 - n_f) * hs] = cand;
            ++n_f;
            in_row = r;
#pragma unroll
            for (int i = 0; i < 5; ++i) in_p(i) = p[i];
          }
          if (!abs_below(to_e<E>(p[2]), SmaxOf<E>::get(P))) go = false;
        } else if (++miss > P.max_miss) {
          go = false;
        }
      }
    }
    if (go) {
      r += up ? 1 : -1;
      go = up ? r < R : r >= 0;
    }
    if (live && !go && up) {
      // switch to the downward pass from the outermost accepted cluster.
      // Final clusters go to slots R-1, R-2, ... (never over an unread upward entry).
      up = false;
#pragma unroll
      for (int i = 0; i < 5; ++i) { p[i] = top(i); in_p(i) = top(i); }
      const C v0 = conv<C>(cluster_var(P, P.sz[top_hit]));
      cov_diag<C>(m, v0, v0, (C)P.c_s, (C)P.c_t, (C)P.c_qpt);
      j_up = n_up - 2;
      n_f = 1;
      hits[(int64_t)(R - 1) * hs] = top_hit;
      in_row = top_row;
      miss = 0;
      r = top_row - 1;
      go = r >= 0;
    }
    if (live && !go) {
      P.tl_nhits[t] = n_f;
      P.tl_rowref[t] = in_row;
      P.tl_cnt[t] = n_step;
      P.tl_cnt[ts + t] = n_upd;
      P.tl_cnt[2 * ts + t] = n_test;
#pragma unroll
      for (int i = 0; i < 5; ++i) P.tl_par[(int64_t)i * ts + t] = to_double(in_p(i));
      t = -1;
    }
  }
}

}  // namespace

void launch_tracklets(const Params& P, int mode, int block, int blocks, cudaStream_t s) {
  if (block <= 0 || block > kMaxBlock) block = 128;
  if (blocks < 1) blocks = 1;
  switch (mode) {
    case 0: k_tracklets<0><<<blocks, block, 0, s>>>(P); break;
    case 1: k_tracklets<1><<<blocks, block, 0, s>>>(P); break;
    case 2: k_tracklets<2><<<blocks, block, 0, s>>>(P); break;
    default: k_tracklets<3><<<blocks, block, 0, s>>>(P); break;
  }
}

int tracklet_blocks_per_sm(int mode, int block) {
  int n = 0;
  cudaError_t e;
  switch (mode) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tracklets<0>, block, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tracklets<1>, block, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tracklets<2>, block, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tracklets<3>, block, 0); break;
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace tpct
