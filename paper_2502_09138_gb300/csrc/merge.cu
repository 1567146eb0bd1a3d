// Cross-sector merging of sector tracks and the refit of merged chains.
//
// A particle crossing a sector boundary leaves one track in each sector
// ("TPC Processing (Tracking)", Tables 1-3 of the paper, counts the whole
// tracking; merging joins what sector tracking splits).  For tracks a, b in
// adjacent sectors of the same side and collision, the inner one I has the
// smaller radius of its reference point (ties: smaller index).  A pair is
// tested iff |tanl_I - tanl_O| <= max_dtanl and I's outermost and O's
// innermost owned clusters are at most max_gap apart in the transverse plane;
// then I's refit state is transported to its outermost cluster, rotated into
// O's frame and transported to O's reference x, and chi2 = dp^T (C_I + C_O)^-1 dp.
// Accepted pairs (chi2 <= chi2_max) compete: every track keeps its best outer
// and best inner partner (smallest chi2, ties to the smaller index) and
// mutual best pairs are linked.  Linked tracks form chains, refitted together
// in FP64 with the reference rotated at every change of sector.
#include "refit_update.cuh"

namespace tpct {
namespace {

constexpr int kBlock = 256;

// A hint to bring the line holding a (a valid address) into L1.
__device__ __forceinline__ void prefetch_l1(const void* a) { asm volatile("prefetch.global.L1 [%0];" :: "l"(a)); }
constexpr int kLenBins = 1024;   // chain-length classes of the refit order (longer chains share the top one)

struct MParams {
  const double* rx;
  int n_rows, n_inst, n_events, n_cap_tracks;
  int32_t cap_pairs, cap_cand;
  double kb, s_max, chi2_max, max_dtanl, max_gap, alpha0, dalpha;
  double c_s, c_t, c_yz_refit, c_qpt_refit, sig_readout, sig_slope, z_max;
  float sig_readout_f, sig_slope_f, z_max_f;
  int n_refit;
  // inputs
  const float *x, *y, *z;
  const uint8_t* row;
  const int32_t *inst_sector, *inst_event;
  tpct_tracks_out trk;
  // workspace
  uint32_t* status;
  int32_t* inst_of;           // [n_events * 36]
  int32_t *first, *last;      // [n_inst] track range of each instance
  double *alpha, *rref, *xout, *inx, *iny, *outx, *outy;   // [cap tracks]
  float4* fq;                  // [cap tracks] float copies for the prefilter: tan lambda, outx, outy, inx
  float* fiy;                  // [cap tracks] iny
  uint64_t *best_out_chi, *best_in_chi;                      // [cap tracks] order-preserving chi2 bits
  int32_t *best_out, *best_in;                               // [cap tracks]
  int32_t* n_cand;                                           // [1]
  int32_t *cand_i, *cand_o;                                  // [cap_cand] prefiltered pairs (inner, outer)
  int32_t* n_pairs;                                          // [1]
  int32_t* pair_i;                                           // [cap_pairs] inner, outer
  int32_t* pair_o;
  double* pair_chi;
  int32_t *head_flag, *head_idx, *nseg, *segoff, *ncl, *cloff;   // [cap tracks + 1] per head
  int32_t* len_cursor;                                       // [kLenBins] chains per length, then cursors
  int32_t* ch_order;                                         // [cap tracks] chains, longest first
  double *ch_est, *ch_ref, *ch_x;                            // [5 cap], [5 cap], [cap] after the leading passes
  int32_t* ch_st;                                            // [cap]
  uint64_t* scan_tmp;
  tpct_chains_out out;
};

__device__ __forceinline__ int nearest_row_m(const MParams& M, float xc) {
  const double x = (double)xc;
  int lo = 0, hi = M.n_rows - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (M.rx[mid] < x) lo = mid + 1; else hi = mid;
  }
  if (lo > 0 && fabs(x - M.rx[lo - 1]) <= fabs(x - M.rx[lo])) lo = lo - 1;
  return lo;
}
__device__ __forceinline__ int row_of(const MParams& M, int id) {
  return M.row ? (int)M.row[id] : nearest_row_m(M, M.x[id]);
}
__device__ __forceinline__ int track_count(const MParams& M) {
  return min(*M.trk.n_tracks, M.trk.capacity_tracks);
}
__device__ __forceinline__ double wrap_pi(double a) {
  const double tp = 6.283185307179586;
  while (a > 3.141592653589793) a -= tp;
  while (a <= -3.141592653589793) a += tp;
  return a;
}

// Rotation of the sector frame by d (new alpha - old alpha).  Position and
// direction rotate exactly; a perturbation of y at fixed x slides back onto
// the new plane along the track (dl = -sin d dy / cos phi'), which scales y by
// cos phi / cos phi', moves z by -t sin d / cos phi' and turns the direction
// by rho dl; a change of sin phi at a fixed point changes sin phi' by
// cos phi' / cos phi.
struct Rot {
  double jyy, jzy, jsy, jss;
};
__device__ __forceinline__ bool rotate_state(double d, double kb, double smax, double x0, double* p, double* x1,
                                             Rot* J) {
  double sd, cd;
  sincos(d, &sd, &cd);
  const double s = p[2];
  if (!(fabs(s) < 1.0)) return false;
  const double c = sqrt(1.0 - s * s);
  const double s1 = s * cd - c * sd, c1 = c * cd + s * sd;
  if (!(c1 > 0.0) || !(fabs(s1) < smax)) return false;
  *x1 = x0 * cd + p[0] * sd;
  const double y1 = -x0 * sd + p[0] * cd;
  if (J) {
    const double rho = -kb * p[4];
    J->jyy = c / c1;
    J->jzy = -p[3] * sd / c1;
    J->jsy = -rho * sd;
    J->jss = c1 / c;
  }
  p[0] = y1;
  p[2] = s1;
  return true;
}

// C <- J C J^T for the rotation Jacobian (rows y, z, s change).
__device__ __forceinline__ void cov_rotate(double* m, const Rot& J) {
  // full symmetric 5x5 from the packed lower triangle
  double C[5][5];
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++idx) C[i][j] = C[j][i] = m[idx];
  double A[5][5];   // J C
  for (int j = 0; j < 5; ++j) {
    A[0][j] = J.jyy * C[0][j];
    A[1][j] = J.jzy * C[0][j] + C[1][j];
    A[2][j] = J.jsy * C[0][j] + J.jss * C[2][j];
    A[3][j] = C[3][j];
    A[4][j] = C[4][j];
  }
  double B[5][5];   // (J C) J^T
  for (int i = 0; i < 5; ++i) {
    B[i][0] = A[i][0] * J.jyy;
    B[i][1] = A[i][0] * J.jzy + A[i][1];
    B[i][2] = A[i][0] * J.jsy + A[i][2] * J.jss;
    B[i][3] = A[i][3];
    B[i][4] = A[i][4];
  }
  idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++idx) m[idx] = B[i][j];
}

// chi2 = dp^T S^-1 dp for symmetric positive S (packed), by Cholesky.
__device__ __forceinline__ bool chi2_packed(const double* S, const double* dp, double* chi2) {
  double L[15];
  int idx = 0;
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j <= i; ++j, ++idx) {
      double sum = S[idx];
      for (int k = 0; k < j; ++k) sum -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      if (i == j) {
        if (!(sum > 0.0)) return false;
        L[idx] = sqrt(sum);
      } else {
        L[idx] = sum / L[j * (j + 1) / 2 + j];
      }
    }
  }
  double w[5];
  double q = 0.0;
  for (int i = 0; i < 5; ++i) {
    double sum = dp[i];
    for (int k = 0; k < i; ++k) sum -= L[i * (i + 1) / 2 + k] * w[k];
    w[i] = sum / L[i * (i + 1) / 2 + i];
    q += w[i] * w[i];
  }
  *chi2 = q;
  return true;
}

__device__ __forceinline__ void load_track(const MParams& M, int k, double* p, double* C) {
  for (int i = 0; i < 5; ++i) p[i] = M.trk.param[(int64_t)k * 5 + i];
  for (int i = 0; i < 15; ++i) C[i] = M.trk.cov[(int64_t)k * 15 + i];
}

__device__ __forceinline__ bool transport(const MParams& M, double x0, double x1, double* p, double* C) {
  Step<double> st;
  if (!helix_step<double>(p[2], p[3], p[4], x1 - x0, M.kb, M.s_max, st)) return false;
  p[0] += st.dy; p[1] += st.dz; p[2] += st.ds;
  if (C) cov_transport<double, double>(C, st);
  return true;
}

// ------------------------------------------------------------------ kernels
struct RowTab {
  double x[kMaxRows];
};
__global__ void k_m_rows(double* rx, int n, const RowTab tab) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) rx[i] = tab.x[i];
}

__global__ void k_m_init(const __grid_constant__ MParams M) {
  const int nt = M.n_cap_tracks;
  const int ni = M.n_events * 36;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(max(max(nt, ni), M.n_inst), kLenBins) + 1;
       i += gridDim.x * blockDim.x) {
    if (i < ni) M.inst_of[i] = -1;
    if (i < M.n_inst) { M.first[i] = 0; M.last[i] = 0; }
    if (i < nt) {
      M.best_out_chi[i] = ~0ull; M.best_in_chi[i] = ~0ull;
      M.best_out[i] = 0x7fffffff; M.best_in[i] = 0x7fffffff;
      M.head_flag[i] = 0; M.nseg[i] = 0; M.ncl[i] = 0;
    }
    if (i < kLenBins) M.len_cursor[i] = 0;
    if (i == 0) { *M.n_pairs = 0; *M.n_cand = 0; }
  }
}

__global__ void k_m_prep(const __grid_constant__ MParams M) {
  const int n = track_count(M);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.n_inst; i += gridDim.x * blockDim.x) {
    const int s = M.inst_sector[i], e = M.inst_event[i];
    if (s >= 0 && s < 36 && e >= 0 && e < M.n_events) M.inst_of[e * 36 + s] = i;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int inst = M.trk.instance[k];
    if (k == 0 || M.trk.instance[k - 1] != inst) M.first[inst] = k;
    if (k == n - 1 || M.trk.instance[k + 1] != inst) M.last[inst] = k + 1;
    const double al = M.alpha0 + (double)(M.inst_sector[inst] % 18) * M.dalpha;
    M.alpha[k] = al;
    const double xr = M.trk.x_ref[k], yr = M.trk.param[(int64_t)k * 5];
    M.rref[k] = sqrt(xr * xr + yr * yr);
    const int off = M.trk.offset[k], ncl = M.trk.n_cl[k];
    const int a = M.trk.cluster_ids[off], b = M.trk.cluster_ids[off + ncl - 1];
    double sa, ca;
    sincos(al, &sa, &ca);
    const double xa = M.rx[row_of(M, a)], xb = M.rx[row_of(M, b)];
    const double ya = (double)M.y[a], yb = (double)M.y[b];
    M.inx[k] = xa * ca - ya * sa; M.iny[k] = xa * sa + ya * ca;
    M.outx[k] = xb * ca - yb * sa; M.outy[k] = xb * sa + yb * ca;
    M.xout[k] = xb;
    M.fq[k] = make_float4((float)M.trk.param[(int64_t)k * 5 + 3], (float)M.outx[k], (float)M.outy[k], (float)M.inx[k]);
    M.fiy[k] = (float)M.iny[k];
  }
}

// Prefilter of all track pairs across one sector boundary, one block per
// (collision, side, sector k | k+1).  The few pairs that pass are compacted
// (warp ballot, one atomic per warp) into a candidate list, so that the FP64
// pair chi2 below runs with full warps instead of a few lanes of each.
__global__ void k_m_cand(const __grid_constant__ MParams M) {
  const int b = blockIdx.x;
  const int e = b / 36, side = (b / 18) % 2, kk = b % 18;
  if (e >= M.n_events) return;
  const int ia = M.inst_of[e * 36 + side * 18 + kk];
  const int ib = M.inst_of[e * 36 + side * 18 + (kk + 1) % 18];
  if (ia < 0 || ib < 0) return;
  const int a0 = M.first[ia], na = M.last[ia] - a0;
  const int b0 = M.first[ib], nb = M.last[ib] - b0;
  if (na <= 0 || nb <= 0) return;
  if ((int64_t)na * nb > 0x7fffffffll) {   // beyond the 32-bit pair index: reported, boundary skipped
    if (threadIdx.x == 0) atomicOr(M.status, kDevCapacity);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)na * nb;
  // every thread runs the same number of rounds, so whole warps reach the ballot
  for (int64_t q0 = 0; q0 < total; q0 += blockDim.x) {
    const int64_t q = q0 + threadIdx.x;
    bool pass = false;
    int I = 0, O = 0;
    if (q < total) {
      const int qi = (int)q;                       // na * nb < 2^31 (checked on entry)
      const int a = a0 + qi / nb, bb = b0 + qi % nb;
      // float pre-test: rejects only pairs outside both cuts by far more than
      // float rounding (either track inner); the rest take the FP64 test
      const float4 fa = M.fq[a], fb = M.fq[bb];
      const float fya = M.fiy[a], fyb = M.fiy[bb];
      const float gab_x = fa.y - fb.w, gab_y = fa.z - fyb;   // a inner
      const float gba_x = fb.y - fa.w, gba_y = fb.z - fya;   // b inner
      const float gcut = (float)M.max_gap + 1e-3f;
      const bool far = fabsf(fa.x - fb.x) > (float)M.max_dtanl * (1.f + 1e-5f) + 1e-6f ||
                       (gab_x * gab_x + gab_y * gab_y > gcut * gcut && gba_x * gba_x + gba_y * gba_y > gcut * gcut);
      if (!far && !M.trk.status[a] && !M.trk.status[bb]) {
        I = a; O = bb;
        if (M.rref[bb] < M.rref[a] || (M.rref[bb] == M.rref[a] && bb < a)) { I = bb; O = a; }
        const double dt = fabs(M.trk.param[(int64_t)I * 5 + 3] - M.trk.param[(int64_t)O * 5 + 3]);
        const double gx = M.outx[I] - M.inx[O], gy = M.outy[I] - M.iny[O];
        pass = dt <= M.max_dtanl && sqrt(gx * gx + gy * gy) <= M.max_gap;
      }
    }
    const uint32_t ball = __ballot_sync(0xffffffffu, pass);
    if (ball) {
      const int leader = __ffs(ball) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(M.n_cand, __popc(ball));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (pass) {
        const int slot = base + __popc(ball & ((1u << lane) - 1u));
        if (slot < M.cap_cand) { M.cand_i[slot] = I; M.cand_o[slot] = O; }
        else atomicOr(M.status, kDevCapacity);
      }
    }
  }
}

// Pair chi2 of every candidate (one thread each): I's refit state transported
// to its outermost cluster, rotated into O's frame, transported to O's
// reference x and compared with O's state.  The candidate order does not
// matter: the best partners come from order-independent atomic minima.
__global__ void k_m_chi(const __grid_constant__ MParams M) {
  const int nc = min(*M.n_cand, M.cap_cand);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    const int I = M.cand_i[q], O = M.cand_o[q];
    double p[5], C[15];
    load_track(M, I, p, C);
    if (!transport(M, M.trk.x_ref[I], M.xout[I], p, C)) continue;
    double x1;
    Rot J;
    if (!rotate_state(wrap_pi(M.alpha[O] - M.alpha[I]), M.kb, M.s_max, M.xout[I], p, &x1, &J)) continue;
    cov_rotate(C, J);
    if (!transport(M, x1, M.trk.x_ref[O], p, C)) continue;
    double dp[5], S[15];
    for (int i = 0; i < 5; ++i) dp[i] = p[i] - M.trk.param[(int64_t)O * 5 + i];
    for (int i = 0; i < 15; ++i) S[i] = C[i] + M.trk.cov[(int64_t)O * 15 + i];
    double chi2;
    if (!chi2_packed(S, dp, &chi2) || !(chi2 <= M.chi2_max)) continue;
    const int slot = atomicAdd(M.n_pairs, 1);
    if (slot >= M.cap_pairs) { atomicOr(M.status, kDevCapacity); continue; }
    M.pair_i[slot] = I; M.pair_o[slot] = O; M.pair_chi[slot] = chi2;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(chi2);   // chi2 >= 0: bits order like values
    atomicMin((unsigned long long*)&M.best_out_chi[I], bits);
    atomicMin((unsigned long long*)&M.best_in_chi[O], bits);
  }
}

__global__ void k_m_best(const __grid_constant__ MParams M) {
  const int np = min(*M.n_pairs, M.cap_pairs);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
    const int I = M.pair_i[q], O = M.pair_o[q];
    const uint64_t bits = (uint64_t)__double_as_longlong(M.pair_chi[q]);
    if (bits == M.best_out_chi[I]) atomicMin(&M.best_out[I], O);
    if (bits == M.best_in_chi[O]) atomicMin(&M.best_in[O], I);
  }
}

// links, chain heads (no inner link, an outer link), segments and clusters per chain
__global__ void k_m_links(const __grid_constant__ MParams M) {
  const int n = track_count(M);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int o = M.best_out[k], i = M.best_in[k];
    const int lo = (o != 0x7fffffff && M.best_in[o] == k) ? o : -1;
    const int li = (i != 0x7fffffff && M.best_out[i] == k) ? i : -1;
    if (M.out.link_out) M.out.link_out[k] = lo;
    if (M.out.link_in) M.out.link_in[k] = li;
  }
}

__device__ __forceinline__ int link_out_of(const MParams& M, int k) {
  const int o = M.best_out[k];
  return (o != 0x7fffffff && M.best_in[o] == k) ? o : -1;
}
__device__ __forceinline__ int link_in_of(const MParams& M, int k) {
  const int i = M.best_in[k];
  return (i != 0x7fffffff && M.best_out[i] == k) ? i : -1;
}

__global__ void k_m_heads(const __grid_constant__ MParams M) {
  const int n = track_count(M);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M.n_cap_tracks; k += gridDim.x * blockDim.x) {
    int flag = 0, segs = 0, cls = 0;
    if (k < n && link_in_of(M, k) < 0 && link_out_of(M, k) >= 0) {
      flag = 1;
      for (int s = k; s >= 0 && segs < 64; s = link_out_of(M, s)) { ++segs; cls += M.trk.n_cl[s]; }
    }
    M.head_flag[k] = flag;
    M.nseg[k] = segs;
    M.ncl[k] = cls;
  }
}

__global__ void k_m_emit(const __grid_constant__ MParams M) {
  const int n = track_count(M);
  const tpct_chains_out& O = M.out;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int nc = M.head_idx[M.n_cap_tracks], ni = M.cloff[M.n_cap_tracks], ns = M.segoff[M.n_cap_tracks];
    *O.n_chains = nc;
    *O.n_ids = ni;
    *O.n_segs = ns;
    if (nc > O.capacity_chains || ni > O.capacity_ids || ns > O.capacity_segs) atomicOr(M.status, kDevCapacity);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (!M.head_flag[k]) continue;
    const int c = M.head_idx[k], off = M.cloff[k], so = M.segoff[k];
    if (c >= O.capacity_chains) continue;
    O.head[c] = k;
    O.n_seg[c] = M.nseg[k];
    O.seg_offset[c] = so;
    O.n_cl[c] = M.ncl[k];
    O.offset[c] = off;
    O.ndf[c] = 2 * M.ncl[k] - 5;
    O.instance[c] = M.trk.instance[k];
    if (off + M.ncl[k] > O.capacity_ids || so + M.nseg[k] > O.capacity_segs) continue;
    int q = off, j = so;
    for (int s = k; s >= 0 && j < so + M.nseg[k]; s = link_out_of(M, s)) {
      O.segs[j++] = s;
      const int to = M.trk.offset[s];
      for (int i = 0; i < M.trk.n_cl[s]; ++i) O.cluster_ids[q++] = M.trk.cluster_ids[to + i];
    }
  }
}

// Chain lengths, longest first: a counting sort on min(n_cl, kLenBins - 1)
// so that consecutive threads of the chain refit take chains of similar
// length and the lanes of a warp finish together.  Each chain's refit is
// independent, so the order changes no result.
__global__ void k_m_len_count(const __grid_constant__ MParams M) {
  const tpct_chains_out& O = M.out;
  const int nc = min(M.head_idx[M.n_cap_tracks], O.capacity_chains);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    atomicAdd(&M.len_cursor[min(O.n_cl[c], kLenBins - 1)], 1);
}

// one block of kLenBins threads: cursor[L] = number of chains in longer classes
__global__ void __launch_bounds__(kLenBins) k_m_len_scan(const __grid_constant__ MParams M) {
  __shared__ int sh[kLenBins];
  const int L = threadIdx.x;
  const int cnt = M.len_cursor[L];
  sh[L] = cnt;
  __syncthreads();
  for (int off = 1; off < kLenBins; off <<= 1) {   // inclusive suffix sums
    const int v = L + off < kLenBins ? sh[L + off] : 0;
    __syncthreads();
    sh[L] += v;
    __syncthreads();
  }
  M.len_cursor[L] = sh[L] - cnt;
}

__global__ void k_m_len_scatter(const __grid_constant__ MParams M) {
  const tpct_chains_out& O = M.out;
  const int nc = min(M.head_idx[M.n_cap_tracks], O.capacity_chains);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    M.ch_order[atomicAdd(&M.len_cursor[min(O.n_cl[c], kLenBins - 1)], 1)] = c;
}

// Rotation Jacobian entry times a deviation or covariance entry, in the
// precision of the latter (float entries for double-float).
__device__ __forceinline__ double mulj(double j, double v) { return j * v; }
__device__ __forceinline__ df64 mulj(double j, df64 v) { return v * narrow(j); }

// C <- J C J^T for a double-float covariance (packed lower triangle; rows
// y, z, s of J differ from the identity: y' = jyy y, z' = jzy y + z,
// s' = jsy y + jss s).
__device__ __forceinline__ void cov_rotate(df64* m, const Rot& J) {
  const df64 a10 = mulj(J.jzy, m[0]) + m[1];                    // (J C)_10
  const df64 a20 = mulj(J.jsy, m[0]) + mulj(J.jss, m[3]);       // (J C)_20
  const df64 a21 = mulj(J.jsy, m[1]) + mulj(J.jss, m[4]);       // (J C)_21
  const df64 a22 = mulj(J.jsy, m[3]) + mulj(J.jss, m[5]);       // (J C)_22
  const df64 a11 = mulj(J.jzy, m[1]) + m[2];                    // (J C)_11
  const df64 c00 = mulj(J.jyy, mulj(J.jyy, m[0]));
  const df64 c10 = mulj(J.jyy, a10);
  const df64 c11 = mulj(J.jzy, a10) + a11;
  const df64 c20 = mulj(J.jyy, a20);
  const df64 c21 = mulj(J.jzy, a20) + a21;
  const df64 c22 = mulj(J.jsy, a20) + mulj(J.jss, a22);
  const df64 m30 = m[6], m40 = m[10];
  m[0] = c00; m[1] = c10; m[2] = c11; m[3] = c20; m[4] = c21; m[5] = c22;
  m[6] = mulj(J.jyy, m30);
  m[7] = mulj(J.jzy, m30) + m[7];
  m[8] = mulj(J.jsy, m30) + mulj(J.jss, m[8]);
  m[10] = mulj(J.jyy, m40);
  m[11] = mulj(J.jzy, m40) + m[11];
  m[12] = mulj(J.jsy, m40) + mulj(J.jss, m[12]);
}

// Chain refit: reference-trajectory Kalman filter over all clusters of the
// chain, outermost to innermost, n_refit passes; pass 0 takes its reference
// from the outermost segment's own fit carried to its outermost cluster;
// later passes carry the previous estimate outward through the chain (kept
// from the previous pass if that carry fails).  As in the sector refit, the
// passes before the last only move the linearisation point (an error e there
// moves the result by O(e^2)): STAGE 1 runs them in double-float with float
// transport and stores the estimate; STAGE 2 runs the last pass, which gives
// the parameters, covariance and chi2, in double.  One thread per chain, in
// the longest-first order.
// Kalman filter of clusters k_hi down to k_lo of a chain of n clusters (a
// pass runs from the outermost cluster inward; the first has no transport) in state type S, transport type E and
// covariance type C, rotating the state at every change of sector; the
// reference, deviation, covariance, chi2, x of the previous cluster and the
// current segment carry over between spans.
template <class S, class E, class C, bool kChi2 = true>
__device__ __forceinline__ void chain_span(const MParams& M, const int* ids, const int* segs, int n, int k_hi,
                                           int k_lo, S* ref, S* d, C* Cm, C& chi2, double& x_prev, int& seg,
                                           int& seg_start, int& status) {
  for (int k = k_hi; k >= k_lo && !status; --k) {
    const int id = ids[k];
    const int id_next = k > k_lo ? ids[k - 1] : -1;   // the next cluster, prefetched after the transport
    const double xk = M.rx[row_of(M, id)];
    if (k < n - 1) {
      if (k < seg_start) {   // the cluster lies in the previous (inner) segment: rotate
        const int from = segs[seg];
        --seg;
        seg_start -= M.trk.n_cl[segs[seg]];
        double x1, rd[5];
        Rot J;
        for (int i = 0; i < 5; ++i) rd[i] = to_double(ref[i]);
        if (!rotate_state(wrap_pi(M.alpha[segs[seg]] - M.alpha[from]), M.kb, M.s_max, x_prev, rd, &x1, &J)) {
          status = 1;
          return;
        }
        for (int i = 0; i < 5; ++i) ref[i] = conv<S>(rd[i]);
        const S d0 = d[0];
        d[0] = mulj(J.jyy, d0);
        d[1] = mulj(J.jzy, d0) + d[1];
        d[2] = mulj(J.jsy, d0) + mulj(J.jss, d[2]);
        cov_rotate(Cm, J);
        x_prev = x1;
      }
      Step<E> st;
      if (!helix_step<E>(to_e<E>(ref[2]), to_e<E>(ref[3]), to_e<E>(ref[4]), conv<E>(xk - x_prev), (E)M.kb,
                         (E)M.s_max, st)) {
        status = 1;
        return;
      }
      ref[0] += conv<S>(st.dy); ref[1] += conv<S>(st.dz); ref[2] += conv<S>(st.ds);
      d[0] += st.j_ys * d[2] + st.j_yq * d[4];
      d[1] += st.j_zs * d[2] + st.j_zt * d[3] + st.j_zq * d[4];
      d[2] += st.j_sq * d[4];
      cov_transport<C, E>(Cm, st);
    }
    if (id_next >= 0) {   // its position and row into L1 while this cluster is filtered
      prefetch_l1(&M.y[id_next]);
      prefetch_l1(&M.z[id_next]);
      if (M.row) prefetch_l1(&M.row[id_next]);
    }
    C var;
    if constexpr (is_df64<C>::value) {
      float dd = M.z_max_f - fabsf(M.z[id]);
      dd = fminf(fmaxf(dd, 0.0f), M.z_max_f);
      const float sg = M.sig_readout_f + M.sig_slope_f * dd;
      var = conv<C>(sg * sg);
    } else {
      const double zc = widen(M.z[id]);
      double dd = M.z_max - fabs(zc);
      dd = dd < 0.0 ? 0.0 : (dd > M.z_max ? M.z_max : dd);
      const double sg = M.sig_readout + M.sig_slope * dd;
      var = sg * sg;
    }
    const C r0 = (conv<C>(M.y[id]) - ref[0]) - d[0], r1 = (conv<C>(M.z[id]) - ref[1]) - d[1];
    const C c2 = refit_update<C, S>(d, Cm, r0, r1, var);
    if constexpr (kChi2) chi2 += c2;   // leading passes: chi2 never read
    x_prev = xk;
  }
}

template <int STAGE>
__global__ void __launch_bounds__(128) k_m_refit(const __grid_constant__ MParams M) {
  using S = typename std::conditional<STAGE == 1, df64, double>::type;
  using E = typename std::conditional<STAGE == 1, float, double>::type;
  using C = S;
  const tpct_chains_out& O = M.out;
  const int nc = min(M.head_idx[M.n_cap_tracks], O.capacity_chains);
  const int pass_begin = STAGE == 1 ? 0 : max(M.n_refit - 1, 0);
  const int pass_end = STAGE == 1 ? M.n_refit - 1 : M.n_refit;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    const int c = M.ch_order[q];
    const int m = O.n_seg[c], n = O.n_cl[c], off = O.offset[c], so = O.seg_offset[c];
    if (off + n > O.capacity_ids || so + m > O.capacity_segs) continue;
    const int* segs = O.segs + so;
    const int* ids = O.cluster_ids + off;
    int status = 0;
    double est[5], ref_out[5], x_cur;
    const int so_t = segs[m - 1];
    const double x_outer = M.xout[so_t];
    if (pass_begin == 0) {
      for (int i = 0; i < 5; ++i) ref_out[i] = M.trk.param[(int64_t)so_t * 5 + i];
      if (!transport(M, M.trk.x_ref[so_t], x_outer, ref_out, nullptr)) status = 1;
      for (int i = 0; i < 5; ++i) est[i] = M.trk.param[(int64_t)segs[0] * 5 + i];
      x_cur = M.trk.x_ref[segs[0]];
    } else {
      for (int i = 0; i < 5; ++i) {
        est[i] = M.ch_est[(int64_t)i * M.n_cap_tracks + c];
        ref_out[i] = M.ch_ref[(int64_t)i * M.n_cap_tracks + c];
      }
      x_cur = M.ch_x[c];
      status = M.ch_st[c];
    }
    S ref[5], d[5];
    C Cm[15], chi2 = conv<C>(0.0);
    for (int pass = pass_begin; pass < pass_end && !status; ++pass) {
      if (pass > 0) {
        double carry[5];
        for (int i = 0; i < 5; ++i) carry[i] = est[i];
        double xf = x_cur;
        bool ok = true;
        for (int j = 0; j < m && ok; ++j) {
          ok = transport(M, xf, M.xout[segs[j]], carry, nullptr);
          xf = M.xout[segs[j]];
          if (ok && j < m - 1) {
            double x1;
            ok = rotate_state(wrap_pi(M.alpha[segs[j + 1]] - M.alpha[segs[j]]), M.kb, M.s_max, xf, carry, &x1, nullptr);
            xf = x1;
          }
        }
        if (ok)
          for (int i = 0; i < 5; ++i) ref_out[i] = carry[i];
      }
      for (int i = 0; i < 5; ++i) { ref[i] = conv<S>(ref_out[i]); d[i] = conv<S>(0.0); }
      cov_diag<C>(Cm, conv<C>(M.c_yz_refit), conv<C>(M.c_yz_refit), conv<C>(M.c_s), conv<C>(M.c_t),
                  conv<C>(M.c_qpt_refit));
      chi2 = conv<C>(0.0);
      double x_prev = x_outer;
      int seg = m - 1;
      int seg_start = n - M.trk.n_cl[segs[m - 1]];   // first cluster index of the current segment
      if constexpr (STAGE == 1) {
        chain_span<S, E, C, false>(M, ids, segs, n, n - 1, 0, ref, d, Cm, chi2, x_prev, seg, seg_start, status);
      } else {
        // the last pass: its first kRefitHead clusters (outermost first) in
        // FP64, where the diffuse prior cancels, the rest in double-float
        const int k_split = max(n - kRefitHead, 0);
        chain_span<S, E, C>(M, ids, segs, n, n - 1, k_split, ref, d, Cm, chi2, x_prev, seg, seg_start, status);
        if (!status && k_split > 0) {
          df64 rf[5], df[5], Cf[15];
          for (int i = 0; i < 5; ++i) { rf[i] = df64(ref[i]); df[i] = df64(d[i]); }
          for (int i = 0; i < 15; ++i) Cf[i] = df64(Cm[i]);
          df64 chi2f = df64(chi2);
          chain_span<df64, float, df64>(M, ids, segs, n, k_split - 1, 0, rf, df, Cf, chi2f, x_prev, seg, seg_start,
                                        status);
          for (int i = 0; i < 5; ++i) { ref[i] = to_double(rf[i]); d[i] = to_double(df[i]); }
          for (int i = 0; i < 15; ++i) Cm[i] = to_double(Cf[i]);
          chi2 = to_double(chi2f);
        }
      }
      if (status) break;
      for (int i = 0; i < 5; ++i) est[i] = to_double(ref[i] + d[i]);
      x_cur = M.rx[row_of(M, ids[0])];
    }
    if (STAGE == 1) {
      for (int i = 0; i < 5; ++i) {
        M.ch_est[(int64_t)i * M.n_cap_tracks + c] = est[i];
        M.ch_ref[(int64_t)i * M.n_cap_tracks + c] = ref_out[i];
      }
      M.ch_x[c] = x_cur;
      M.ch_st[c] = status;
      continue;
    }
    O.status[c] = status;
    O.chi2[c] = status ? 0.0 : to_double(chi2);
    O.x_ref[c] = status ? M.trk.x_ref[segs[0]] : x_cur;
    for (int i = 0; i < 5; ++i)
      O.param[(int64_t)c * 5 + i] = status ? M.trk.param[(int64_t)segs[0] * 5 + i] : est[i];
    for (int i = 0; i < 15; ++i) O.cov[(int64_t)c * 15 + i] = status ? 0.0 : to_double(Cm[i]);
  }
}

int blocks_for(int64_t work, int block) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace carve (device pointers; base may be null to measure).
size_t merge_carve(char* base, int cap_tracks, int n_inst, int n_events, int cap_pairs, int cap_cand,
                   MParams* M) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* { char* p = base ? base + off : nullptr; off += align256(b ? b : 1); return p; };
  const size_t nt = (size_t)cap_tracks + 1;
  MParams q{};
  q.status = (uint32_t*)take(16);
  q.rx = (const double*)take(8 * kMaxRows);
  q.inst_of = (int32_t*)take(4 * (size_t)n_events * 36);
  q.first = (int32_t*)take(4 * (size_t)n_inst);
  q.last = (int32_t*)take(4 * (size_t)n_inst);
  q.alpha = (double*)take(8 * nt);
  q.rref = (double*)take(8 * nt);
  q.xout = (double*)take(8 * nt);
  q.inx = (double*)take(8 * nt);
  q.iny = (double*)take(8 * nt);
  q.outx = (double*)take(8 * nt);
  q.outy = (double*)take(8 * nt);
  q.fq = (float4*)take(16 * nt);
  q.fiy = (float*)take(4 * nt);
  q.best_out_chi = (uint64_t*)take(8 * nt);
  q.best_in_chi = (uint64_t*)take(8 * nt);
  q.best_out = (int32_t*)take(4 * nt);
  q.best_in = (int32_t*)take(4 * nt);
  q.n_cand = (int32_t*)take(16);
  q.cand_i = (int32_t*)take(4 * (size_t)cap_cand);
  q.cand_o = (int32_t*)take(4 * (size_t)cap_cand);
  q.n_pairs = (int32_t*)take(16);
  q.pair_i = (int32_t*)take(4 * (size_t)cap_pairs);
  q.pair_o = (int32_t*)take(4 * (size_t)cap_pairs);
  q.pair_chi = (double*)take(8 * (size_t)cap_pairs);
  q.head_flag = (int32_t*)take(4 * nt);
  q.head_idx = (int32_t*)take(4 * nt);
  q.nseg = (int32_t*)take(4 * nt);
  q.segoff = (int32_t*)take(4 * nt);
  q.ncl = (int32_t*)take(4 * nt);
  q.cloff = (int32_t*)take(4 * nt);
  q.len_cursor = (int32_t*)take(4 * (size_t)kLenBins);
  q.ch_order = (int32_t*)take(4 * nt);
  q.ch_est = (double*)take(8 * 5 * nt);
  q.ch_ref = (double*)take(8 * 5 * nt);
  q.ch_x = (double*)take(8 * nt);
  q.ch_st = (int32_t*)take(4 * nt);
  q.scan_tmp = (uint64_t*)take(8 * (size_t)(scan_tmp_elems(nt) + 32));
  if (M) {
    M->status = q.status; M->rx = q.rx; M->inst_of = q.inst_of; M->first = q.first; M->last = q.last; M->alpha = q.alpha;
    M->rref = q.rref; M->xout = q.xout; M->inx = q.inx; M->iny = q.iny; M->outx = q.outx; M->outy = q.outy;
    M->fq = q.fq; M->fiy = q.fiy;
    M->best_out_chi = q.best_out_chi; M->best_in_chi = q.best_in_chi; M->best_out = q.best_out;
    M->best_in = q.best_in; M->n_pairs = q.n_pairs; M->pair_i = q.pair_i; M->pair_o = q.pair_o;
    M->pair_chi = q.pair_chi; M->head_flag = q.head_flag; M->head_idx = q.head_idx; M->nseg = q.nseg;
    M->segoff = q.segoff; M->ncl = q.ncl; M->cloff = q.cloff; M->scan_tmp = q.scan_tmp;
    M->n_cand = q.n_cand; M->cand_i = q.cand_i; M->cand_o = q.cand_o; M->len_cursor = q.len_cursor;
    M->ch_order = q.ch_order; M->ch_est = q.ch_est; M->ch_ref = q.ch_ref; M->ch_x = q.ch_x; M->ch_st = q.ch_st;
  }
  return off;
}

}  // namespace

size_t merge_workspace_bytes(int cap_tracks, int n_inst, int n_events) {
  return merge_carve(nullptr, cap_tracks, n_inst, n_events, 4 * cap_tracks + 1024, 16 * cap_tracks + 4096, nullptr);
}

// Enqueue the merge; returns the number of kernels launched (or -1 on a bad workspace).
int enqueue_merge(const double* row_x_host, int n_rows, double kb, const tpct_cuts& cuts, double z_max,
                  const tpct_merge_cuts& mc, const tpct_clusters& cl, const int32_t* inst_sector,
                  const int32_t* inst_event, int n_events, const tpct_tracks_out& trk, void* ws, size_t ws_bytes,
                  const tpct_chains_out& out, cudaStream_t s) {
  const int cap = trk.capacity_tracks;
  const int cap_pairs = 4 * cap + 1024;
  const int cap_cand = 16 * cap + 4096;
  if (merge_carve(nullptr, cap, cl.n_instances, n_events, cap_pairs, cap_cand, nullptr) > ws_bytes) return -1;
  MParams M{};
  merge_carve((char*)ws, cap, cl.n_instances, n_events, cap_pairs, cap_cand, &M);
  RowTab tab;
  for (int i = 0; i < n_rows; ++i) tab.x[i] = row_x_host[i];
  M.n_rows = n_rows;
  M.n_inst = cl.n_instances;
  M.n_events = n_events;
  M.n_cap_tracks = cap;
  M.cap_pairs = cap_pairs;
  M.cap_cand = cap_cand;
  M.kb = kb;
  M.s_max = cuts.s_max;
  M.chi2_max = mc.chi2_max; M.max_dtanl = mc.max_dtanl; M.max_gap = mc.max_gap;
  M.alpha0 = mc.alpha0; M.dalpha = mc.dalpha;
  M.c_s = cuts.c_s; M.c_t = cuts.c_t; M.c_yz_refit = cuts.c_yz_refit; M.c_qpt_refit = cuts.c_qpt_refit;
  M.sig_readout = cuts.sig_readout; M.sig_slope = (cuts.sig_cathode - cuts.sig_readout) / z_max; M.z_max = z_max;
  M.n_refit = cuts.n_refit;
  M.sig_readout_f = (float)M.sig_readout; M.sig_slope_f = (float)M.sig_slope; M.z_max_f = (float)z_max;
  M.x = cl.x; M.y = cl.y; M.z = cl.z; M.row = cl.row;
  M.inst_sector = inst_sector; M.inst_event = inst_event;
  M.trk = trk;
  M.out = out;
  int k = 0;
  cudaMemsetAsync(M.status, 0, 16, s);
  k_m_rows<<<1, 256, 0, s>>>(const_cast<double*>(M.rx), n_rows, tab); ++k;
  const int big = max(max(cap, n_events * 36), cl.n_instances) + 1;
  k_m_init<<<blocks_for(big, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_prep<<<blocks_for(max(cap, cl.n_instances), kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_cand<<<max(1, n_events * 36), kBlock, 0, s>>>(M); ++k;
  k_m_chi<<<blocks_for(cap_cand, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_best<<<blocks_for(cap_pairs, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_links<<<blocks_for(cap, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_heads<<<blocks_for(cap, kBlock), kBlock, 0, s>>>(M); ++k;
  launch_scan_i32(M.head_flag, M.head_idx, cap, M.scan_tmp, s); k += 3;
  launch_scan_i32(M.nseg, M.segoff, cap, M.scan_tmp, s); k += 3;
  launch_scan_i32(M.ncl, M.cloff, cap, M.scan_tmp, s); k += 3;
  k_m_emit<<<blocks_for(cap, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_len_count<<<blocks_for(cap, kBlock), kBlock, 0, s>>>(M); ++k;
  k_m_len_scan<<<1, kLenBins, 0, s>>>(M); ++k;
  k_m_len_scatter<<<blocks_for(cap, kBlock), kBlock, 0, s>>>(M); ++k;
  if (cuts.n_refit >= 2) { k_m_refit<1><<<blocks_for(cap, 128), 128, 0, s>>>(M); ++k; }
  k_m_refit<2><<<blocks_for(cap, 128), 128, 0, s>>>(M); ++k;
  return k;
}

}  // namespace tpct
