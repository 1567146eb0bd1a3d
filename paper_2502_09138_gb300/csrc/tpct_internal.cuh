// Internal declarations of the GB300 sector tracker (not part of the ABI).
//
// Index spaces
//   input id  c   position in the caller's cluster arrays
//   sorted    p   position after the grid scatter: instance-major, row-major,
//                 bin-major inside a row; every per-cluster work array
//                 (links, flags, weights) lives in this space
//   row key   ir  instance * n_rows + row
//   tracklet  t   one per start hit, in (instance, row, start-hit id) order
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "tpct.h"
#include "df64.cuh"

namespace tpct {

constexpr int kMaxRows = 256;
constexpr int kRankBits = 20;                  // selection weight = nhits << 20 | (2^20-1-rank)
constexpr uint32_t kRankMask = (1u << kRankBits) - 1u;
constexpr int kStageEvents = 7;               // step boundaries timed by tpct_set_stage_events
constexpr int kMaxBlock = 256;                 // largest tracklet / refit block
constexpr int kLenClasses = 256;               // track-length classes of the refit order
// The refit's last pass runs its first kRefitHead clusters (outermost first)
// in FP64 and the rest in double-float (modes 1 and 3): the diffuse prior
// cancels in the first updates, where FP64 is needed; afterwards the
// covariance is data-dominated.
constexpr int kRefitHead = 8;
constexpr int kRefitState = 27;                 // ref[5], d[5], C[15], chi2, x of the last cluster
constexpr double kKbPerTesla = 0.299792458e-2; // curvature [1/cm] per (q/pT [c/GeV]) per tesla

enum StopReason { kStopEnd = 0, kStopProp = 1, kStopEdge = 2, kStopMiss = 3, kStopSinphi = 4 };
// Sticky device status bits.  (No kernel waits for another, so none can time
// out: bit 2 is unused.)  kDevBounds: an index outside its array, raised only
// by the bounds-checked build.
enum DevStatus : uint32_t { kDevCapacity = 1u, kDevTrackletCap = 4u, kDevBadRow = 8u, kDevBounds = 16u };

// ------------------------------------------------------------------ bounds-checked build
// Compiled with -DTPCT_CHECKED (build.py --checked), every workspace and input
// array of Params is an Arr: subscripts are range-checked against the
// array's allocated length before the access; an index outside sets
// kDevBounds in the status word and the access goes to a scratch cell instead
// (reads return whatever it holds; no trap, no write outside the arrays).  In
// the normal build TPCT_ARR(T) is a plain T* and mk_arr returns the pointer.
#ifdef TPCT_CHECKED
static __device__ __align__(64) unsigned char g_bounds_sink[64];
template <class T>
struct Arr {
  T* p = nullptr;
  int64_t n = 0;
  uint32_t* st = nullptr;
  __host__ __device__ Arr() {}
  __host__ __device__ Arr(T* p_, int64_t n_, uint32_t* st_) : p(p_), n(n_), st(st_) {}
  __host__ __device__ operator T*() const { return p; }
  __device__ T& operator[](int64_t i) const {
    if ((uint64_t)i < (uint64_t)n) return p[i];
    if (st) atomicOr(st, (uint32_t)kDevBounds);
    return *reinterpret_cast<T*>(g_bounds_sink);
  }
  __host__ __device__ Arr operator+(int64_t k) const { return Arr(p + k, n - k, st); }
};
template <class T> inline Arr<T> mk_arr(T* p, int64_t n, uint32_t* st) { return Arr<T>(p, n, st); }
#define TPCT_ARR(T) ::tpct::Arr<T>
template <class T>
__host__ __device__ inline Arr<T> writable(const Arr<const T>& a) { return Arr<T>(const_cast<T*>(a.p), a.n, a.st); }
#else
template <class T> inline T* mk_arr(T* p, int64_t, uint32_t*) { return p; }
#define TPCT_ARR(T) T*
#endif
// Write access to a table that every kernel but the one filling it reads as const.
template <class T>
__host__ __device__ inline T* writable(const T* p) { return const_cast<T*>(p); }

// Per-row grid: bins cover [y0, y0 + ny/idy) x [z0, z0 + nz/idz); indices
// outside are clamped to the border bins, so every cluster has a bin and the
// bin index is monotonic in y and in z.
struct RowGrid {
  float y0, z0, idy, idz;
  int32_t bin_base;   // first entry of this row in bin_start
  int16_t ny, nz;
};

// Everything a kernel needs, passed by value (uniform, lives in the constant bank).
struct Params {
  // sizes
  int32_t n_rows, n_inst, n, tcap, nbin_cap;
  int32_t hits_by_tracklet;    // tl_hits layout: 1 tracklet-major, 0 slot-major (hits_by_tracklet_for)
  int32_t clusters_per_bin;
  // geometry and cuts
  double tan_half, z_max, kb;
  double nf_wy, nf_wz, nf_dmax, s_max, edge_margin, search_k, chi2_max, f_shared;
  double sig_readout, sig_cathode, c_s, c_t, c_qpt, c_yz_refit, c_qpt_refit;
  double sig_slope;            // (sig_cathode - sig_readout) / z_max
  float sig_readout_f, sig_slope_f, z_max_f;
  float search_k_f, sig_hi_f, chi2_max_f;   // search_k, max(sig_readout, sig_cathode), chi2_max in float
  int32_t max_miss, n_min, n_refit;
  // input (device, caller-owned)
  TPCT_ARR(const float) x;
  TPCT_ARR(const float) y;
  TPCT_ARR(const float) z;
  TPCT_ARR(const uint8_t) row;
  TPCT_ARR(const int64_t) inst_off;
  // workspace
  TPCT_ARR(const double) rx;   // [n_rows] row x (double)
  TPCT_ARR(const float) rxf;   // [n_rows] row x (float)
  TPCT_ARR(const double) rdx;  // [n_rows] rx[r] - rx[r-1] (0 at r = 0)
  TPCT_ARR(const float) rdxf;  // [n_rows] the same rounded to float
  TPCT_ARR(const double) edge; // [n_rows] rx[r] * tan_half + edge_margin
  TPCT_ARR(const float) edgef; // [n_rows] the same rounded to float
  TPCT_ARR(const float) nf_tab;  // [5 n_rows] neighbour test per row r: f = (x_r - x_r-1) / (x_r+1 - x_r-1),
                                 // window half-widths up (y, z) and down (y, z); computed in double, rounded
  float s_max_f;               // s_max rounded to float
  uint32_t* status;            // sticky device status bits
  uint32_t* work;              // [2] work-queue heads of the tracklet and refit kernels
  TPCT_ARR(int32_t) row_count; // [n_inst*n_rows + 1]
  TPCT_ARR(int32_t) row_start; // [n_inst*n_rows + 1]
  TPCT_ARR(RowGrid) grid;      // [n_inst*n_rows]
  TPCT_ARR(int32_t) c_ir;      // [n] row key of each input cluster
  TPCT_ARR(int32_t) bin_count; // [nbin_cap + 1]
  TPCT_ARR(int32_t) bin_start; // [nbin_cap + 1]
  TPCT_ARR(float) sy;          // [n] sorted positions
  TPCT_ARR(float) sz;
  TPCT_ARR(int32_t) sid;       // [n] input id of each sorted position
  TPCT_ARR(uint8_t) srow;      // [n] row of each sorted position
  TPCT_ARR(int32_t) up;        // [n]
  TPCT_ARR(int32_t) down;
  TPCT_ARR(int32_t) upc;
  TPCT_ARR(uint8_t) sflag;     // [n] start-hit flag
  TPCT_ARR(int32_t) row_tl_count;  // [n_inst*n_rows + 1]
  TPCT_ARR(int32_t) row_tl_base;   // [n_inst*n_rows + 1]; [n_inst*n_rows] = tracklet count
  TPCT_ARR(int32_t) tl_start;  // [tcap]
  TPCT_ARR(int32_t) tl_ir;     // [tcap]
  TPCT_ARR(int32_t) tl_hits;   // [n_rows * tcap]: slot j of tracklet t at hit_at(P, t, j)
  TPCT_ARR(int32_t) tl_nhits;  // [tcap]
  TPCT_ARR(int32_t) tl_rowref; // [tcap]
  TPCT_ARR(double) tl_par;     // [5 * tcap]
  TPCT_ARR(uint32_t) W;        // [n]
  TPCT_ARR(uint64_t) tl_sel;   // [tcap + 1]  (accepted << 32 | owned) then its exclusive scan
  TPCT_ARR(uint64_t) tl_sel_scan;  // [tcap + 1]
  TPCT_ARR(int32_t) tl_cnt;    // [3 * tcap] helix steps, updates, chi2 tests of each tracklet
  TPCT_ARR(double) trk_est;    // [5 * tcap] refit estimate after the leading passes (mode 3)
  TPCT_ARR(double) trk_x;      // [tcap] its x
  TPCT_ARR(int32_t) trk_st;    // [tcap] transport failure in the leading passes
  TPCT_ARR(int32_t) trk_tl;    // [tcap] tracklet of each output track
  TPCT_ARR(int32_t) trk_pos;   // [n]    sorted position of each output cluster
  TPCT_ARR(int32_t) trk_order; // [tcap] output tracks, longest first (the refit's work order)
  TPCT_ARR(int32_t) len_cnt;   // [kLenClasses] tracks per length class, then cursors
  TPCT_ARR(double) rf_state;   // [kRefitState * tcap] last-pass state handed from the FP64 head to the tail
  TPCT_ARR(int32_t) rf_j;      // [tcap] next cluster of the tail, -1: the track finished in the head
  uint64_t* scan_tmp;          // block sums of the scans
  // output (device, caller-owned)
  tpct_tracks_out out;
};

// ------------------------------------------------------------------ precision
// S: track state, E: helix-transport / neighbour / search arithmetic,
// C: covariance, Kalman update; RS/RE/RC: the same for the refit.
// MODE 0 FP32; 1 mixed (float E, double C, double-float S: float transport
// increments added to a double-float state on the FP32 pipes, double Kalman
// gain and covariance update); 2 FP64; 3 mixed double-float (float E, double-float
// S/C in the tracklets).  The last refit pass is all-double in modes 1-3: its
// covariance starts from a diffuse prior and amplifies rounding by ~1e12,
// beyond what the 48-bit double-float keeps.
template <int MODE> struct Prec;
// PS/PE/PC: the refit passes before the last, which only move the
// linearisation point of a Gauss-Newton iteration (an error e there moves the
// final estimate by O(e^2)): modes 1 and 3 run them in double-float with float
// transport; the last pass, which gives the estimate and the covariance, in
// double.
template <> struct Prec<0> { using S = float;  using E = float;  using C = float;
                             using RS = float;  using RE = float;  using RC = float;
                             using PS = float;  using PE = float;  using PC = float; };
template <> struct Prec<1> { using S = df64;   using E = float;  using C = double;
                             using RS = double; using RE = double; using RC = double;
                             using PS = df64;   using PE = float;  using PC = df64; };
template <> struct Prec<2> { using S = double; using E = double; using C = double;
                             using RS = double; using RE = double; using RC = double;
                             using PS = double; using PE = double; using PC = double; };
template <> struct Prec<3> { using S = df64;   using E = float;  using C = df64;
                             using RS = double; using RE = double; using RC = double;
                             using PS = df64;   using PE = float;  using PC = df64; };

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint32_t float_order_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_key(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// Cluster resolution at measured z: linear in drift length clamp(z_max - |z|, 0, z_max).
template <class T>
__device__ __forceinline__ T sigma_of(const Params& P, T z) {
  T d = (T)P.z_max - fabs(z);
  d = d < (T)0 ? (T)0 : d;
  d = d > (T)P.z_max ? (T)P.z_max : d;
  return (T)P.sig_readout + (T)P.sig_slope * d;
}
template <>
__device__ __forceinline__ float sigma_of<float>(const Params& P, float z) {
  float d = P.z_max_f - fabsf(z);
  d = fminf(fmaxf(d, 0.f), P.z_max_f);
  return P.sig_readout_f + P.sig_slope_f * d;
}

// Cluster variance sigma(z)^2 in float: the tracklet filter takes the
// measurement model in float and converts it once (the FP64 covariance
// arithmetic itself is unchanged; 1e-7 relative on a variance moves chi2 by
// 1e-7 relative).  The refit keeps sigma in its own precision.
__device__ __forceinline__ float cluster_var(const Params& P, float z);

// Double-float callers take sigma in float: it enters only as the cluster
// variance, where 1e-7 relative is far below every tolerance.
template <>
__device__ __forceinline__ df64 sigma_of<df64>(const Params& P, df64 z) {
  return df64(sigma_of<float>(P, to_float(z)));
}

__device__ __forceinline__ float cluster_var(const Params& P, float z) {
  const float sg = sigma_of<float>(P, z);
  return sg * sg;
}

// Row-table access in the precision of the caller.
template <class E> __device__ __forceinline__ E row_dx(const Params& P, int r);
template <> __device__ __forceinline__ float row_dx<float>(const Params& P, int r) { return P.rdxf[r]; }
template <> __device__ __forceinline__ double row_dx<double>(const Params& P, int r) { return P.rdx[r]; }
template <class S> struct EdgeOf { __device__ static float get(const Params& P, int r) { return P.edgef[r]; } };
template <> struct EdgeOf<double> { __device__ static double get(const Params& P, int r) { return P.edge[r]; } };
template <class S> struct SmaxOf { __device__ static float get(const Params& P) { return P.s_max_f; } };
template <> struct SmaxOf<double> { __device__ static double get(const Params& P) { return P.s_max; } };

// Bin of (y, z) in a row grid (monotonic, clamped).
__device__ __forceinline__ int bin_y(const RowGrid& g, float y) {
  float t = (y - g.y0) * g.idy;
  t = fminf(fmaxf(t, 0.0f), (float)(g.ny - 1));
  return (int)t;
}
__device__ __forceinline__ int bin_z(const RowGrid& g, float z) {
  float t = (z - g.z0) * g.idz;
  t = fminf(fmaxf(t, 0.0f), (float)(g.nz - 1));
  return (int)t;
}

// Layout of the tracklet hit slots.  Tracklet-major (slot j of tracklet t at
// t * n_rows + j) keeps one partly written 32-byte sector per tracklet in
// flight, where slot-major (j * tcap + t) leaves one per slot row and
// tracklet, whose dirty lines crowd the cluster data out of L2 (3.3x the
// tracklet kernel's DRAM traffic).  The FP64-bound mixed filter keeps
// slot-major: with tracklet-major its FP64 loop ran 4 % slower.
__host__ __device__ constexpr bool hits_by_tracklet_for(int mode) { return mode != 1; }
__device__ __forceinline__ int64_t hit_at(const Params& P, int t, int j) {
  return P.hits_by_tracklet ? (int64_t)t * P.n_rows + j : (int64_t)j * P.tcap + t;
}

// Launch wrappers (defined in the .cu files).
void launch_grid_build(const Params& P, cudaStream_t s);
void launch_init_rows(const Params& P, cudaStream_t s);
void launch_scan_i32(const int32_t* in, int32_t* out, int64_t m, uint64_t* tmp, cudaStream_t s);
void launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t m, uint64_t* tmp, cudaStream_t s);
int64_t scan_tmp_elems(int64_t m);
void launch_neighbours(const Params& P, int mode, cudaStream_t s);
void launch_clean_start(const Params& P, cudaStream_t s);
void launch_start_fill(const Params& P, cudaStream_t s);
void launch_tracklets(const Params& P, int mode, int block, int blocks, cudaStream_t s);
int tracklet_blocks_per_sm(int mode, int block);
int refit_blocks_per_sm(int mode, int block);
void launch_weights(const Params& P, cudaStream_t s);
void launch_refit_order(const Params& P, cudaStream_t s);
int enqueue_clusters(const double* row_x, int n_rows, double tan_half, double z_max, const tpct_cf_params& prm,
                     const tpct_digits& dg, void* ws, size_t ws_bytes, const tpct_cf_out& out, cudaStream_t s,
                     cudaError_t* err);
size_t cf_workspace_bytes(int64_t n_digits, int32_t n_instances, int32_t n_rows, int32_t capacity);
size_t tm_encode_workspace_bytes(int64_t n, int32_t cap_tracks, int32_t n_blocks);
size_t tm_decode_workspace_bytes(int32_t n_tracks, int32_t n_blocks);
int enqueue_tm_encode(const double* row_x, int n_rows, const tpct_clusters& cl, int64_t n, const tpct_tracks_out& tr,
                      void* ws, size_t ws_bytes, const tpct_tm_stream& out, cudaStream_t s);
int enqueue_tm_decode(const double* row_x, int n_rows, const uint8_t* data, int64_t n_bytes, const int64_t* track_off,
                      int32_t n_tracks, const int64_t* row_off, int32_t n_blocks, void* ws, size_t ws_bytes,
                      const tpct_tm_decoded& out, cudaStream_t s);
void launch_own(const Params& P, cudaStream_t s);
void launch_emit(const Params& P, cudaStream_t s);
// stage 0: all refit passes; 1: all but the last (PS/PE/PC types); 2: the last
void launch_refit(const Params& P, int mode, int stage, int block, int blocks, cudaStream_t s);
void launch_export_links(const Params& P, const tpct_debug_out& d, cudaStream_t s);
void launch_export_tracklets(const Params& P, const tpct_debug_out& d, cudaStream_t s);
int kernels_per_track(void);
size_t merge_workspace_bytes(int cap_tracks, int n_inst, int n_events);
int enqueue_merge(const double* row_x_host, int n_rows, double kb, const tpct_cuts& cuts, double z_max,
                  const tpct_merge_cuts& mc, const tpct_clusters& cl, const int32_t* inst_sector,
                  const int32_t* inst_event, int n_events, const tpct_tracks_out& trk, void* ws, size_t ws_bytes,
                  const tpct_chains_out& out, cudaStream_t s);

}  // namespace tpct
