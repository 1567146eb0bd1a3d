// C ABI of the sector tracker: context, workspace layout, launch sequences.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include "tpct_internal.cuh"
#include "tpct_diag.h"

using namespace tpct;

struct tpct_ctx {
  int n_rows = 0;
  std::vector<double> row_x;
  double tan_half = 0, z_max = 0, bz = 0;
  tpct_cuts cuts{};
  tpct_precision prec = TPCT_PREC_MIXED;
  int clusters_per_bin = 2, tracklet_block = 128, refit_block = 128;
  int n_sm = 0, tl_blocks = 0, rf_blocks = 0;   // persistent grid sizes (0: not yet queried)
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int64_t plan_n = 0;
  int32_t plan_inst = 0;
  bool clear_status = false;  // the status word of a newly attached workspace is cleared by the next call
  Params last{};              // parameters of the last call (for debug export)
  bool have_last = false;
  cudaStream_t last_stream = nullptr;
  int64_t launches = 0;
  // step-boundary events (caller-owned)
  cudaEvent_t stage_ev[kStageEvents] = {};
  bool stage_on = false;
  // graph cache of the batched form
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;   // kept alive: its nodes address the exec's event nodes
  Params gparams{};
  bool gstage_on = false;
  cudaGraphNode_t gev_nodes[kStageEvents] = {};
  int gkernels = 0;
  cudaError_t last_err = cudaSuccess;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Sizes of every workspace array for a plan (n clusters, ni instances).
struct Plan {
  int64_t n, nr, tcap, nbin;
};

Plan make_plan(int n_rows, int64_t n, int32_t ni, int clusters_per_bin_min) {
  Plan p;
  p.n = n;
  p.nr = (int64_t)ni * n_rows;
  p.tcap = n / 3 + 1;
  p.nbin = n / clusters_per_bin_min + 2 * p.nr + 2;
  return p;
}

// An array of `count` elements of T taken from the workspace (with its
// length, which the bounds-checked build checks every subscript against).
template <class T, class Take>
TPCT_ARR(T) take_arr(Take& take, int64_t count, uint32_t* status) {
  return mk_arr((T*)take(sizeof(T) * (size_t)count), count, status);
}

// Assign pointers inside the workspace; returns the bytes used.
size_t carve(char* base, const Plan& pl, int n_rows, Params* P) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = align_up(off + (bytes ? bytes : 1));
    return p;
  };
  const int64_t n = pl.n > 0 ? pl.n : 1;
  const int64_t nr1 = pl.nr + 1;
  const int64_t scan_tmp = scan_tmp_elems(std::max<int64_t>(std::max<int64_t>(nr1, pl.nbin), pl.tcap + 1)) + 32;
  Params q{};
  q.status = (uint32_t*)take(sizeof(uint32_t) * 4);
  q.work = (uint32_t*)take(sizeof(uint32_t) * 4);
  q.rx = take_arr<const double>(take, n_rows, q.status);
  q.rxf = take_arr<const float>(take, n_rows, q.status);
  q.rdx = take_arr<const double>(take, n_rows, q.status);
  q.rdxf = take_arr<const float>(take, n_rows, q.status);
  q.edge = take_arr<const double>(take, n_rows, q.status);
  q.edgef = take_arr<const float>(take, n_rows, q.status);
  q.nf_tab = take_arr<const float>(take, (int64_t)5 * n_rows, q.status);
  q.row_count = take_arr<int32_t>(take, nr1, q.status);
  q.row_start = take_arr<int32_t>(take, nr1, q.status);
  q.row_tl_count = take_arr<int32_t>(take, nr1, q.status);
  q.row_tl_base = take_arr<int32_t>(take, nr1, q.status);
  q.grid = take_arr<RowGrid>(take, nr1, q.status);
  q.c_ir = take_arr<int32_t>(take, n, q.status);
  q.bin_count = take_arr<int32_t>(take, (pl.nbin + 1), q.status);
  q.bin_start = take_arr<int32_t>(take, (pl.nbin + 1), q.status);
  q.sy = take_arr<float>(take, n, q.status);
  q.sz = take_arr<float>(take, n, q.status);
  q.sid = take_arr<int32_t>(take, n, q.status);
  q.srow = take_arr<uint8_t>(take, n, q.status);
  q.up = take_arr<int32_t>(take, n, q.status);
  q.down = take_arr<int32_t>(take, n, q.status);
  q.upc = take_arr<int32_t>(take, n, q.status);
  q.sflag = take_arr<uint8_t>(take, n, q.status);
  q.W = take_arr<uint32_t>(take, n, q.status);
  q.tl_start = take_arr<int32_t>(take, pl.tcap, q.status);
  q.tl_ir = take_arr<int32_t>(take, pl.tcap, q.status);
  q.tl_nhits = take_arr<int32_t>(take, pl.tcap, q.status);
  q.tl_rowref = take_arr<int32_t>(take, pl.tcap, q.status);
  q.tl_hits = take_arr<int32_t>(take, (size_t)pl.tcap * n_rows, q.status);
  q.tl_par = take_arr<double>(take, 5 * (size_t)pl.tcap, q.status);
  q.tl_sel = take_arr<uint64_t>(take, (pl.tcap + 1), q.status);
  q.tl_sel_scan = take_arr<uint64_t>(take, (pl.tcap + 1), q.status);
  q.tl_cnt = take_arr<int32_t>(take, 3 * (size_t)pl.tcap, q.status);
  q.trk_est = take_arr<double>(take, 5 * (size_t)pl.tcap, q.status);
  q.trk_x = take_arr<double>(take, (size_t)pl.tcap, q.status);
  q.trk_st = take_arr<int32_t>(take, (size_t)pl.tcap, q.status);
  q.trk_tl = take_arr<int32_t>(take, pl.tcap, q.status);
  q.trk_pos = take_arr<int32_t>(take, n, q.status);
  q.trk_order = take_arr<int32_t>(take, (size_t)pl.tcap, q.status);
  q.len_cnt = take_arr<int32_t>(take, (size_t)kLenClasses, q.status);
  q.rf_state = take_arr<double>(take, (size_t)kRefitState * pl.tcap, q.status);
  q.rf_j = take_arr<int32_t>(take, (size_t)pl.tcap, q.status);
  q.scan_tmp = (uint64_t*)take(8 * scan_tmp);
  if (P) {
    P->status = q.status; P->work = q.work; P->rx = q.rx; P->rxf = q.rxf;
    P->rdx = q.rdx; P->rdxf = q.rdxf; P->edge = q.edge; P->edgef = q.edgef; P->nf_tab = q.nf_tab;
    P->row_count = q.row_count; P->row_start = q.row_start;
    P->row_tl_count = q.row_tl_count; P->row_tl_base = q.row_tl_base;
    P->grid = q.grid; P->c_ir = q.c_ir;
    P->bin_count = q.bin_count; P->bin_start = q.bin_start;
    P->sy = q.sy; P->sz = q.sz; P->sid = q.sid; P->srow = q.srow;
    P->up = q.up; P->down = q.down; P->upc = q.upc; P->sflag = q.sflag; P->W = q.W;
    P->tl_start = q.tl_start; P->tl_ir = q.tl_ir; P->tl_nhits = q.tl_nhits; P->tl_rowref = q.tl_rowref;
    P->tl_hits = q.tl_hits; P->tl_par = q.tl_par; P->tl_sel = q.tl_sel; P->tl_sel_scan = q.tl_sel_scan;
    P->tl_cnt = q.tl_cnt; P->trk_tl = q.trk_tl;
    P->trk_est = q.trk_est; P->trk_x = q.trk_x; P->trk_st = q.trk_st; P->trk_pos = q.trk_pos; P->scan_tmp = q.scan_tmp;
    P->trk_order = q.trk_order; P->len_cnt = q.len_cnt; P->rf_state = q.rf_state; P->rf_j = q.rf_j;
  }
  return off;
}

struct RowTable {
  double x[kMaxRows];
};
// Row tables: x, the step to the previous row, the sector edge plus margin,
// in double and float; the float constants of the neighbour test of every
// inner row (formed in double once here instead of per row and lane).
__global__ void k_set_tables_v(const Params P, const RowTable tab) {
  for (int i = threadIdx.x; i < P.n_rows; i += blockDim.x) {
    const double x = tab.x[i];
    const double dx = i > 0 ? x - tab.x[i - 1] : 0.0;
    const double e = x * P.tan_half + P.edge_margin;
    writable(P.rx)[i] = x;
    writable(P.rxf)[i] = (float)x;
    writable(P.rdx)[i] = dx;
    writable(P.rdxf)[i] = (float)dx;
    writable(P.edge)[i] = e;
    writable(P.edgef)[i] = (float)e;
    float f = 0.f, wyu = 0.f, wzu = 0.f, wyd = 0.f, wzd = 0.f;
    if (i > 0 && i + 1 < P.n_rows) {
      const double xu = tab.x[i + 1], xd = tab.x[i - 1];
      f = (float)((x - xd) / (xu - xd));
      wyu = (float)(P.nf_wy * (xu - x)); wzu = (float)(P.nf_wz * (xu - x));
      wyd = (float)(P.nf_wy * (x - xd)); wzd = (float)(P.nf_wz * (x - xd));
    }
    writable(P.nf_tab)[5 * i] = f;
    writable(P.nf_tab)[5 * i + 1] = wyu;
    writable(P.nf_tab)[5 * i + 2] = wzu;
    writable(P.nf_tab)[5 * i + 3] = wyd;
    writable(P.nf_tab)[5 * i + 4] = wzd;
  }
}

void drop_graph(tpct_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
}

tpct_status fail_cuda(tpct_ctx* ctx, cudaError_t e) {
  if (ctx) ctx->last_err = e;
  return e == cudaSuccess ? TPCT_OK : TPCT_E_CUDA;
}

bool valid_cuts(const tpct_cuts& c) {
  return c.nf_wy > 0 && c.nf_wz > 0 && c.nf_dmax >= 0 && c.s_max > 0 && c.s_max < 1 &&
         c.search_k > 0 && c.chi2_max > 0 && c.max_miss >= 0 && c.n_min >= 3 && c.f_shared >= 0 &&
         c.n_refit >= 1 && c.sig_readout > 0 && c.sig_cathode > 0 && c.c_s > 0 && c.c_t > 0 &&
         c.c_qpt > 0 && c.c_yz_refit > 0 && c.c_qpt_refit > 0 && c.edge_margin >= 0;
}

tpct_status check_cuda(cudaError_t e) { return e == cudaSuccess ? TPCT_OK : TPCT_E_CUDA; }

// Validates a call's clusters and outputs (the checks every tracking entry point makes).
tpct_status check_call(const tpct_clusters* cl, int64_t n, const tpct_tracks_out* out) {
  if (!cl || !out || n < 0) return TPCT_E_INVALID;
  if (n > 0 && (!cl->y || !cl->z || (!cl->row && !cl->x))) return TPCT_E_INVALID;
  if (!cl->sector_offsets) return TPCT_E_INVALID;
  if (!out->n_tracks || !out->n_ids || out->capacity_tracks < 0 || out->capacity_ids < 0) return TPCT_E_INVALID;
  if (out->capacity_tracks > 0 && (!out->instance || !out->n_cl || !out->offset || !out->ndf ||
                                   !out->status || !out->x_ref || !out->param || !out->cov || !out->chi2))
    return TPCT_E_INVALID;
  if (out->capacity_ids > 0 && !out->cluster_ids) return TPCT_E_INVALID;
  return TPCT_OK;
}

// Persistent grid sizes of the context (queried on its first call).
tpct_status ensure_grids(tpct_ctx* ctx) {
  if (ctx->tl_blocks != 0 && ctx->rf_blocks != 0) return TPCT_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_cuda(ctx, e);
  ctx->tl_blocks = ctx->n_sm * tracklet_blocks_per_sm((int)ctx->prec, ctx->tracklet_block);
  ctx->rf_blocks = ctx->n_sm * refit_blocks_per_sm((int)ctx->prec, ctx->refit_block);
  return TPCT_OK;
}

// The per-call parameters: the workspace `base` carved for `plan_ws`, the
// constants of the context's cut set and geometry, the call's sizes and
// buffers.  The one place every tracking entry point fills them.
void fill_params(const tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, const tpct_tracks_out* out, char* base,
                 const Plan& plan_ws, Params* P) {
  Params p{};
  const Plan pl = make_plan(ctx->n_rows, n, cl->n_instances, ctx->clusters_per_bin);
  carve(base, plan_ws, ctx->n_rows, &p);
  p.n_rows = ctx->n_rows;
  p.n_inst = cl->n_instances;
  p.n = (int32_t)n;
  p.tcap = (int32_t)pl.tcap;
  p.nbin_cap = (int32_t)pl.nbin;
  p.hits_by_tracklet = hits_by_tracklet_for((int)ctx->prec) ? 1 : 0;
  p.clusters_per_bin = ctx->clusters_per_bin;
  p.tan_half = ctx->tan_half;
  p.z_max = ctx->z_max;
  p.kb = kKbPerTesla * ctx->bz;
  const tpct_cuts& c = ctx->cuts;
  p.nf_wy = c.nf_wy; p.nf_wz = c.nf_wz; p.nf_dmax = c.nf_dmax; p.s_max = c.s_max;
  p.edge_margin = c.edge_margin; p.search_k = c.search_k; p.chi2_max = c.chi2_max;
  p.f_shared = c.f_shared; p.sig_readout = c.sig_readout; p.sig_cathode = c.sig_cathode;
  p.c_s = c.c_s; p.c_t = c.c_t; p.c_qpt = c.c_qpt; p.c_yz_refit = c.c_yz_refit;
  p.c_qpt_refit = c.c_qpt_refit; p.sig_slope = (c.sig_cathode - c.sig_readout) / ctx->z_max;
  p.s_max_f = (float)c.s_max;
  p.sig_readout_f = (float)c.sig_readout;
  p.sig_slope_f = (float)p.sig_slope;
  p.z_max_f = (float)ctx->z_max;
  p.search_k_f = (float)c.search_k;
  p.sig_hi_f = (float)(c.sig_readout > c.sig_cathode ? c.sig_readout : c.sig_cathode);
  p.chi2_max_f = (float)c.chi2_max;
  p.max_miss = c.max_miss; p.n_min = c.n_min; p.n_refit = c.n_refit;
  p.x = mk_arr(cl->x, n, p.status);
  p.y = mk_arr(cl->y, n, p.status);
  p.z = mk_arr(cl->z, n, p.status);
  p.row = mk_arr(cl->row, n, p.status);
  p.inst_off = mk_arr(cl->sector_offsets, (int64_t)cl->n_instances + 1, p.status);
  p.out = *out;
  *P = p;
}

// Build the per-call parameters of a call on the attached workspace; validates sizes.
tpct_status make_params(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, const tpct_tracks_out* out,
                        Params* P) {
  if (!ctx || !cl || !out || n < 0) return TPCT_E_INVALID;
  if (!ctx->ws) return TPCT_E_STATE;
  tpct_status st = check_call(cl, n, out);
  if (st != TPCT_OK) return st;
  if (n > ctx->plan_n || cl->n_instances > ctx->plan_inst || cl->n_instances < 1) return TPCT_E_NOMEM;
  st = ensure_grids(ctx);
  if (st != TPCT_OK) return st;
  fill_params(ctx, cl, n, out, ctx->ws, make_plan(ctx->n_rows, ctx->plan_n, ctx->plan_inst, 1), P);
  return TPCT_OK;
}

// Clears the status word of a newly attached workspace in the order of the
// call's stream (tpct_set_workspace itself touches no device memory).
tpct_status clear_status_if_new(tpct_ctx* ctx, const Params& P, cudaStream_t s) {
  if (!ctx->clear_status) return TPCT_OK;
  const cudaError_t e = cudaMemsetAsync(P.status, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return fail_cuda(ctx, e);
  ctx->clear_status = false;
  return TPCT_OK;
}

// The step sequence; returns the number of kernels launched.  With stage
// events on, an event is recorded at every step boundary.
int enqueue_track(tpct_ctx* ctx, const Params& P, cudaStream_t s) {
  int k = 0;
  const int mode = (int)ctx->prec;
  // External records: inside a stream capture they become event-record nodes.
  auto mark = [&](int b) {
    if (ctx->stage_on) cudaEventRecordWithFlags(ctx->stage_ev[b], s, cudaEventRecordExternal);
  };
  RowTable tab;
  for (int i = 0; i < ctx->n_rows; ++i) tab.x[i] = ctx->row_x[i];
  const int64_t nr = (int64_t)P.n_inst * P.n_rows;
  const int scan_k = 3;
  mark(0);
  k_set_tables_v<<<1, 256, 0, s>>>(P, tab); ++k;
  launch_init_rows(P, s); ++k;
  cudaMemsetAsync(P.work, 0, sizeof(uint32_t) * 4, s);
  launch_grid_build(P, s); ++k;
  mark(1);
  launch_neighbours(P, mode, s); ++k;
  mark(2);
  launch_clean_start(P, s); ++k;
  launch_scan_i32(P.row_tl_count, P.row_tl_base, nr, P.scan_tmp, s); k += scan_k;
  launch_start_fill(P, s); ++k;
  mark(3);
  cudaMemsetAsync(P.work, 0, sizeof(uint32_t) * 4, s);
  launch_tracklets(P, mode, ctx->tracklet_block, ctx->tl_blocks, s); ++k;
  mark(4);
  launch_weights(P, s); ++k;
  launch_own(P, s); ++k;
  launch_scan_u64(P.tl_sel, P.tl_sel_scan, P.tcap, P.scan_tmp, s); k += scan_k;
  launch_emit(P, s); ++k;
  mark(5);
  cudaMemsetAsync(P.len_cnt, 0, sizeof(int32_t) * kLenClasses, s);
  launch_refit_order(P, s); k += 3;
  if ((mode == 1 || mode == 3) && P.n_refit >= 2) {
    // leading passes in double-float; the last pass in double for its first
    // kRefitHead clusters and in double-float for the rest
    launch_refit(P, mode, 1, ctx->refit_block, ctx->rf_blocks, s); ++k;
    launch_refit(P, mode, 2, ctx->refit_block, ctx->rf_blocks, s); ++k;
    launch_refit(P, mode, 3, ctx->refit_block, ctx->rf_blocks, s); ++k;
  } else {
    launch_refit(P, mode, 0, ctx->refit_block, ctx->rf_blocks, s); ++k;
  }
  mark(6);
  return k;
}

}  // namespace

extern "C" {

// The TPC readout of the workload: 152 pad rows in three regions (63 rows at
// 0.75 cm pitch from x = 85.2 cm, 64 at 1.0 cm from 135.1 cm, 25 at 1.5 cm
// from 199.4 cm), 20-degree sectors (acceptance |y| <= x tan 10 deg), 250 cm
// of drift.  The radii live in static storage of the library.
void tpct_default_geometry(tpct_geometry* g) {
  if (!g) return;
  static const std::vector<double> rows = [] {
    std::vector<double> r(152);
    for (int i = 0; i < 152; ++i)
      r[i] = i < 63 ? 85.2 + 0.75 * i : i < 127 ? 135.1 + 1.0 * (i - 63) : 199.4 + 1.5 * (i - 127);
    return r;
  }();
  g->n_rows = 152;
  g->row_x = rows.data();
  g->tan_half_sector = 0.17632698070846498;   // tan(10 deg)
  g->z_max = 250.0;
}

void tpct_default_cuts(tpct_cuts* c) {
  if (!c) return;
  c->nf_wy = 2.0; c->nf_wz = 2.0; c->nf_dmax = 0.25; c->s_max = 0.999; c->edge_margin = 1.0;
  c->search_k = 5.0; c->chi2_max = 25.0; c->max_miss = 8; c->n_min = 20; c->f_shared = 0.1;
  c->n_refit = 3; c->sig_readout = 0.1; c->sig_cathode = 0.1; c->c_s = 1.0; c->c_t = 1.0;
  c->c_qpt = 100.0; c->c_yz_refit = 100.0; c->c_qpt_refit = 1.0e4;
}

tpct_status tpct_create(const tpct_geometry* g, double bz, const tpct_cuts* cuts, tpct_precision prec,
                        tpct_ctx** out) {
  if (!g || !cuts || !out || !g->row_x || g->n_rows < 3 || g->n_rows > kMaxRows) return TPCT_E_INVALID;
  if (!(g->tan_half_sector > 0) || !(g->z_max > 0)) return TPCT_E_INVALID;
  for (int i = 1; i < g->n_rows; ++i)
    if (!(g->row_x[i] > g->row_x[i - 1])) return TPCT_E_INVALID;
  if (!valid_cuts(*cuts) || (int)prec < 0 || (int)prec > 3) return TPCT_E_INVALID;
  tpct_ctx* c = new (std::nothrow) tpct_ctx();
  if (!c) return TPCT_E_NOMEM;
  c->n_rows = g->n_rows;
  c->row_x.assign(g->row_x, g->row_x + g->n_rows);
  c->tan_half = g->tan_half_sector;
  c->z_max = g->z_max;
  c->bz = bz;
  c->cuts = *cuts;
  c->prec = prec;
  *out = c;
  return TPCT_OK;
}

void tpct_destroy(tpct_ctx* ctx) {
  if (!ctx) return;
  drop_graph(ctx);
  delete ctx;
}

tpct_status tpct_set_tuning(tpct_ctx* ctx, int cpb, int tl_block, int rf_block) {
  if (!ctx || cpb < 0 || tl_block < 0 || rf_block < 0) return TPCT_E_INVALID;
  if (tl_block && (tl_block % 32 || tl_block > kMaxBlock)) return TPCT_E_INVALID;
  if (rf_block && (rf_block % 32 || rf_block > kMaxBlock)) return TPCT_E_INVALID;
  ctx->clusters_per_bin = cpb ? cpb : 2;
  ctx->tracklet_block = tl_block ? tl_block : 128;
  ctx->refit_block = rf_block ? rf_block : 128;
  ctx->tl_blocks = ctx->rf_blocks = 0;
  drop_graph(ctx);
  return TPCT_OK;
}

size_t tpct_workspace_bytes(const tpct_ctx* ctx, int64_t max_clusters, int32_t max_instances) {
  if (!ctx || max_clusters < 0 || max_instances < 1 || max_clusters > INT32_MAX / 4) return 0;
  Plan pl = make_plan(ctx->n_rows, max_clusters, max_instances, 1);
  return carve(nullptr, pl, ctx->n_rows, nullptr);
}

tpct_status tpct_set_workspace(tpct_ctx* ctx, void* ptr, size_t bytes, int64_t max_clusters,
                               int32_t max_instances) {
  if (!ctx || !ptr || ((uintptr_t)ptr % kAlign)) return TPCT_E_INVALID;
  size_t need = tpct_workspace_bytes(ctx, max_clusters, max_instances);
  if (need == 0) return TPCT_E_INVALID;
  if (bytes < need) return TPCT_E_NOMEM;
  ctx->ws = (char*)ptr;
  ctx->ws_bytes = bytes;
  ctx->plan_n = max_clusters;
  ctx->plan_inst = max_instances;
  ctx->have_last = false;
  ctx->clear_status = true;
  drop_graph(ctx);
  return TPCT_OK;
}

tpct_status tpct_track(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, tpct_tracks_out* out,
                       tpct_stream stream) {
  Params P;
  tpct_status st = make_params(ctx, cl, n, out, &P);
  if (st != TPCT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = clear_status_if_new(ctx, P, s);
  if (st != TPCT_OK) return st;
  ctx->launches += enqueue_track(ctx, P, s);
  ctx->last = P;
  ctx->have_last = true;
  ctx->last_stream = s;
  return fail_cuda(ctx, cudaGetLastError());
}

tpct_status tpct_track_batch(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, tpct_tracks_out* out,
                             tpct_stream stream) {
  Params P;
  tpct_status st = make_params(ctx, cl, n, out, &P);
  if (st != TPCT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = clear_status_if_new(ctx, P, s);
  if (st != TPCT_OK) return st;
  if (!ctx->gexec || ctx->gstage_on != ctx->stage_on || std::memcmp(&ctx->gparams, &P, sizeof(Params)) != 0) {
    drop_graph(ctx);
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      ctx->gkernels = enqueue_track(ctx, P, cap);
      e = cudaStreamEndCapture(cap, &graph);
    }
    for (int b = 0; b < kStageEvents; ++b) ctx->gev_nodes[b] = nullptr;
    if (e == cudaSuccess && ctx->stage_on) {
      // the event-record nodes in boundary order (matched by event handle)
      size_t nn = 0;
      e = cudaGraphGetNodes(graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
      for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
        for (int b = 0; b < kStageEvents; ++b)
          if (ev == ctx->stage_ev[b]) ctx->gev_nodes[b] = nodes[i];
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      ctx->gexec = nullptr;
      return fail_cuda(ctx, e);
    }
    ctx->graph = graph;
    ctx->gparams = P;
    ctx->gstage_on = ctx->stage_on;
  } else if (ctx->stage_on) {
    for (int b = 0; b < kStageEvents; ++b) {
      if (!ctx->gev_nodes[b]) continue;
      cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(ctx->gexec, ctx->gev_nodes[b], ctx->stage_ev[b]);
      if (e != cudaSuccess) return fail_cuda(ctx, e);
    }
  }
  cudaError_t le = cudaGraphLaunch(ctx->gexec, s);
  if (le != cudaSuccess) return fail_cuda(ctx, le);
  ctx->launches += ctx->gkernels;
  ctx->last = P;
  ctx->have_last = true;
  ctx->last_stream = s;
  return TPCT_OK;
}

tpct_status tpct_set_stage_events(tpct_ctx* ctx, void* const* events, int n_events) {
  if (!ctx || (n_events != 0 && n_events != kStageEvents) || (n_events && !events)) return TPCT_E_INVALID;
  for (int b = 0; b < kStageEvents; ++b) {
    ctx->stage_ev[b] = n_events ? (cudaEvent_t)events[b] : nullptr;
    if (n_events && !events[b]) return TPCT_E_INVALID;
  }
  ctx->stage_on = n_events != 0;
  return TPCT_OK;
}

tpct_status tpct_debug_export(tpct_ctx* ctx, tpct_debug_out* dbg, tpct_stream stream) {
  if (!ctx || !dbg) return TPCT_E_INVALID;
  if (!ctx->have_last) return TPCT_E_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  launch_export_links(ctx->last, *dbg, s);
  launch_export_tracklets(ctx->last, *dbg, s);
  ctx->launches += 2;
  return check_cuda(cudaGetLastError());
}

tpct_status tpct_last_device_status(tpct_ctx* ctx) {
  if (!ctx || !ctx->ws) return TPCT_E_STATE;
  if (ctx->clear_status) return TPCT_OK;   // no call since the workspace was attached
  if (ctx->have_last && cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return TPCT_E_CUDA;
  Params p{};
  carve(ctx->ws, make_plan(ctx->n_rows, ctx->plan_n, ctx->plan_inst, 1), ctx->n_rows, &p);
  uint32_t h = 0;
  if (cudaMemcpy(&h, p.status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return TPCT_E_CUDA;
  if (cudaMemset(p.status, 0, sizeof(uint32_t)) != cudaSuccess) return TPCT_E_CUDA;
  if (h & kDevBounds) return TPCT_E_BOUNDS;
  if (h & (kDevCapacity | kDevTrackletCap)) return TPCT_E_CAPACITY;
  if (h & kDevBadRow) return TPCT_E_INVALID;
  return TPCT_OK;
}

const char* tpct_status_str(tpct_status s) {
  switch (s) {
    case TPCT_OK: return "ok";
    case TPCT_E_INVALID: return "invalid argument";
    case TPCT_E_NOMEM: return "out of memory or workspace too small";
    case TPCT_E_CAPACITY: return "output capacity exceeded";
    case TPCT_E_CUDA: return "CUDA error";
    case TPCT_E_TIMEOUT: return "wait timed out";
    case TPCT_E_BUDGET: return "request exceeds the memory budget";
    case TPCT_E_STATE: return "invalid state";
    case TPCT_E_BOUNDS: return "device index out of bounds (checked build)";
  }
  return "unknown status";
}

int64_t tpct_kernel_launches(const tpct_ctx* ctx) { return ctx ? ctx->launches : -1; }

void tpct_default_merge_cuts(tpct_merge_cuts* c) {
  if (!c) return;
  c->chi2_max = 50.0;
  c->max_dtanl = 0.1;
  c->max_gap = 40.0;
  c->alpha0 = 0.17453292519943295;   // 10 degrees
  c->dalpha = 0.3490658503988659;    // 20 degrees
}

size_t tpct_merge_workspace_bytes(int32_t max_tracks, int32_t n_instances, int32_t n_events) {
  if (max_tracks < 1 || n_instances < 1 || n_events < 1) return 0;
  return merge_workspace_bytes(max_tracks, n_instances, n_events);
}

tpct_status tpct_merge(tpct_ctx* ctx, const tpct_clusters* cl, const int32_t* inst_sector, const int32_t* inst_event,
                       int32_t n_events, const tpct_tracks_out* tracks, const tpct_merge_cuts* cuts, void* ws,
                       size_t ws_bytes, tpct_chains_out* out, tpct_stream stream) {
  if (!ctx || !cl || !inst_sector || !inst_event || n_events < 1 || !tracks || !cuts || !ws || !out)
    return TPCT_E_INVALID;
  if (((uintptr_t)ws % kAlign) || cl->n_instances < 1 || (!cl->row && !cl->x) || !cl->y || !cl->z)
    return TPCT_E_INVALID;
  if (tracks->capacity_tracks < 1 || !tracks->n_tracks || !tracks->instance || !tracks->cluster_ids)
    return TPCT_E_INVALID;
  if (!out->n_chains || !out->n_ids || !out->n_segs || out->capacity_chains < 0 || out->capacity_ids < 0 ||
      out->capacity_segs < 0)
    return TPCT_E_INVALID;
  if (out->capacity_chains > 0 && (!out->head || !out->n_seg || !out->seg_offset || !out->instance ||
                                   !out->n_cl || !out->offset || !out->ndf || !out->status || !out->x_ref ||
                                   !out->param || !out->cov || !out->chi2))
    return TPCT_E_INVALID;
  if ((out->capacity_ids > 0 && !out->cluster_ids) || (out->capacity_segs > 0 && !out->segs)) return TPCT_E_INVALID;
  const int k = enqueue_merge(ctx->row_x.data(), ctx->n_rows, kKbPerTesla * ctx->bz, ctx->cuts, ctx->z_max, *cuts,
                              *cl, inst_sector, inst_event, n_events, *tracks, ws, ws_bytes, *out,
                              (cudaStream_t)stream);
  if (k < 0) return TPCT_E_NOMEM;
  ctx->launches += k;
  return fail_cuda(ctx, cudaGetLastError());
}

void tpct_default_cf_params(tpct_cf_params* p) {
  if (!p) return;
  p->pad_pitch_inner = 0.4; p->pad_pitch_outer = 0.6; p->n_inner_rows = 63;
  p->time_bin = 0.5; p->n_time = 500; p->q_peak_min = 7; p->valley_delta = 2;
}

size_t tpct_cf_workspace_bytes(int64_t n_digits, int32_t n_instances, int32_t n_rows, int32_t capacity) {
  if (n_digits < 0 || n_instances < 0 || n_rows < 1 || capacity < 0) return 0;
  return cf_workspace_bytes(n_digits, n_instances, n_rows, capacity);
}

tpct_status tpct_find_clusters(tpct_ctx* ctx, const tpct_digits* dg, const tpct_cf_params* prm, void* ws,
                               size_t ws_bytes, tpct_cf_out* out, tpct_stream stream) {
  if (!ctx || !dg || !prm || !ws || !out || dg->n_instances < 0 || ((uintptr_t)ws % kAlign)) return TPCT_E_INVALID;
  if (dg->n_instances > 0 && (!dg->row_offsets || !dg->inst_sector)) return TPCT_E_INVALID;
  if (!out->n_clusters || !out->status || out->capacity < 0) return TPCT_E_INVALID;
  if (out->capacity > 0 && (!out->x || !out->y || !out->z || !out->pad || !out->time || !out->sigma_pad ||
                            !out->sigma_time || !out->q_tot || !out->q_max || !out->row || !out->flags))
    return TPCT_E_INVALID;
  if (prm->q_peak_min < 1 || prm->valley_delta < 0 || prm->n_inner_rows < 0) return TPCT_E_INVALID;
  cudaError_t err = cudaSuccess;
  const int k = enqueue_clusters(ctx->row_x.data(), ctx->n_rows, ctx->tan_half, ctx->z_max, *prm, *dg, ws,
                                 ws_bytes, *out, (cudaStream_t)stream, &err);
  if (k == -1 || k == -3) return TPCT_E_INVALID;
  if (k == -2) return TPCT_E_NOMEM;
  if (k < 0) return fail_cuda(ctx, err);
  ctx->launches += k;
  return TPCT_OK;
}

size_t tpct_tm_encode_workspace_bytes(int64_t n, int32_t capacity_tracks, int32_t n_instances, int32_t n_rows) {
  if (n < 0 || capacity_tracks < 0 || n_instances < 0 || n_rows < 1) return 0;
  return tm_encode_workspace_bytes(n, capacity_tracks, n_instances * n_rows);
}

tpct_status tpct_tm_encode(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, const tpct_tracks_out* tr, void* ws,
                           size_t ws_bytes, tpct_tm_stream* out, tpct_stream stream) {
  if (!ctx || !cl || !tr || !ws || !out || n < 0 || n > INT32_MAX || ((uintptr_t)ws % kAlign)) return TPCT_E_INVALID;
  if (cl->n_instances < 1 || !cl->sector_offsets || (n > 0 && (!cl->y || !cl->z || !cl->row))) return TPCT_E_INVALID;
  if (tr->capacity_tracks < 0 || !tr->n_tracks || (tr->capacity_tracks > 0 && (!tr->offset || !tr->n_cl ||
                                                                               !tr->cluster_ids)))
    return TPCT_E_INVALID;
  if (!out->n_bytes || out->capacity < 0 || (out->capacity > 0 && !out->data)) return TPCT_E_INVALID;
  const int k = enqueue_tm_encode(ctx->row_x.data(), ctx->n_rows, *cl, n, *tr, ws, ws_bytes, *out,
                                  (cudaStream_t)stream);
  if (k < 0) return TPCT_E_NOMEM;
  ctx->launches += k;
  return fail_cuda(ctx, cudaGetLastError());
}

size_t tpct_tm_decode_workspace_bytes(int32_t n_tracks, int32_t n_instances, int32_t n_rows) {
  if (n_tracks < 0 || n_instances < 0 || n_rows < 1) return 0;
  return tm_decode_workspace_bytes(n_tracks, n_instances * n_rows);
}

tpct_status tpct_tm_decode(tpct_ctx* ctx, const uint8_t* data, int64_t n_bytes, const int64_t* track_off,
                           int32_t n_tracks, const int64_t* row_off, int32_t n_instances, void* ws, size_t ws_bytes,
                           tpct_tm_decoded* out, tpct_stream stream) {
  if (!ctx || !ws || !out || n_tracks < 0 || n_instances < 0 || n_bytes < 0 || ((uintptr_t)ws % kAlign))
    return TPCT_E_INVALID;
  if ((n_tracks > 0 && !track_off) || (n_instances > 0 && !row_off) || (n_bytes > 0 && !data)) return TPCT_E_INVALID;
  if (!out->n || !out->status || out->capacity < 0 ||
      (out->capacity > 0 && (!out->x || !out->y || !out->z || !out->charge || !out->row)))
    return TPCT_E_INVALID;
  const int k = enqueue_tm_decode(ctx->row_x.data(), ctx->n_rows, data, n_bytes, track_off, n_tracks, row_off,
                                  n_instances * ctx->n_rows, ws, ws_bytes, *out, (cudaStream_t)stream);
  if (k < 0) return TPCT_E_NOMEM;
  ctx->launches += k;
  return fail_cuda(ctx, cudaGetLastError());
}

tpct_status tpct_get_tuning(const tpct_ctx* ctx, tpct_tuning* t) {
  if (!ctx || !t) return TPCT_E_INVALID;
  t->clusters_per_bin = ctx->clusters_per_bin;
  t->tracklet_block = ctx->tracklet_block;
  t->refit_block = ctx->refit_block;
  t->precision = (int)ctx->prec;
  t->n_rows = ctx->n_rows;
  t->ms = 0.f;
  t->from_cache = 0;
  return TPCT_OK;
}

const char* tpct_last_cuda_error(const tpct_ctx* ctx) {
  return ctx ? cudaGetErrorString(ctx->last_err) : "no context";
}

}  // extern "C"

// ------------------------------------------------------------------ FMA probe
namespace {
__device__ double g_probe_sink[2];

template <class T>
__global__ void k_fma_probe(int iters, T a, T b, T* sink) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-12345.0) sink[0] = s;   // never true for these a, b; keeps the chains alive
}
}  // namespace

extern "C" tpct_status tpct_probe_fma(int use_fp64, int blocks, int iters, tpct_stream stream, float* ms) {
  if (blocks < 1 || iters < 1 || !ms) return TPCT_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  void* sink = nullptr;
  if (cudaGetSymbolAddress(&sink, g_probe_sink) != cudaSuccess) return TPCT_E_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TPCT_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TPCT_E_CUDA;
  }
  cudaEventRecord(e0, s);
  if (use_fp64) k_fma_probe<double><<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7, (double*)sink);
  else k_fma_probe<float><<<blocks, 256, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return check_cuda(e == cudaSuccess ? cudaGetLastError() : e);
}

// ------------------------------------------------------------------ conversion check
namespace {
__global__ void k_diag_convert(const float* f_in, double* d_out, const double* d_in, float* f_out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (f_in) d_out[i] = widen(f_in[i]);
    if (d_in) f_out[i] = narrow(d_in[i]);
  }
}
}  // namespace

extern "C" tpct_status tpct_diag_convert(const float* f_in, double* d_out, const double* d_in, float* f_out,
                                         int64_t n, tpct_stream stream) {
  if (n < 0 || (f_in && !d_out) || (d_in && !f_out)) return TPCT_E_INVALID;
  if (n == 0 || (!f_in && !d_in)) return TPCT_OK;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_diag_convert<<<blocks, 256, 0, (cudaStream_t)stream>>>(f_in, d_out, d_in, f_out, n);
  return check_cuda(cudaGetLastError());
}

// ------------------------------------------------------------------ allocation-free entry point
// tpct_track_static: the tracking chain of tpct_track with its scratch in a
// fixed device array of this library instead of a caller-attached workspace,
// for callers that cannot allocate device memory.  Host code must not pass
// g_static_ws itself to a kernel (on the host it is only a stand-in for the
// symbol); the device address comes from cudaGetSymbolAddress, looked up once
// per device on the first call made with that device current.
#include <mutex>

namespace {
constexpr int64_t kStaticMaxClusters = 65536;
constexpr int32_t kStaticMaxInstances = 1;
constexpr size_t kStaticBytes = (size_t)24 << 20;   // 24 MiB; the plan above needs 23.2 MiB at 152 rows
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Device address of g_static_ws on the current device (looked up once per device).
cudaError_t static_ws_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" tpct_status tpct_track_static(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n,
                                         tpct_tracks_out* out, tpct_stream stream) {
  if (!ctx) return TPCT_E_INVALID;
  tpct_status st = check_call(cl, n, out);
  if (st != TPCT_OK) return st;
  if (n > kStaticMaxClusters || cl->n_instances > kStaticMaxInstances) return TPCT_E_NOMEM;
  if (cl->n_instances < 1) return TPCT_E_INVALID;
  const Plan plan_ws = make_plan(ctx->n_rows, kStaticMaxClusters, kStaticMaxInstances, 1);
  if (carve(nullptr, plan_ws, ctx->n_rows, nullptr) > kStaticBytes) return TPCT_E_NOMEM;   // too many rows
  void* base = nullptr;
  cudaError_t e = static_ws_address(&base);
  if (e != cudaSuccess) return fail_cuda(ctx, e);
  st = ensure_grids(ctx);
  if (st != TPCT_OK) return st;
  Params p;
  fill_params(ctx, cl, n, out, (char*)base, plan_ws, &p);
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: the status word starts at zero;
  // every other array the chain reads is written earlier in the same chain
  e = cudaMemsetAsync(p.status, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return fail_cuda(ctx, e);
  ctx->launches += enqueue_track(ctx, p, s);
  return fail_cuda(ctx, cudaGetLastError());
}
