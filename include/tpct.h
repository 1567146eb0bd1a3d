/*
 * tpct.h -- C ABI of the GB300 TPC sector track finder.
 *
 * The library implements the sector track-finding part of "TPC Processing
 * (Tracking)", the step that dominates the reconstruction time tables of the
 * paper (Table 1: 99.37 % of synchronous reconstruction together with
 * clustering and compression; Tables 2 and 3: 61.41 % and 52.39 % of
 * asynchronous reconstruction).  The paper names the step but prints no
 * algorithm; the steps and constants are the stated reading (tpct_cuts):
 *   1. per sector instance and pad row, bin the clusters in a y/z grid;
 *   2. link every cluster to the best pair of clusters in the rows above and
 *      below by a straight-line criterion;
 *   3. keep reciprocal links only;
 *   4. start hits: bottoms of linked chains of at least three clusters;
 *   5. grow a tracklet from every start hit with a Kalman filter on
 *      (y, z, sin phi, tan lambda, q/pT) with a 5x5 covariance, first upward
 *      (following links, else searching the grid), then downward;
 *   6. select tracklets by owned-cluster count and shared fraction;
 *   7. refit the selected tracks (iterated, FP64 in the default precision).
 *
 * Conventions
 *   - Every pointer inside tpct_clusters, tpct_tracks_out, tpct_debug_out and
 *     every workspace pointer is DEVICE memory owned by the caller; the
 *     library never allocates or frees device memory.  Host pointers are
 *     marked "host".
 *   - A "sector instance" is one sector of one collision; a batch holds many.
 *     Clusters are grouped by instance: instance i owns cluster ids
 *     [sector_offsets[i], sector_offsets[i+1]).  A cluster id is the position
 *     in the caller's arrays.
 *   - Calls that take a stream only enqueue work and return; results are
 *     ready when the stream reaches them.  Errors the host can see are
 *     returned at once; errors found on the device (output overflow, a
 *     tracklet count beyond the workspace plan) set a sticky device status
 *     word read by tpct_last_device_status().
 *   - A context is not thread-safe; use one context per stream.
 */
#ifndef TPCT_H
#define TPCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpct_ctx tpct_ctx;
typedef struct CUstream_st* tpct_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  TPCT_OK = 0,
  TPCT_E_INVALID = 1,    /* bad argument (NULL pointer, negative size, bad geometry) */
  TPCT_E_NOMEM = 2,      /* host allocation failed, or the workspace is too small */
  TPCT_E_CAPACITY = 3,   /* device: an output buffer was too small (needed sizes written) */
  TPCT_E_CUDA = 4,       /* a CUDA runtime call failed */
  TPCT_E_TIMEOUT = 5,    /* device: a bounded wait gave up */
  TPCT_E_BUDGET = 6,     /* serving: request larger than the memory budget */
  TPCT_E_STATE = 7,      /* call not valid in the current state (e.g. no workspace) */
  TPCT_E_BOUNDS = 8      /* device: an index left its array (reported only by the bounds-checked
                            build of the library, compiled with TPCT_CHECKED) */
} tpct_status;

/* Readout geometry (host, copied by tpct_create). */
typedef struct {
  int n_rows;                 /* pad rows, 3..256 (152 for the TPC) */
  const double* row_x;        /* host [n_rows]: local x of each row [cm], strictly ascending */
  double tan_half_sector;     /* acceptance |y| <= x * tan_half_sector (tan 10 deg) */
  double z_max;               /* drift length [cm] (250) */
} tpct_geometry;

/* Tracking constants.  tpct_default_cuts() fills the stated readings. */
typedef struct {
  double nf_wy, nf_wz;        /* neighbour window |dy|,|dz| <= w * dx            (2, 2) */
  double nf_dmax;             /* accept best pair iff D <= nf_dmax [cm^2]        (0.25) */
  double s_max;               /* |sin phi| limit                                  (0.999) */
  double edge_margin;         /* stop when |y| > x tan + edge_margin [cm]         (1) */
  double search_k;            /* grid search window in sigmas                    (5) */
  double chi2_max;            /* per-cluster chi2 cut                            (25) */
  int max_miss;               /* stop after more consecutive missed rows         (8) */
  int n_min;                  /* minimum owned clusters per track                (20) */
  double f_shared;            /* maximum shared fraction                         (0.1) */
  int n_refit;                /* refit passes                                    (3) */
  double sig_readout;         /* cluster sigma at drift length 0 [cm]            (0.1) */
  double sig_cathode;         /* cluster sigma at drift length z_max [cm]        (0.1) */
  double c_s, c_t, c_qpt;     /* initial variances of sin phi, tan l, q/pT      (1, 1, 100) */
  double c_yz_refit;          /* refit prior variance of y, z [cm^2]            (100) */
  double c_qpt_refit;         /* refit prior variance of q/pT                    (1e4) */
} tpct_cuts;

/* Arithmetic of steps 2-7.  FP32: everything in float.  MIXED (default):
 * neighbour tests, grid search and helix-transport arithmetic in float; track
 * state, covariance, Kalman update and the whole refit in double.  FP64: all
 * double.  MIXED_DF: as MIXED, but the tracklet state and covariance are
 * double-float pairs (48-bit significand) on the FP32 pipes, which GB300 runs
 * at 64x its FP64 rate; the refit stays double. */
typedef enum { TPCT_PREC_FP32 = 0, TPCT_PREC_MIXED = 1, TPCT_PREC_FP64 = 2, TPCT_PREC_MIXED_DF = 3 } tpct_precision;

/* Input clusters (device, caller-owned, read-only). */
typedef struct {
  const float* x;                 /* [n] local x; used only when row == NULL (nearest row) */
  const float* y;                 /* [n] local y [cm] */
  const float* z;                 /* [n] z [cm] */
  const uint16_t* charge;         /* [n] may be NULL (carried, not used by tracking) */
  const uint8_t* row;             /* [n] pad row, or NULL */
  const int64_t* sector_offsets;  /* [n_instances+1], non-decreasing, [0] = 0, [n_instances] = n */
  int32_t n_instances;
} tpct_clusters;

/* Output tracks (device, caller-owned).  Tracks are ordered by (instance,
 * rank of the start hit); each holds its owned clusters, row-ascending. */
typedef struct {
  int32_t capacity_tracks;        /* rows of the per-track arrays */
  int32_t capacity_ids;           /* length of cluster_ids */
  int32_t* n_tracks;              /* [1] number of tracks (also written on overflow) */
  int32_t* n_ids;                 /* [1] total cluster ids (also written on overflow) */
  int32_t* instance;              /* [K] sector instance */
  int32_t* n_cl;                  /* [K] owned clusters */
  int32_t* offset;                /* [K] first entry in cluster_ids */
  int32_t* ndf;                   /* [K] 2 n_cl - 5 */
  int32_t* status;                /* [K] 0 = refit converged, 1 = transport failed */
  double* x_ref;                  /* [K] x of the innermost cluster */
  double* param;                  /* [K*5] y, z, sin phi, tan lambda, q/pT at x_ref */
  double* cov;                    /* [K*15] covariance, lower triangle row-major */
  double* chi2;                   /* [K] */
  int32_t* cluster_ids;           /* [capacity_ids] */
} tpct_tracks_out;

/* Intermediate results for parity checks (device, caller-owned; any pointer
 * may be NULL to skip it).  Ids are input cluster ids. */
typedef struct {
  int32_t* up;                    /* [n] best neighbour in row r+1 or -1 */
  int32_t* down;                  /* [n] best neighbour in row r-1 or -1 */
  int32_t* upc;                   /* [n] reciprocal up link or -1 */
  int32_t* downc;                 /* [n] reciprocal down link or -1 */
  uint32_t* weight;               /* [n] selection weight W */
  int32_t capacity_tracklets;
  int32_t* n_tracklets;           /* [1] */
  int32_t* tl_start;              /* [T] start hit id, in (instance, row, id) order */
  int32_t* tl_nhits;              /* [T] */
  int32_t* tl_hits;               /* [T*n_rows] row-indexed cluster ids, -1 = none */
  double* tl_param;               /* [T*5] state at the innermost hit */
  int32_t* tl_row_ref;            /* [T] row of the innermost hit */
  int32_t* tr_tracklet;           /* [K] tracklet of each output track (K <= capacity_tracklets) */
  int64_t* counters;              /* [4] totals over tracklets: helix steps, Kalman updates,
                                     chi2 tests, grid candidates examined (added to) */
} tpct_debug_out;

/* ---------------------------------------------------------------- context */
/* Fills the stated readings of the method's constants (the values in
 * brackets above).  Source: the paper names the tracking step (Tables 1-3)
 * but fixes none of its constants; these are the readings every result of
 * this library is defined by. */
void tpct_default_cuts(tpct_cuts* cuts);

/* Fills the TPC readout the workloads use: 152 pad rows (63 at 0.75 cm pitch
 * from x = 85.2 cm, 64 at 1.0 cm from 135.1 cm, 25 at 1.5 cm from 199.4 cm),
 * tan 10 deg sector acceptance, 250 cm drift.  row_x points to static storage
 * of the library.  Source: the TPC whose processing Tables 1-3 time; the
 * radii are a reading (the paper gives no geometry). */
void tpct_default_geometry(tpct_geometry* geometry);

/* Create a context for one geometry, field and cut set.  bz_tesla: field
 * along +z.  Returns TPCT_E_INVALID for a bad geometry or cut set.  Source:
 * the sector tracking of "TPC Processing (Tracking)", Tables 1-3; the
 * precision modes are this library's (the paper prints no arithmetic). */
tpct_status tpct_create(const tpct_geometry* geometry, double bz_tesla, const tpct_cuts* cuts,
                        tpct_precision precision, tpct_ctx** out);
void tpct_destroy(tpct_ctx* ctx);

/* Tuning knobs that never change results (only speed): clusters per grid
 * bin (>= 1), threads per block of the tracklet and refit kernels (a
 * multiple of 32, at most 256).  0 = default.  No counterpart in the paper
 * (launch shapes of this GPU implementation). */
tpct_status tpct_set_tuning(tpct_ctx* ctx, int clusters_per_bin, int tracklet_block, int refit_block);

/* Launch shapes of a context (no counterpart in the paper). */
typedef struct {
  int clusters_per_bin, tracklet_block, refit_block;
  int precision, n_rows;          /* of the context (read-only here) */
  float ms;                       /* autotuner: median time of the chosen shapes */
  int from_cache;                 /* autotuner: 1 if read from the cache file */
} tpct_tuning;
tpct_status tpct_get_tuning(const tpct_ctx* ctx, tpct_tuning* out);

/* Autotuner: times tpct_track on the given workload for candidate launch
 * shapes (coordinate descent over clusters per bin 1/2/4/8 and tracklet and
 * refit blocks of 64/128/256 threads), keeps the fastest in the context and
 * appends it to the text file cache_path (may be NULL) under a key of device
 * name, precision, rows and the size class (log2 clusters per instance, log2
 * instances).  A cached key is reused without timing.  Synchronises `stream`;
 * needs an attached workspace; overwrites `out`.  The shapes never change
 * results.  No counterpart in the paper (this implementation's autotuner). */
tpct_status tpct_autotune(tpct_ctx* ctx, const tpct_clusters* clusters, int64_t n, tpct_tracks_out* out,
                          tpct_stream stream, const char* cache_path, tpct_tuning* result);

/* ---------------------------------------------------------------- workspace */
/* Device bytes needed to track up to max_clusters clusters in up to
 * max_instances sector instances in one call (this library's memory plan;
 * no counterpart in the paper). */
size_t tpct_workspace_bytes(const tpct_ctx* ctx, int64_t max_clusters, int32_t max_instances);
/* Attach caller-owned device memory (256-byte aligned, >= the size above).
 * Touches no device memory: the context's status word in it is cleared in
 * stream order by the next tracking call. */
tpct_status tpct_set_workspace(tpct_ctx* ctx, void* device_ptr, size_t bytes,
                               int64_t max_clusters, int32_t max_instances);

/* ---------------------------------------------------------------- tracking */
/* Track n clusters (all instances of `clusters`) on `stream`: the plain
 * form, one launch per step.  Source: steps 1-7 above, the sector tracking of
 * "TPC Processing (Tracking)" (Tables 1-3), with the stated readings of
 * tpct_cuts.  A cluster whose row[] is >= the geometry's n_rows is tracked on
 * the last row and makes tpct_last_device_status return TPCT_E_INVALID. */
tpct_status tpct_track(tpct_ctx* ctx, const tpct_clusters* clusters, int64_t n,
                       tpct_tracks_out* out, tpct_stream stream);

/* Batched form: the same result as tpct_track on the same batch, run by
 * persistent kernels that pull work items from device queues, captured once
 * into a CUDA graph per (n, n_instances) and replayed.  Source: the same
 * steps; batching many collisions into one call is this implementation's
 * (the paper's farm processes whole time frames per GPU, Section 1). */
tpct_status tpct_track_batch(tpct_ctx* ctx, const tpct_clusters* clusters, int64_t n,
                             tpct_tracks_out* out, tpct_stream stream);

/* Timing hooks (no counterpart in the paper): n_events = 7 CUDA events (cudaEvent_t) recorded on the
 * tracking stream at the step boundaries: before step 1, after the grid
 * (step 1), neighbours (2), cleaning and start hits (3-4), tracklets (5),
 * selection (6) and refit (7).  Inside the batched form's graph they are
 * event-record nodes, re-pointed to the events given here on every call.
 * n_events = 0 disables.  The events stay owned by the caller. */
tpct_status tpct_set_stage_events(tpct_ctx* ctx, void* const* events, int n_events);

/* Allocation-free variant of tpct_track (no counterpart in the paper).  For
 * callers that cannot allocate device memory -- a plug-in that receives only
 * its input and output buffers from a host framework that owns all device
 * memory, a process whose memory is fully planned at start-up, or a latency-
 * critical path where a cudaMalloc would synchronise the device -- and so
 * cannot attach a workspace.  The scratch is a fixed 24 MiB array inside this
 * library, held on every GPU that loads the library until the process exits;
 * it fits ONE sector instance of at most 65536 clusters (n_instances must be
 * 1).  Larger requests return TPCT_E_NOMEM, more instances too; contexts with
 * more pad rows than fit return TPCT_E_NOMEM.  The caller still owns
 * `clusters` and `out`.  The call allocates nothing (no cudaMalloc, no
 * cudaFree) and enqueues the same kernels as tpct_track on `stream`.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * outside any stream capture.  All calls share the one array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (other streams,
 * other threads, other contexts) race and corrupt each other -- serialise
 * them.  The device status of such a call is not kept: an output overflow
 * shows as *n_tracks > capacity_tracks or *n_ids > capacity_ids, a cluster
 * whose row[] is >= n_rows is tracked on the last row without a warning, and
 * tpct_last_device_status / tpct_debug_export do not describe the call.  The
 * looked-up address is kept for the life of the process: do not call this
 * entry point on a device after cudaDeviceReset on it. */
tpct_status tpct_track_static(tpct_ctx* ctx, const tpct_clusters* clusters, int64_t n,
                              tpct_tracks_out* out, tpct_stream stream);

/* Copy intermediate arrays of the last tpct_track / tpct_track_batch call on
 * this context (enqueued on `stream`): the links, start hits and tracklets of
 * steps 2-6, for parity checks against a reference implementation. */
tpct_status tpct_debug_export(tpct_ctx* ctx, tpct_debug_out* dbg, tpct_stream stream);

/* Sticky device status of this context (synchronises the context's last
 * stream): TPCT_OK; TPCT_E_BOUNDS if an index left its array (bounds-checked
 * build only); TPCT_E_CAPACITY if an output or the tracklet plan overflowed;
 * TPCT_E_INVALID if an input row was outside the geometry.
 * Reading it clears it.  (No kernel waits for another, so no call on a
 * context times out on the device; TPCT_E_TIMEOUT comes only from
 * tpct_server_wait.)  Error reporting of this library (no counterpart in the
 * paper). */
tpct_status tpct_last_device_status(tpct_ctx* ctx);

/* Text of a status code (static storage). */
const char* tpct_status_str(tpct_status s);

/* Text of the CUDA error behind the context's last TPCT_E_CUDA (host-owned, static). */
const char* tpct_last_cuda_error(const tpct_ctx* ctx);

/* ---------------------------------------------------------------- cross-sector merging */
/* A particle crossing a sector boundary leaves one track in each sector;
 * merging joins them and refits each chain across the sector frames (the
 * tracking step of "TPC Processing (Tracking)", Tables 1-3, spans the whole
 * TPC).  Reading: for tracks a, b in adjacent sectors of the same side and
 * collision, the one whose reference point has the smaller radius is inner;
 * a pair is tested iff |tanl_a - tanl_b| <= max_dtanl and the inner track's
 * outermost and the outer track's innermost clusters are at most max_gap
 * apart in the transverse plane; chi2 compares the inner track, transported
 * to its outermost cluster, rotated into the outer frame and transported to
 * the outer reference x, with the outer track; chi2 <= chi2_max is accepted;
 * mutual best partners (smallest chi2, ties to the smaller index) are linked;
 * chains are refitted in FP64 (reference-trajectory Kalman filter, 3 passes,
 * frame rotation at each sector change). */
typedef struct {
  double chi2_max;            /* (50) */
  double max_dtanl;           /* (0.1) */
  double max_gap;             /* [cm] (40) */
  double alpha0, dalpha;      /* sector k centred at alpha0 + (k mod 18) dalpha [rad] (10, 20 deg) */
} tpct_merge_cuts;
/* Fills the merging readings above (source: the tracking of Tables 1-3 spans
 * the whole TPC; the paper fixes no merging constant). */
void tpct_default_merge_cuts(tpct_merge_cuts* cuts);

/* Merged chains (device, caller-owned), ordered by head (innermost) track.
 * Parameters are at the innermost cluster in the head track's sector frame. */
typedef struct {
  int32_t capacity_chains, capacity_ids, capacity_segs;
  int32_t* n_chains;          /* [1] (also written on overflow) */
  int32_t* n_ids;             /* [1] */
  int32_t* n_segs;            /* [1] */
  int32_t* head;              /* [M] innermost track */
  int32_t* n_seg;             /* [M] tracks in the chain */
  int32_t* seg_offset;        /* [M] first entry in segs */
  int32_t* segs;              /* [capacity_segs] track indices, inner to outer */
  int32_t* instance;          /* [M] sector instance of the head */
  int32_t* n_cl;              /* [M] */
  int32_t* offset;            /* [M] first entry in cluster_ids */
  int32_t* ndf;               /* [M] */
  int32_t* status;            /* [M] 0 = refit converged, 1 = transport or rotation failed */
  double* x_ref;              /* [M] */
  double* param;              /* [M*5] */
  double* cov;                /* [M*15] */
  double* chi2;               /* [M] */
  int32_t* cluster_ids;       /* [capacity_ids] inner track first, rows ascending in each track */
  int32_t* link_out;          /* [capacity of the input tracks] outer partner of every track or -1 (may be NULL) */
  int32_t* link_in;           /* [capacity of the input tracks] inner partner or -1 (may be NULL) */
} tpct_chains_out;

/* Device workspace of tpct_merge for up to max_tracks input tracks (this
 * library's memory plan). */
size_t tpct_merge_workspace_bytes(int32_t max_tracks, int32_t n_instances, int32_t n_events);

/* Source: cross-sector merging, part of "TPC Processing (Tracking)",
 * Tables 1-3, with the readings above.
 * Merge the output of tpct_track / tpct_track_batch (`tracks`, on the same
 * `clusters`; tracks ordered by instance).  inst_sector, inst_event: device
 * [n_instances] sector number (0..35) and collision (0..n_events-1) of every
 * instance.  Asynchronous on `stream`; an overflow of `out` shows as
 * *n_chains > capacity_chains (or ids, segs): those counters are always
 * written, the rows that do not fit are not.  TPCT_E_NOMEM if the workspace
 * is smaller than tpct_merge_workspace_bytes(tracks->capacity_tracks, ...). */
tpct_status tpct_merge(tpct_ctx* ctx, const tpct_clusters* clusters, const int32_t* inst_sector,
                       const int32_t* inst_event, int32_t n_events, const tpct_tracks_out* tracks,
                       const tpct_merge_cuts* cuts, void* workspace, size_t workspace_bytes,
                       tpct_chains_out* out, tpct_stream stream);

/* ---------------------------------------------------------------- cluster finding */
/* TPC cluster finding, the step upstream of track finding: zero-suppressed
 * digits -> clusters.  The paper names clustering inside "TPC Processing
 * (Tracking, Clustering, Compression)" (Table 1, 99.37 % of synchronous
 * reconstruction) without describing it.  Readings: row r has
 * n_pad = 2 ceil(x_r tan_half / pitch - 1e-9) pads (pitch: pad_pitch_inner
 * below n_inner_rows, else pad_pitch_outer) and n_time time bins; a digit of
 * charge q at (pad p, time t) is a PEAK iff q >= q_peak_min, q > each of its 8
 * neighbours that comes before it in (time, pad) order and q >= the others
 * (cells without a digit hold 0); a peak is DROPPED iff a higher peak (equal:
 * the earlier one) lies at Chebyshev distance 2 and the cell one step from
 * the peak towards it holds >= q - valley_delta (no valley between them); a
 * kept peak's CLUSTER sums its 3x3 cells plus every cell of the distance-2
 * ring whose inner neighbour towards the peak holds at least its charge:
 * pad / time = peak + charge-weighted mean offset, sigma_pad / sigma_time =
 * the charge-weighted standard deviation, q_tot = the sum, q_max = the peak
 * charge, y = (pad + 0.5 - n_pad/2) * pitch, z = +-(z_max - (time + 0.5) *
 * time_bin) on side A / C (instance sector < 18 / >= 18), x = the row
 * radius of the context's geometry. */
typedef struct {
  double pad_pitch_inner;      /* [cm] (0.4) */
  double pad_pitch_outer;      /* [cm] (0.6) */
  int32_t n_inner_rows;        /* rows with the inner pitch (63) */
  double time_bin;             /* drift length per time bin [cm] (0.5) */
  int32_t n_time;              /* time bins per row (500); at most 512, every row at most 252 pads */
  int32_t q_peak_min;          /* (7) */
  int32_t valley_delta;        /* (2) */
} tpct_cf_params;
/* Fills the cluster-finding readings above (source: clustering inside "TPC
 * Processing", Table 1; the paper fixes no constant). */
void tpct_default_cf_params(tpct_cf_params* p);

/* Digits (device, caller-owned, read-only): SoA, grouped by (instance, row),
 * any order inside a row, each (pad, time) cell at most once per row, ADC
 * values below 32768.  The kernel works on tiles of 128 time bins of a row:
 * at most 2048 clusters with their peak in one tile (more:
 * TPCT_CF_ROW_OVERFLOW, the rest ignored). */
typedef struct {
  const uint16_t *pad, *time, *adc;   /* [row_offsets[last]]; may be NULL when there are no digits */
  const int64_t* row_offsets;  /* [n_instances * n_rows + 1] */
  const int32_t* inst_sector;  /* [n_instances] sector number 0..35 of each instance */
  int32_t n_instances;
} tpct_digits;

/* Clusters (device, caller-owned): SoA in (instance, row) order, inside a
 * row in (time, pad) order of the peaks; x, y, z are the tracker's
 * cluster input (tpct_clusters) for these instances. */
typedef struct {
  int32_t capacity;
  int32_t* n_clusters;         /* [1] always written (may exceed capacity) */
  uint32_t* status;            /* [1] TPCT_CF_* bits, zeroed by each call */
  float *x, *y, *z, *pad, *time, *sigma_pad, *sigma_time;
  uint32_t* q_tot;
  uint16_t* q_max;
  uint8_t *row, *flags;        /* flags: 1 = peak on the first/last pad, 2 = on the first/last time bin */
  int64_t* inst_offsets;       /* [n_instances + 1] first cluster of each instance (may be NULL) */
} tpct_cf_out;
#define TPCT_CF_BAD_DIGIT 1u      /* a digit outside its row's pads or time bins, or ADC >= 32768 (skipped) */
#define TPCT_CF_TIMEOUT 2u        /* (not raised: the kernels do not wait for one another) */
#define TPCT_CF_ROW_OVERFLOW 4u   /* a tile of a row held more clusters than the limit above */
#define TPCT_CF_WORKSPACE 16u     /* the workspace was sized for fewer digits than the rows hold (rows skipped) */
#define TPCT_CF_CAPACITY 8u       /* more clusters than capacity: *n_clusters is the size needed, the
                                     output arrays hold no defined result */

/* Device workspace of tpct_find_clusters for n_digits digits (the sum over
 * all rows) of n_instances instances and an output of `capacity` clusters
 * (the digits are sorted by time bin and the clusters staged there before
 * they are put in order). */
size_t tpct_cf_workspace_bytes(int64_t n_digits, int32_t n_instances, int32_t n_rows, int32_t capacity);

/* Source: the clustering of "TPC Processing (Tracking, Clustering,
 * Compression)", Table 1, with the readings above.
 * Find the clusters of all rows of all instances; asynchronous on `stream`.
 * TPCT_E_INVALID for bad arguments or readout parameters that give a row more
 * than 252 pads or more than 512 time bins; TPCT_E_NOMEM if the workspace
 * (256-byte aligned) cannot hold even the per-item and staging areas (the
 * rest holds the sorted digits: rows that end beyond it are skipped and
 * raise TPCT_CF_WORKSPACE).  Device conditions are reported in
 * *out->status. */
tpct_status tpct_find_clusters(tpct_ctx* ctx, const tpct_digits* digits, const tpct_cf_params* params,
                               void* workspace, size_t workspace_bytes, tpct_cf_out* out, tpct_stream stream);

/* ---------------------------------------------------------------- track-model compression */
/* Compression of a frame's clusters with the tracks as the model, and its
 * decoding (the paper counts compression inside "TPC Processing (Tracking,
 * Clustering, Compression)", Table 1, and reports a 1.2-3 % faster offline
 * reconstruction from GPU track-model decoding, Section 2; the format is a
 * reading): positions on a 50 um grid (Y = rint(200 y), Z = rint(200 z), row
 * X = rint(200 x_r)); per track (clusters rows ascending): count, first row,
 * Y0, Z0, charge, then per cluster the rows skipped, the residuals of Y and Z
 * against the value predicted from the track's previous decoded clusters
 * (previous value; the line through two; the parabola through three, exact
 * integer arithmetic, quotient rounded half away from zero) and the charge;
 * clusters in no track, per (instance, row) sorted by (Y, Z, charge): count,
 * Y (first absolute, then differences), Z, charge; every value a LEB128
 * varint (signed: zigzag); tracks first, then the rows.  Decoding returns
 * x = row radius, y = Y/200, z = Z/200 (float), charge, row, in the order
 * tracks (clusters row-ascending) then rows. */
typedef struct {
  int64_t capacity;            /* bytes of data */
  uint8_t* data;
  int64_t* n_bytes;            /* [1] the stream's size, always written (may exceed capacity: nothing written) */
  int64_t* track_offsets;      /* [tracks->capacity_tracks + 1] byte offset of every track, then the end of the tracks */
  int64_t* row_offsets;        /* [n_instances * n_rows + 1] byte offset of every (instance, row) block, then the end */
} tpct_tm_stream;
typedef struct {
  int64_t capacity;            /* clusters */
  int64_t* n;                  /* [1] clusters in the stream, always written (may exceed capacity) */
  float *x, *y, *z;
  uint16_t* charge;
  uint8_t* row;
  uint32_t* status;            /* [1] TPCT_TD_* bits of this call (cleared by the call) */
} tpct_tm_decoded;
enum {
  TPCT_TD_BAD_STREAM = 1u,     /* an item's offsets leave the stream, a varint runs past its item or beyond 10
                                  bytes, a count needs more bytes than its item holds, a row lies outside the
                                  geometry or a charge above 65535: that item decodes no further, the output is
                                  not a valid decoding */
  TPCT_TD_CAPACITY = 2u        /* more clusters than out->capacity: only the first capacity are written */
};
/* Device workspace of tpct_tm_encode (this library's memory plan). */
size_t tpct_tm_encode_workspace_bytes(int64_t n_clusters, int32_t capacity_tracks, int32_t n_instances, int32_t n_rows);
/* Source: the compression of "TPC Processing", Table 1, with the format
 * readings above.
 * Encode the clusters (device; row[] required) with the tracks of
 * tpct_track / tpct_track_batch on them (device; n_tracks read on the device).
 * TPCT_E_NOMEM if the workspace is too small. */
tpct_status tpct_tm_encode(tpct_ctx* ctx, const tpct_clusters* clusters, int64_t n, const tpct_tracks_out* tracks,
                           void* workspace, size_t workspace_bytes, tpct_tm_stream* out, tpct_stream stream);
/* Device workspace of tpct_tm_decode (this library's memory plan). */
size_t tpct_tm_decode_workspace_bytes(int32_t n_tracks, int32_t n_instances, int32_t n_rows);
/* Source: GPU track-model decoding, Section 2 (1.2-3 % faster offline
 * reconstruction), with the format readings above.
 * Decode a stream (device data and offsets; n_bytes, n_tracks and n_instances
 * on the host).  data holds n_bytes bytes; track_offsets[n_tracks + 1] and
 * row_offsets[n_instances * n_rows + 1] delimit every item (the layout
 * tpct_tm_encode writes).  The stream is not trusted: every read stays inside
 * [0, n_bytes) and inside its item, and a malformed item sets
 * TPCT_TD_BAD_STREAM in out->status instead (no read or write outside the
 * buffers).  TPCT_E_INVALID on bad arguments, TPCT_E_NOMEM if the workspace
 * is too small. */
tpct_status tpct_tm_decode(tpct_ctx* ctx, const uint8_t* data, int64_t n_bytes, const int64_t* track_offsets,
                           int32_t n_tracks, const int64_t* row_offsets, int32_t n_instances, void* workspace,
                           size_t workspace_bytes, tpct_tm_decoded* out, tpct_stream stream);

/* ---------------------------------------------------------------- publishing-rate control */
/* Pacing of an offline source that feeds frames into a processing chain
 * (host-side; no device code).  Section 3 of the paper: publishing as fast as
 * possible and throttling only by the collisions in flight makes work arrive
 * in waves that leave stages idle behind a slower serial one; ALICE smooths
 * the publishing rate with a heuristic that slowly shortens the delay between
 * publications until back pressure appears.  Reading implemented here:
 *   NAIVE   publish whenever fewer than max_in_flight frames are in flight
 *           (published and not yet consumed);
 *   SMOOTH  also wait until `delay` has passed since the last publication
 *           and no frames wait downstream (backlog == 0);
 *           after every consumed frame delay *= (1 - decrease) if no back
 *           pressure was seen since the previous one, else delay *=
 *           (1 + increase); back pressure = a publication attempt met the
 *           in-flight limit or frames waiting downstream (backlog > 0);
 *           delay stays in [min_delay_s, max_delay_s].
 * The caller passes its own clock (seconds); the pacer keeps no thread. */
typedef enum { TPCT_PUBLISH_NAIVE = 0, TPCT_PUBLISH_SMOOTH = 1 } tpct_publish_policy;
typedef struct {
  tpct_publish_policy policy;  /* (SMOOTH) */
  int32_t max_in_flight;       /* (8) */
  double initial_delay_s;      /* (0.05) */
  double decrease;             /* (0.02) */
  double increase;             /* (0.05) */
  double min_delay_s, max_delay_s;   /* (0, 10) */
} tpct_pacer_config;
typedef struct tpct_pacer tpct_pacer;
/* Fills the defaults in brackets above (readings of Section 3). */
void tpct_default_pacer_config(tpct_pacer_config* config);
/* Source of the pacer calls: Section 3 (publishing-rate smoothing), with
 * the reading above.  TPCT_E_INVALID for a bad configuration. */
tpct_status tpct_pacer_create(const tpct_pacer_config* config, tpct_pacer** out);
/* Frees the pacer (host memory). */
void tpct_pacer_destroy(tpct_pacer* pacer);
/* 1: publish now (recorded as published); 0: not now, *wait_s = the time
 * until the delay has passed (0 when waiting for a consumed frame). */
int tpct_pacer_try_publish(tpct_pacer* pacer, double now_s, int32_t in_flight, int32_t backlog, double* wait_s);
/* A frame left the chain; adapts the delay (SMOOTH). */
void tpct_pacer_on_consumed(tpct_pacer* pacer, double now_s, int32_t in_flight, int32_t backlog);
/* Current delay between publications [s] (SMOOTH). */
double tpct_pacer_delay(const tpct_pacer* pacer);
/* Number of times back pressure started. */
int64_t tpct_pacer_pressure_events(const tpct_pacer* pacer);

/* ---------------------------------------------------------------- serving */
/* A serving runtime: time frames (batches of sector instances) submitted from
 * host memory are tracked concurrently in up to n_slots streams.  A frame is
 * admitted, in arrival order, when a slot is idle and the caller's device
 * arena has room for its inputs, workspace and outputs; inputs and workspace
 * are returned to the arena the moment the frame finishes, so frames queued
 * behind it start while others are still running (continuous batching).  A
 * scheduler thread of the library does the admission.  Outputs stay in the
 * arena until tpct_server_release.  A frame's results do not depend on what
 * else runs: every frame has its own context, workspace and outputs. */
typedef struct tpct_server tpct_server;

typedef struct {
  int n_slots;                 /* frames on the device at once, 1..64 (one stream + context each) */
  void* arena;                 /* device memory budget, caller-owned, 256-byte aligned */
  size_t arena_bytes;
} tpct_server_config;

typedef struct {
  /* HOST pointers, caller-owned, read until the frame has finished; pinned
   * (page-locked) memory lets the copies overlap other frames' work */
  const float *x, *y, *z;
  const uint16_t* charge;          /* may be NULL */
  const uint8_t* row;              /* may be NULL (then x gives the row) */
  const int64_t* sector_offsets;   /* [n_instances+1] */
  int32_t n_instances;
  int64_t n;
} tpct_host_frame;

typedef struct {
  int32_t state;                   /* 0 queued, 1 running, 2 done, 3 failed */
  tpct_status status;              /* of a finished or failed frame */
  int32_t n_tracks, n_ids;         /* of a finished frame */
  double queue_us;                 /* submit -> admission (-1 while queued) */
  double latency_us;               /* submit -> finish observed by the scheduler (-1 before) */
} tpct_frame_info;

typedef struct {
  /* HOST arrays, caller-owned; same layout as tpct_tracks_out */
  int32_t capacity_tracks, capacity_ids;
  int32_t n_tracks, n_ids;         /* written by tpct_server_fetch */
  int32_t *instance, *n_cl, *offset, *ndf, *status;
  double *x_ref, *param, *cov, *chi2;
  int32_t* cluster_ids;
} tpct_host_tracks;

typedef struct {
  int64_t submitted, completed, retries, clusters_completed;
  int32_t queued, in_flight, peak_in_flight;
  uint64_t bytes_in_use, peak_bytes, budget_bytes;
} tpct_server_stats;

/* Source of the serving calls: continuous batching of time frames is this
 * library's reading of serving; the paper's Section 3 supplies the idea of
 * admitting work by the resources in flight.  TPCT_E_INVALID for bad
 * arguments; the arena is the caller's and is never freed here. */
tpct_status tpct_server_create(const tpct_geometry* geometry, double bz_tesla, const tpct_cuts* cuts,
                               tpct_precision precision, const tpct_server_config* config,
                               tpct_server** out);
/* Stops the scheduler after the frames on the device finish; outstanding
 * tickets become invalid. */
void tpct_server_destroy(tpct_server* server);
/* Queue a frame; TPCT_E_BUDGET if it could never fit the arena. */
tpct_status tpct_server_submit(tpct_server* server, const tpct_host_frame* frame, uint64_t* ticket);
/* State of a frame (never blocks). */
tpct_status tpct_server_poll(tpct_server* server, uint64_t ticket, tpct_frame_info* info);
/* Blocks until the frame is done or failed (TPCT_E_TIMEOUT after timeout_s seconds). */
tpct_status tpct_server_wait(tpct_server* server, uint64_t ticket, double timeout_s);
/* Copy a finished frame's tracks to host arrays (TPCT_E_CAPACITY if they do
 * not fit; n_tracks and n_ids are written either way). */
tpct_status tpct_server_fetch(tpct_server* server, uint64_t ticket, tpct_host_tracks* out);
/* Return a finished frame's outputs to the arena and forget the ticket. */
tpct_status tpct_server_release(tpct_server* server, uint64_t ticket);
/* Counters of the server since creation. */
tpct_status tpct_server_get_stats(tpct_server* server, tpct_server_stats* out);

/* Diagnostics (launch counts, pipe probes, a conversion check) are declared
 * in tpct_diag.h. */

#ifdef __cplusplus
}
#endif
#endif
