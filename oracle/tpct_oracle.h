/*
 * tpct_oracle.h -- plain, single-threaded FP64 CPU oracle of TPC sector track
 * finding.  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library and
 * is never called by it.  It shares no code, header or constant table with
 * the CUDA path.
 *
 * The method is the "TPC Processing (Tracking)" step that dominates the time
 * tables of the paper (Table 1: 99.37 % of synchronous reconstruction
 * together with clustering and compression; Tables 2-3: 61.41 % and 52.39 %
 * of asynchronous reconstruction).  The paper names the step but does not
 * describe the algorithm; every constant and tie-break below is a stated
 * reading, passed in through orc_cuts.
 *
 * Cluster ids are positions in the caller's arrays.  All sizes are int64.
 */
#ifndef TPCT_ORACLE_H
#define TPCT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ROWS 256

typedef struct {
  int n_rows;               /* pad rows, <= ORC_MAX_ROWS */
  const double* row_x;      /* [n_rows] local x of each row, ascending (copied) */
  double tan_half_sector;   /* tan(10 deg): sector acceptance |y| <= x tan */
  double z_max;             /* drift length (250 cm) */
} orc_geometry;

typedef struct {
  double bz;                /* field along +z [T] */
  double nf_wy, nf_wz;      /* neighbour windows |dy| <= wy dx, |dz| <= wz dx */
  double nf_dmax;           /* accept best pair iff D <= dmax [cm^2] */
  double s_max;             /* |sin phi| limit */
  double edge_margin;       /* tracklets stop when |y| > x tan + edge_margin [cm] */
  double search_k;          /* search window in sigmas */
  double chi2_max;          /* per-hit chi2 cut */
  int max_miss;             /* stop after more than this many consecutive misses */
  int n_min;                /* minimum owned clusters of a track */
  double f_shared;          /* maximum shared fraction */
  int n_refit;              /* refit passes */
  double sig_readout;       /* cluster sigma at drift length 0 */
  double sig_cathode;       /* cluster sigma at drift length z_max */
  double c_s, c_t, c_qpt;   /* initial variances of sin phi, tan lambda, q/pT */
  double c_yz_refit;        /* refit prior variance of y and z [cm^2] (diffuse) */
  double c_qpt_refit;       /* refit prior variance of q/pT (diffuse) */
} orc_cuts;

typedef struct orc_result orc_result;

/*
 * Track all sector instances.  inst_offsets[n_inst+1] delimit each instance's
 * clusters.  y, z: local coordinates (double).  row: pad row of each cluster,
 * or NULL to take the row whose x is nearest to x[] (x may be NULL if row is
 * given).  brute_force_nf != 0 replaces the neighbour-window scan by an
 * all-pairs scan of the rows.  Returns NULL on allocation failure or invalid
 * arguments.
 */
orc_result* orc_track(const orc_geometry* g, const orc_cuts* c, int64_t n_inst,
                      const int64_t* inst_offsets, const double* x, const double* y,
                      const double* z, const int32_t* row, int brute_force_nf);
void orc_free(orc_result* r);

/* Array access: orc_count gives the element count, orc_array the pointer. */
enum {
  ORC_UP = 0, ORC_DOWN, ORC_UPC, ORC_DOWNC,      /* int32 [N]            */
  ORC_NF_MARGIN,                                 /* double [N]           */
  ORC_WEIGHT,                                    /* uint32 [N]           */
  ORC_TL_INST, ORC_TL_START, ORC_TL_NHITS,       /* int32 [T]            */
  ORC_TL_STOP_UP, ORC_TL_STOP_DOWN, ORC_TL_ROWREF,/* int32 [T]           */
  ORC_TL_XREF, ORC_TL_MARGIN,                    /* double [T]           */
  ORC_TL_PARAM,                                  /* double [T*5]         */
  ORC_TL_HITS,                                   /* int32 [T*n_rows] row-indexed, -1 = none */
  ORC_TR_INST, ORC_TR_TRACKLET, ORC_TR_NCL, ORC_TR_OFFSET, ORC_TR_NDF, ORC_TR_STATUS, /* int32 [K] */
  ORC_TR_XREF, ORC_TR_CHI2, ORC_TR_MARGIN,       /* double [K]           */
  ORC_TR_PARAM,                                  /* double [K*5]         */
  ORC_TR_COV,                                    /* double [K*15] packed lower triangle, row-major */
  ORC_TR_IDS,                                    /* int32 [sum ncl]      */
  ORC_N_ARRAYS
};
int64_t orc_count(const orc_result* r, int which);
const void* orc_array(const orc_result* r, int which);

/* ---------------------------------------------------------------- cross-sector merging */
typedef struct {
  double chi2_max;         /* accept a pair iff chi2 <= chi2_max */
  double max_dtanl;        /* consider a pair only if |tanl_a - tanl_b| <= max_dtanl ... */
  double max_gap;          /* ... and the facing end clusters are <= max_gap apart (transverse, cm) */
  double alpha0, dalpha;   /* sector k is centred at alpha0 + (k mod 18) dalpha [rad] */
} orc_merge_cuts;

typedef struct orc_merge_result orc_merge_result;

/* Merge the sector tracks of `tracks` (from orc_track on the same clusters)
 * across adjacent sectors of the same side and collision.  inst_sector,
 * inst_event: sector number and collision of every instance.  row: pad row of
 * every cluster.  Returns NULL on allocation failure or bad arguments. */
orc_merge_result* orc_merge(const orc_geometry* g, const orc_cuts* c, const orc_merge_cuts* mc,
                            const orc_result* tracks, int64_t n_inst, const int32_t* inst_sector,
                            const int32_t* inst_event, const double* y, const double* z, const int32_t* row);
void orm_free(orc_merge_result* r);
enum {
  ORM_LINK_OUT = 0, ORM_LINK_IN,                 /* int32 [K] partner track or -1 */
  ORM_MARGIN,                                    /* double [K] smallest decision margin of the track */
  ORM_CH_HEAD, ORM_CH_NSEG, ORM_CH_NCL, ORM_CH_OFFSET, ORM_CH_NDF, ORM_CH_STATUS, ORM_CH_INST, /* int32 [M] */
  ORM_CH_XREF, ORM_CH_CHI2, ORM_CH_MARGIN,       /* double [M] */
  ORM_CH_PARAM,                                  /* double [M*5] */
  ORM_CH_COV,                                    /* double [M*15] */
  ORM_CH_SEGS,                                   /* int32 [sum nseg] track indices, inner to outer */
  ORM_CH_IDS,                                    /* int32 [sum ncl] cluster ids, inner segment first */
  ORM_PAIRS,                                     /* double [P*3]: inner track, outer track, chi2 of tested pairs */
  ORM_N_ARRAYS
};
int64_t orm_count(const orc_merge_result* r, int which);
const void* orm_array(const orc_merge_result* r, int which);

/* Stand-alone pieces, exposed for the oracle's own tests. */
/* Exact helix transport of p = (y, z, sin phi, tan lambda, q/pT) from x0 to x1;
 * F (row-major 5x5, may be NULL) receives d p1 / d p0.  Returns 0 on success,
 * 1 if |sin phi| reaches s_max. */
int orc_propagate(double bz, double s_max, double x0, double x1, double p[5], double F[25]);
/* Rotate a state at local x of one sector frame into a frame turned by dalpha
 * (radians, new alpha minus old): position and direction exactly; the state is
 * then at *x1 of the new frame.  F (may be NULL) receives the derivative of the
 * new state at that plane, for perturbations that keep the track on it.
 * Returns 0, or 1 if |sin phi| in the new frame reaches s_max or the new
 * direction points inward. */
int orc_rotate(double bz, double s_max, double dalpha, double x0, const double p0[5], double* x1,
               double p1[5], double F[25]);
/* One Kalman update with measurement (my, mz), variances (vy, vz); C is a full
 * row-major 5x5 matrix.  Returns chi2 of the residual. */
double orc_kf_update(double p[5], double C[25], double my, double mz, double vy, double vz);

#ifdef __cplusplus
}
#endif
#endif
