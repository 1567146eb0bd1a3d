"""ctypes binding of libtpct.so (include/tpct.h).  Argument marshalling only:
every step of track finding runs in the library's CUDA kernels.  PyTorch
provides device memory and streams."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# TPCT_CHECKED=1 selects the bounds-checked build (build.py --checked), in
# which every subscript of the tracking chain's arrays is range-checked on the
# device and a violation is reported as TPCT_E_BOUNDS
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("TPCT_CHECKED") == "1" else "_build", "libtpct.so")

c_int, c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)

TPCT_OK, TPCT_E_INVALID, TPCT_E_NOMEM, TPCT_E_CAPACITY, TPCT_E_CUDA, TPCT_E_TIMEOUT, TPCT_E_BUDGET, \
    TPCT_E_STATE, TPCT_E_BOUNDS = range(9)
PRECISION = {"fp32": 0, "mixed": 1, "fp64": 2, "mixed_df": 3}


class Geometry(ctypes.Structure):
    _fields_ = [("n_rows", c_int), ("row_x", ctypes.POINTER(c_double)),
                ("tan_half_sector", c_double), ("z_max", c_double)]


class Cuts(ctypes.Structure):
    _fields_ = [("nf_wy", c_double), ("nf_wz", c_double), ("nf_dmax", c_double), ("s_max", c_double),
                ("edge_margin", c_double), ("search_k", c_double), ("chi2_max", c_double),
                ("max_miss", c_int), ("n_min", c_int), ("f_shared", c_double), ("n_refit", c_int),
                ("sig_readout", c_double), ("sig_cathode", c_double), ("c_s", c_double),
                ("c_t", c_double), ("c_qpt", c_double), ("c_yz_refit", c_double),
                ("c_qpt_refit", c_double)]


class Clusters(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("z", c_void_p), ("charge", c_void_p),
                ("row", c_void_p), ("sector_offsets", c_void_p), ("n_instances", c_int32)]


class TracksOut(ctypes.Structure):
    _fields_ = [("capacity_tracks", c_int32), ("capacity_ids", c_int32), ("n_tracks", c_void_p),
                ("n_ids", c_void_p), ("instance", c_void_p), ("n_cl", c_void_p), ("offset", c_void_p),
                ("ndf", c_void_p), ("status", c_void_p), ("x_ref", c_void_p), ("param", c_void_p),
                ("cov", c_void_p), ("chi2", c_void_p), ("cluster_ids", c_void_p)]


class DebugOut(ctypes.Structure):
    _fields_ = [("up", c_void_p), ("down", c_void_p), ("upc", c_void_p), ("downc", c_void_p),
                ("weight", c_void_p), ("capacity_tracklets", c_int32), ("n_tracklets", c_void_p),
                ("tl_start", c_void_p), ("tl_nhits", c_void_p), ("tl_hits", c_void_p),
                ("tl_param", c_void_p), ("tl_row_ref", c_void_p), ("tr_tracklet", c_void_p),
                ("counters", c_void_p)]


class MergeCuts(ctypes.Structure):
    _fields_ = [("chi2_max", c_double), ("max_dtanl", c_double), ("max_gap", c_double), ("alpha0", c_double),
                ("dalpha", c_double)]


class ChainsOut(ctypes.Structure):
    _fields_ = [("capacity_chains", c_int32), ("capacity_ids", c_int32), ("capacity_segs", c_int32),
                ("n_chains", c_void_p), ("n_ids", c_void_p), ("n_segs", c_void_p), ("head", c_void_p),
                ("n_seg", c_void_p), ("seg_offset", c_void_p), ("segs", c_void_p), ("instance", c_void_p),
                ("n_cl", c_void_p), ("offset", c_void_p), ("ndf", c_void_p), ("status", c_void_p),
                ("x_ref", c_void_p), ("param", c_void_p), ("cov", c_void_p), ("chi2", c_void_p),
                ("cluster_ids", c_void_p), ("link_out", c_void_p), ("link_in", c_void_p)]


class CfParams(ctypes.Structure):
    _fields_ = [("pad_pitch_inner", c_double), ("pad_pitch_outer", c_double), ("n_inner_rows", c_int32),
                ("time_bin", c_double), ("n_time", c_int32), ("q_peak_min", c_int32), ("valley_delta", c_int32)]


class Digits(ctypes.Structure):
    _fields_ = [("pad", c_void_p), ("time", c_void_p), ("adc", c_void_p), ("row_offsets", c_void_p),
                ("inst_sector", c_void_p), ("n_instances", c_int32)]


class CfOut(ctypes.Structure):
    _fields_ = [("capacity", c_int32), ("n_clusters", c_void_p), ("status", c_void_p), ("x", c_void_p),
                ("y", c_void_p), ("z", c_void_p), ("pad", c_void_p), ("time", c_void_p), ("sigma_pad", c_void_p),
                ("sigma_time", c_void_p), ("q_tot", c_void_p), ("q_max", c_void_p), ("row", c_void_p),
                ("flags", c_void_p), ("inst_offsets", c_void_p)]


TPCT_CF_BAD_DIGIT, TPCT_CF_TIMEOUT, TPCT_CF_ROW_OVERFLOW, TPCT_CF_CAPACITY, TPCT_CF_WORKSPACE = 1, 2, 4, 8, 16
TPCT_TD_BAD_STREAM, TPCT_TD_CAPACITY = 1, 2
TPCT_PUBLISH_NAIVE, TPCT_PUBLISH_SMOOTH = 0, 1


class TmStream(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("data", c_void_p), ("n_bytes", c_void_p), ("track_offsets", c_void_p),
                ("row_offsets", c_void_p)]


class TmDecoded(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("n", c_void_p), ("x", c_void_p), ("y", c_void_p), ("z", c_void_p),
                ("charge", c_void_p), ("row", c_void_p), ("status", c_void_p)]


class PacerConfig(ctypes.Structure):
    _fields_ = [("policy", c_int), ("max_in_flight", c_int32), ("initial_delay_s", c_double),
                ("decrease", c_double), ("increase", c_double), ("min_delay_s", c_double),
                ("max_delay_s", c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_slots", c_int), ("arena", c_void_p), ("arena_bytes", c_size_t)]


class HostFrame(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("z", c_void_p), ("charge", c_void_p), ("row", c_void_p),
                ("sector_offsets", c_void_p), ("n_instances", c_int32), ("n", c_int64)]


class FrameInfo(ctypes.Structure):
    _fields_ = [("state", c_int32), ("status", c_int), ("n_tracks", c_int32), ("n_ids", c_int32),
                ("queue_us", c_double), ("latency_us", c_double)]


class HostTracks(ctypes.Structure):
    _fields_ = [("capacity_tracks", c_int32), ("capacity_ids", c_int32), ("n_tracks", c_int32),
                ("n_ids", c_int32), ("instance", c_void_p), ("n_cl", c_void_p), ("offset", c_void_p),
                ("ndf", c_void_p), ("status", c_void_p), ("x_ref", c_void_p), ("param", c_void_p),
                ("cov", c_void_p), ("chi2", c_void_p), ("cluster_ids", c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("retries", c_int64),
                ("clusters_completed", c_int64), ("queued", c_int32), ("in_flight", c_int32),
                ("peak_in_flight", c_int32), ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("clusters_per_bin", c_int), ("tracklet_block", c_int), ("refit_block", c_int),
                ("precision", c_int), ("n_rows", c_int), ("ms", ctypes.c_float), ("from_cache", c_int)]


EXPORTS = {
    "tpct_default_cuts": (None, [ctypes.POINTER(Cuts)]),
    "tpct_default_geometry": (None, [ctypes.POINTER(Geometry)]),
    "tpct_create": (c_int, [ctypes.POINTER(Geometry), c_double, ctypes.POINTER(Cuts), c_int,
                            ctypes.POINTER(c_void_p)]),
    "tpct_destroy": (None, [c_void_p]),
    "tpct_set_tuning": (c_int, [c_void_p, c_int, c_int, c_int]),
    "tpct_workspace_bytes": (c_size_t, [c_void_p, c_int64, c_int32]),
    "tpct_set_workspace": (c_int, [c_void_p, c_void_p, c_size_t, c_int64, c_int32]),
    "tpct_track": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_int64, ctypes.POINTER(TracksOut), c_void_p]),
    "tpct_track_batch": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_int64, ctypes.POINTER(TracksOut),
                                 c_void_p]),
    "tpct_set_stage_events": (c_int, [c_void_p, ctypes.POINTER(c_void_p), c_int]),
    "tpct_track_static": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_int64, ctypes.POINTER(TracksOut),
                                  c_void_p]),
    "tpct_debug_export": (c_int, [c_void_p, ctypes.POINTER(DebugOut), c_void_p]),
    "tpct_last_device_status": (c_int, [c_void_p]),
    "tpct_status_str": (ctypes.c_char_p, [c_int]),
    "tpct_last_cuda_error": (ctypes.c_char_p, [c_void_p]),
    "tpct_kernel_launches": (c_int64, [c_void_p]),
    "tpct_default_merge_cuts": (None, [ctypes.POINTER(MergeCuts)]),
    "tpct_merge_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "tpct_merge": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_void_p, c_void_p, c_int32, ctypes.POINTER(TracksOut),
                           ctypes.POINTER(MergeCuts), c_void_p, c_size_t, ctypes.POINTER(ChainsOut), c_void_p]),
    "tpct_get_tuning": (c_int, [c_void_p, ctypes.POINTER(Tuning)]),
    "tpct_default_cf_params": (None, [ctypes.POINTER(CfParams)]),
    "tpct_default_pacer_config": (None, [ctypes.POINTER(PacerConfig)]),
    "tpct_tm_encode_workspace_bytes": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "tpct_tm_encode": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_int64, ctypes.POINTER(TracksOut), c_void_p,
                               c_size_t, ctypes.POINTER(TmStream), c_void_p]),
    "tpct_tm_decode_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "tpct_tm_decode": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                               c_size_t, ctypes.POINTER(TmDecoded), c_void_p]),
    "tpct_pacer_create": (c_int, [ctypes.POINTER(PacerConfig), ctypes.POINTER(c_void_p)]),
    "tpct_pacer_destroy": (None, [c_void_p]),
    "tpct_pacer_try_publish": (c_int, [c_void_p, c_double, c_int32, c_int32, ctypes.POINTER(c_double)]),
    "tpct_pacer_on_consumed": (None, [c_void_p, c_double, c_int32, c_int32]),
    "tpct_pacer_delay": (c_double, [c_void_p]),
    "tpct_pacer_pressure_events": (c_int64, [c_void_p]),
    "tpct_cf_workspace_bytes": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "tpct_find_clusters": (c_int, [c_void_p, ctypes.POINTER(Digits), ctypes.POINTER(CfParams), c_void_p, c_size_t,
                                   ctypes.POINTER(CfOut), c_void_p]),
    "tpct_autotune": (c_int, [c_void_p, ctypes.POINTER(Clusters), c_int64, ctypes.POINTER(TracksOut), c_void_p,
                              ctypes.c_char_p, ctypes.POINTER(Tuning)]),
    "tpct_server_create": (c_int, [ctypes.POINTER(Geometry), c_double, ctypes.POINTER(Cuts), c_int,
                                   ctypes.POINTER(ServerConfig), ctypes.POINTER(c_void_p)]),
    "tpct_server_destroy": (None, [c_void_p]),
    "tpct_server_submit": (c_int, [c_void_p, ctypes.POINTER(HostFrame), ctypes.POINTER(ctypes.c_uint64)]),
    "tpct_server_poll": (c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(FrameInfo)]),
    "tpct_server_wait": (c_int, [c_void_p, ctypes.c_uint64, c_double]),
    "tpct_server_fetch": (c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(HostTracks)]),
    "tpct_server_release": (c_int, [c_void_p, ctypes.c_uint64]),
    "tpct_server_get_stats": (c_int, [c_void_p, ctypes.POINTER(ServerStats)]),
    "tpct_probe_fma": (c_int, [c_int, c_int, c_int, c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "tpct_diag_convert": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
}

_lib = None


def load():
    """Load libtpct.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_09138_gb300/build.py "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TpctError(RuntimeError):
    def __init__(self, code, where, ctx=None):
        self.code = code
        msg = load().tpct_status_str(code).decode()
        if code == TPCT_E_CUDA and ctx is not None:
            msg += ": " + load().tpct_last_cuda_error(ctx).decode()
        super().__init__(f"{where}: {msg} (status {code})")


def check(code, where, ctx=None):
    if code != TPCT_OK:
        raise TpctError(code, where, ctx)
