"""FP64 CPU oracle of TPC sector track finding -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
load this package.  It wraps ``tpct_oracle.c`` (plain single-threaded C,
double precision, compiled with FMA contraction off) through ctypes and
shares no code with the CUDA library.

Parity status of each oracle function (what pins it, in tests/test_oracle_*):
  propagation       closed form: exact circle geometry (analytic helix), straight
                    lines, round trip, mirror symmetry
  Jacobian          central finite differences
  Kalman update     batch least squares on linear problems; noiseless helices
  neighbour finder  brute-force all-pairs search on small events; hand-built fixture
  clean/start/select brute-force set definitions on small events
  tracklet growth   hand-worked fixture (tests/golden/tracklet_hand_fixture.json):
                    miss counter at max_miss and max_miss + 1, a chi2-rejected
                    link, the downward pass's rejected hits, the edge margin,
                    the search tie-break; each planted mistake fails it
  whole tracker     generator truth (efficiency, fake rate, chi2/ndf, pulls);
                    the absolute efficiency level is parity unpinned (the paper
                    prints no tracking-efficiency number)
  compression       hand-encoded fixture (tests/golden/tm_hand_fixture.json);
                    exact round trip of the quantised clusters; parabola
                    residuals of noiseless helices within one grid unit
  cluster finding   hand-computed fixture (tests/golden/cf_hand_fixture.json);
                    generator truth of isolated crossings (efficiency,
                    centroid residuals, charge); translation and input-order
                    invariance
"""
import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass, asdict
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpct_oracle.c")
_SRC_CF = os.path.join(_HERE, "cluster_oracle.c")
_SRC_TM = os.path.join(_HERE, "compress_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libtpct_oracle.so")
_lib = None
_CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]

(ORC_UP, ORC_DOWN, ORC_UPC, ORC_DOWNC, ORC_NF_MARGIN, ORC_WEIGHT, ORC_TL_INST, ORC_TL_START,
 ORC_TL_NHITS, ORC_TL_STOP_UP, ORC_TL_STOP_DOWN, ORC_TL_ROWREF, ORC_TL_XREF, ORC_TL_MARGIN,
 ORC_TL_PARAM, ORC_TL_HITS, ORC_TR_INST, ORC_TR_TRACKLET, ORC_TR_NCL, ORC_TR_OFFSET, ORC_TR_NDF,
 ORC_TR_STATUS, ORC_TR_XREF, ORC_TR_CHI2, ORC_TR_MARGIN, ORC_TR_PARAM, ORC_TR_COV,
 ORC_TR_IDS) = range(28)

_DTYPES = {ORC_NF_MARGIN: np.float64, ORC_WEIGHT: np.uint32, ORC_TL_XREF: np.float64,
           ORC_TL_MARGIN: np.float64, ORC_TL_PARAM: np.float64, ORC_TR_XREF: np.float64,
           ORC_TR_CHI2: np.float64, ORC_TR_MARGIN: np.float64, ORC_TR_PARAM: np.float64,
           ORC_TR_COV: np.float64}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_CF), os.path.getmtime(_SRC_TM),
            os.path.getmtime(os.path.join(_HERE, "tpct_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc"] + _CFLAGS + ["-o", tmp, _SRC, _SRC_CF, _SRC_TM, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(tracker_source: str, workdir: str) -> str:
    """Compile the oracle with ``tracker_source`` in place of tpct_oracle.c
    (same flags, same other sources) into ``workdir``; returns the library
    path.  Used by the tests that plant a mistake in a copy of the oracle."""
    import shutil
    os.makedirs(workdir, exist_ok=True)
    shutil.copy(os.path.join(_HERE, "tpct_oracle.h"), workdir)
    src = os.path.join(workdir, "tpct_oracle.c")
    with open(src, "w") as f:
        f.write(tracker_source)
    out = os.path.join(workdir, "libtpct_oracle_variant.so")
    subprocess.check_call(["gcc"] + _CFLAGS + ["-I", workdir, "-o", out, src, _SRC_CF, _SRC_TM, "-lm"])
    return out


class _Geom(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int), ("row_x", ctypes.POINTER(ctypes.c_double)),
                ("tan_half_sector", ctypes.c_double), ("z_max", ctypes.c_double)]


class _Cuts(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_double), ("nf_wy", ctypes.c_double), ("nf_wz", ctypes.c_double),
                ("nf_dmax", ctypes.c_double), ("s_max", ctypes.c_double),
                ("edge_margin", ctypes.c_double),
                ("search_k", ctypes.c_double), ("chi2_max", ctypes.c_double),
                ("max_miss", ctypes.c_int), ("n_min", ctypes.c_int), ("f_shared", ctypes.c_double),
                ("n_refit", ctypes.c_int), ("sig_readout", ctypes.c_double),
                ("sig_cathode", ctypes.c_double), ("c_s", ctypes.c_double), ("c_t", ctypes.c_double),
                ("c_qpt", ctypes.c_double), ("c_yz_refit", ctypes.c_double),
                ("c_qpt_refit", ctypes.c_double)]


def load_library(path):
    """Load an oracle shared library from ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    L.orc_track.restype = ctypes.c_void_p
    L.orc_track.argtypes = [ctypes.POINTER(_Geom), ctypes.POINTER(_Cuts), ctypes.c_int64,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_int]
    L.orc_free.argtypes = [ctypes.c_void_p]
    L.orc_count.restype = ctypes.c_int64
    L.orc_count.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_array.restype = ctypes.c_void_p
    L.orc_array.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_propagate.restype = ctypes.c_int
    L.orc_propagate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_void_p, ctypes.c_void_p]
    L.orc_merge.restype = ctypes.c_void_p
    L.orc_merge.argtypes = [ctypes.POINTER(_Geom), ctypes.POINTER(_Cuts), ctypes.POINTER(_MergeCuts),
                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p]
    L.orm_free.argtypes = [ctypes.c_void_p]
    L.orm_count.restype = ctypes.c_int64
    L.orm_count.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orm_array.restype = ctypes.c_void_p
    L.orm_array.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_rotate.restype = ctypes.c_int
    L.orc_rotate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_kf_update.restype = ctypes.c_double
    L.orc_kf_update.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


@contextlib.contextmanager
def using_library(L):
    """Route the oracle's Python functions through another build of it (the
    tests load copies with a deliberately planted mistake to show that the
    pins catch it)."""
    global _lib
    saved = lib()
    _lib = L
    try:
        yield L
    finally:
        _lib = saved


@dataclass
class Cuts:
    """Tracking constants (the stated readings; the paper gives none)."""
    bz: float = 0.5
    nf_wy: float = 2.0
    nf_wz: float = 2.0
    nf_dmax: float = 0.25
    s_max: float = 0.999
    edge_margin: float = 1.0
    search_k: float = 5.0
    chi2_max: float = 25.0
    max_miss: int = 8
    n_min: int = 20
    f_shared: float = 0.1
    n_refit: int = 3
    sig_readout: float = 0.1
    sig_cathode: float = 0.1
    c_s: float = 1.0
    c_t: float = 1.0
    c_qpt: float = 100.0
    c_yz_refit: float = 100.0
    c_qpt_refit: float = 1.0e4

    @classmethod
    def for_event(cls, ev, **over):
        c = cls(bz=ev.bz, sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode)
        for k, v in over.items():
            setattr(c, k, v)
        return c


class _MergeCuts(ctypes.Structure):
    _fields_ = [("chi2_max", ctypes.c_double), ("max_dtanl", ctypes.c_double), ("max_gap", ctypes.c_double),
                ("alpha0", ctypes.c_double), ("dalpha", ctypes.c_double)]


@dataclass
class MergeCuts:
    """Cross-sector merging constants (stated readings)."""
    chi2_max: float = 50.0
    max_dtanl: float = 0.1
    max_gap: float = 40.0
    alpha0: float = 0.17453292519943295    # 10 degrees
    dalpha: float = 0.3490658503988659     # 20 degrees


(ORM_LINK_OUT, ORM_LINK_IN, ORM_MARGIN, ORM_CH_HEAD, ORM_CH_NSEG, ORM_CH_NCL, ORM_CH_OFFSET, ORM_CH_NDF,
 ORM_CH_STATUS, ORM_CH_INST, ORM_CH_XREF, ORM_CH_CHI2, ORM_CH_MARGIN, ORM_CH_PARAM, ORM_CH_COV, ORM_CH_SEGS,
 ORM_CH_IDS, ORM_PAIRS) = range(18)
_ORM_DT = {ORM_MARGIN: np.float64, ORM_CH_XREF: np.float64, ORM_CH_CHI2: np.float64, ORM_CH_MARGIN: np.float64,
           ORM_CH_PARAM: np.float64, ORM_CH_COV: np.float64, ORM_PAIRS: np.float64}


class MergeResult:
    """Cross-sector merging output as numpy arrays."""

    def __init__(self, handle):
        L = lib()
        names = {ORM_LINK_OUT: "link_out", ORM_LINK_IN: "link_in", ORM_MARGIN: "margin", ORM_CH_HEAD: "ch_head",
                 ORM_CH_NSEG: "ch_nseg", ORM_CH_NCL: "ch_ncl", ORM_CH_OFFSET: "ch_offset", ORM_CH_NDF: "ch_ndf",
                 ORM_CH_STATUS: "ch_status", ORM_CH_INST: "ch_inst", ORM_CH_XREF: "ch_x_ref",
                 ORM_CH_CHI2: "ch_chi2", ORM_CH_MARGIN: "ch_margin", ORM_CH_PARAM: "ch_param",
                 ORM_CH_COV: "ch_cov", ORM_CH_SEGS: "ch_segs", ORM_CH_IDS: "ch_ids", ORM_PAIRS: "pairs"}
        for w, name in names.items():
            n = L.orm_count(handle, w)
            dt = _ORM_DT.get(w, np.int32)
            p = L.orm_array(handle, w)
            if n <= 0 or not p:
                arr = np.zeros(0, dt)
            else:
                buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(p)
                arr = np.frombuffer(buf, dtype=dt).copy()
            setattr(self, name, arr)
        self.ch_param = self.ch_param.reshape(-1, 5)
        self.ch_cov = self.ch_cov.reshape(-1, 15)
        self.pairs = self.pairs.reshape(-1, 3)

    @property
    def n_chains(self):
        return int(self.ch_head.shape[0])

    def chain_ids(self, k):
        o = int(self.ch_offset[k])
        return self.ch_ids[o:o + int(self.ch_ncl[k])]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Result:
    """Oracle output as numpy arrays (copied out of the C result)."""

    def __init__(self, handle, n_rows):
        L = lib()
        self.n_rows = n_rows
        names = {
            ORC_UP: "up", ORC_DOWN: "down", ORC_UPC: "upc", ORC_DOWNC: "downc",
            ORC_NF_MARGIN: "nf_margin", ORC_WEIGHT: "weight", ORC_TL_INST: "tl_inst",
            ORC_TL_START: "tl_start", ORC_TL_NHITS: "tl_nhits", ORC_TL_STOP_UP: "tl_stop_up",
            ORC_TL_STOP_DOWN: "tl_stop_down", ORC_TL_ROWREF: "tl_row_ref", ORC_TL_XREF: "tl_x_ref",
            ORC_TL_MARGIN: "tl_margin", ORC_TL_PARAM: "tl_param", ORC_TL_HITS: "tl_hits",
            ORC_TR_INST: "tr_inst", ORC_TR_TRACKLET: "tr_tracklet", ORC_TR_NCL: "tr_ncl",
            ORC_TR_OFFSET: "tr_offset", ORC_TR_NDF: "tr_ndf", ORC_TR_STATUS: "tr_status",
            ORC_TR_XREF: "tr_x_ref", ORC_TR_CHI2: "tr_chi2", ORC_TR_MARGIN: "tr_margin",
            ORC_TR_PARAM: "tr_param", ORC_TR_COV: "tr_cov", ORC_TR_IDS: "tr_ids"}
        for w, name in names.items():
            n = L.orc_count(handle, w)
            dt = _DTYPES.get(w, np.int32)
            p = L.orc_array(handle, w)
            if n <= 0 or not p:
                arr = np.zeros(0, dt)
            else:
                buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(p)
                arr = np.frombuffer(buf, dtype=dt).copy()
            setattr(self, name, arr)
        self.tl_param = self.tl_param.reshape(-1, 5)
        self.tl_hits = self.tl_hits.reshape(-1, n_rows)
        self.tr_param = self.tr_param.reshape(-1, 5)
        self.tr_cov = self.tr_cov.reshape(-1, 15)

    @property
    def n_tracks(self):
        return int(self.tr_inst.shape[0])

    @property
    def n_tracklets(self):
        return int(self.tl_inst.shape[0])

    def track_ids(self, k):
        o = int(self.tr_offset[k])
        return self.tr_ids[o:o + int(self.tr_ncl[k])]


def track(geometry, cuts, sector_offsets, y, z, row=None, x=None, brute_force_nf=False) -> Result:
    """Run the oracle on all sector instances.  y, z are converted to float64."""
    L = lib()
    rx = np.ascontiguousarray(geometry.row_x, dtype=np.float64)
    g = _Geom(int(rx.shape[0]), rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
              float(geometry.tan_half_sector), float(geometry.z_max))
    c = _Cuts(**asdict(cuts))
    offs = np.ascontiguousarray(sector_offsets, dtype=np.int64)
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    z64 = np.ascontiguousarray(z, dtype=np.float64)
    r32 = None if row is None else np.ascontiguousarray(row, dtype=np.int32)
    x64 = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
    h = L.orc_track(ctypes.byref(g), ctypes.byref(c), offs.shape[0] - 1, _ptr(offs), _ptr(x64),
                    _ptr(y64), _ptr(z64), _ptr(r32), int(bool(brute_force_nf)))
    if not h:
        raise RuntimeError("oracle failed (invalid arguments or out of memory)")
    try:
        return Result(h, int(rx.shape[0]))
    finally:
        L.orc_free(h)


def track_merge(geometry, cuts, mcuts, sector_offsets, y, z, row, inst_sector, inst_event):
    """Sector tracking followed by cross-sector merging; returns (Result, MergeResult)."""
    L = lib()
    rx = np.ascontiguousarray(geometry.row_x, dtype=np.float64)
    g = _Geom(int(rx.shape[0]), rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
              float(geometry.tan_half_sector), float(geometry.z_max))
    c = _Cuts(**asdict(cuts))
    mc = _MergeCuts(**asdict(mcuts))
    offs = np.ascontiguousarray(sector_offsets, dtype=np.int64)
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    z64 = np.ascontiguousarray(z, dtype=np.float64)
    r32 = np.ascontiguousarray(row, dtype=np.int32)
    sec = np.ascontiguousarray(inst_sector, dtype=np.int32)
    evi = np.ascontiguousarray(inst_event, dtype=np.int32)
    h = L.orc_track(ctypes.byref(g), ctypes.byref(c), offs.shape[0] - 1, _ptr(offs), None, _ptr(y64), _ptr(z64),
                    _ptr(r32), 0)
    if not h:
        raise RuntimeError("oracle failed (invalid arguments or out of memory)")
    try:
        res = Result(h, int(rx.shape[0]))
        hm = L.orc_merge(ctypes.byref(g), ctypes.byref(c), ctypes.byref(mc), h, offs.shape[0] - 1, _ptr(sec),
                         _ptr(evi), _ptr(y64), _ptr(z64), _ptr(r32))
        if not hm:
            raise RuntimeError("oracle merge failed")
        try:
            mres = MergeResult(hm)
        finally:
            L.orm_free(hm)
    finally:
        L.orc_free(h)
    return res, mres


def event_instances(ev):
    """Sector number and collision index of every instance of an Event."""
    ni = ev.n_instances
    sec = np.asarray(ev.sectors, dtype=np.int32)
    evi = (np.arange(ni) // max(1, ev.sectors_per_event)).astype(np.int32)
    return sec, evi


def track_merge_event(ev, cuts=None, mcuts=None, geometry=None, exact=False):
    from synth import default_geometry
    geometry = geometry or default_geometry()
    cuts = cuts or Cuts.for_event(ev)
    mcuts = mcuts or MergeCuts()
    sec, evi = event_instances(ev)
    y = ev.y64 if exact else ev.y
    z = ev.z64 if exact else ev.z
    return track_merge(geometry, cuts, mcuts, ev.sector_offsets, y, z, ev.row, sec, evi)


def track_event(ev, cuts=None, geometry=None, exact=False, **kw) -> Result:
    """Oracle on a synthetic Event (FP32 positions widened to FP64, or the
    exact FP64 positions if ``exact``)."""
    from synth import default_geometry
    geometry = geometry or default_geometry()
    cuts = cuts or Cuts.for_event(ev)
    y = ev.y64 if exact else ev.y
    z = ev.z64 if exact else ev.z
    return track(geometry, cuts, ev.sector_offsets, y, z, row=ev.row, **kw)


def propagate(bz, s_max, x0, x1, p, want_jacobian=True):
    L = lib()
    p = np.ascontiguousarray(p, dtype=np.float64).copy()
    F = np.zeros(25) if want_jacobian else None
    rc = L.orc_propagate(bz, s_max, x0, x1, _ptr(p), _ptr(F))
    return rc, p, (F.reshape(5, 5) if F is not None else None)


def rotate(bz, s_max, dalpha, x0, p, want_jacobian=True):
    L = lib()
    p = np.ascontiguousarray(p, dtype=np.float64)
    p1 = np.zeros(5)
    x1 = ctypes.c_double()
    F = np.zeros(25) if want_jacobian else None
    rc = L.orc_rotate(bz, s_max, dalpha, x0, _ptr(p), ctypes.byref(x1), _ptr(p1), _ptr(F))
    return rc, x1.value, p1, (F.reshape(5, 5) if F is not None else None)


def kf_update(p, C, my, mz, vy, vz):
    L = lib()
    p = np.ascontiguousarray(p, dtype=np.float64).copy()
    C = np.ascontiguousarray(C, dtype=np.float64).copy()
    chi2 = L.orc_kf_update(_ptr(p), _ptr(C), my, mz, vy, vz)
    return chi2, p, C


# ---------------------------------------------------------------- cluster finding
class _CfParams(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int), ("row_x", ctypes.POINTER(ctypes.c_double)),
                ("tan_half", ctypes.c_double), ("z_max", ctypes.c_double),
                ("pad_pitch_inner", ctypes.c_double), ("pad_pitch_outer", ctypes.c_double),
                ("n_inner_rows", ctypes.c_int), ("time_bin", ctypes.c_double), ("n_time", ctypes.c_int),
                ("q_peak_min", ctypes.c_int), ("valley_delta", ctypes.c_int)]


@dataclass
class CfParams:
    """Readings of cluster finding (see cluster_oracle.c): readout geometry,
    peak threshold and valley depth."""
    pad_pitch_inner: float = 0.4
    pad_pitch_outer: float = 0.6
    n_inner_rows: int = 63
    time_bin: float = 0.5
    n_time: int = 500
    q_peak_min: int = 7
    valley_delta: int = 2


(OCF_X, OCF_Y, OCF_Z, OCF_PAD, OCF_TIME, OCF_SPAD, OCF_STIME, OCF_QTOT, OCF_QMAX, OCF_ROW, OCF_FLAGS,
 OCF_INST, OCF_PEAK) = range(13)
_CF_FIELDS = [("x", OCF_X, np.float64), ("y", OCF_Y, np.float64), ("z", OCF_Z, np.float64),
              ("pad", OCF_PAD, np.float64), ("time", OCF_TIME, np.float64), ("sigma_pad", OCF_SPAD, np.float64),
              ("sigma_time", OCF_STIME, np.float64), ("q_tot", OCF_QTOT, np.uint32),
              ("q_max", OCF_QMAX, np.uint16), ("row", OCF_ROW, np.uint8), ("flags", OCF_FLAGS, np.uint8),
              ("instance", OCF_INST, np.int32), ("peak", OCF_PEAK, np.int64)]


class ClusterResult:
    """Clusters of the oracle (numpy arrays, one entry per cluster)."""

    def __init__(self, fields):
        self.__dict__.update(fields)

    @property
    def n(self):
        return int(self.instance.shape[0])


def find_clusters(digits, params: CfParams = None, geometry=None) -> ClusterResult:
    """Cluster finding on a synth.digits.Digits (or an object with the same
    fields: pad, time, adc, row_offsets, sectors)."""
    from synth import default_geometry
    L = lib()
    if not getattr(L, "_cf_ready", False):
        L.orc_find_clusters.restype = ctypes.c_void_p
        L.orc_find_clusters.argtypes = [ctypes.POINTER(_CfParams), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_int)]
        L.orc_cf_count.restype = ctypes.c_int64
        L.orc_cf_count.argtypes = [ctypes.c_void_p]
        L.orc_cf_array.restype = ctypes.c_void_p
        L.orc_cf_array.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_cf_free.argtypes = [ctypes.c_void_p]
        L._cf_ready = True
    g = geometry or default_geometry()
    prm = params or CfParams()
    row_x = np.ascontiguousarray(g.row_x, dtype=np.float64)
    cp = _CfParams(g.n_rows, row_x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), g.tan_half_sector, g.z_max,
                   prm.pad_pitch_inner, prm.pad_pitch_outer, prm.n_inner_rows, prm.time_bin, prm.n_time,
                   prm.q_peak_min, prm.valley_delta)
    pad = np.ascontiguousarray(digits.pad, dtype=np.uint16)
    tim = np.ascontiguousarray(digits.time, dtype=np.uint16)
    adc = np.ascontiguousarray(digits.adc, dtype=np.uint16)
    offs = np.ascontiguousarray(digits.row_offsets, dtype=np.int64)
    sec = np.ascontiguousarray(digits.sectors, dtype=np.int32)
    err = ctypes.c_int(0)
    h = L.orc_find_clusters(ctypes.byref(cp), int(sec.shape[0]), _ptr(sec), _ptr(offs), _ptr(pad), _ptr(tim),
                            _ptr(adc), ctypes.byref(err))
    if not h:
        raise ValueError(f"oracle cluster finding failed (code {err.value})")
    try:
        n = int(L.orc_cf_count(h))
        out = {}
        for name, w, dt in _CF_FIELDS:
            p = L.orc_cf_array(h, w)
            out[name] = (np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                                shape=(n,)).copy() if n and p else np.zeros(0, dt))
    finally:
        L.orc_cf_free(h)
    return ClusterResult(out)


# ---------------------------------------------------------------- track-model compression
class _TmGeom(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int), ("row_x", ctypes.POINTER(ctypes.c_double))]


class TmStream:
    """An encoded frame: bytes, per-track and per-(instance, row) block offsets."""

    def __init__(self, data, track_off, row_off):
        self.data, self.track_off, self.row_off = data, track_off, row_off

    @property
    def nbytes(self):
        return int(self.data.shape[0])


def _tm_lib():
    L = lib()
    if not getattr(L, "_tm_ready", False):
        L.orc_tm_encode.restype = ctypes.c_void_p
        L.orc_tm_encode.argtypes = [ctypes.POINTER(_TmGeom), ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        for f in ("orc_tm_bytes",):
            getattr(L, f).restype = ctypes.c_int64
            getattr(L, f).argtypes = [ctypes.c_void_p]
        for f in ("orc_tm_data", "orc_tm_track_offsets", "orc_tm_row_offsets"):
            getattr(L, f).restype = ctypes.c_void_p
            getattr(L, f).argtypes = [ctypes.c_void_p]
        L.orc_tm_free.argtypes = [ctypes.c_void_p]
        L.orc_tm_decode.restype = ctypes.c_int64
        L.orc_tm_decode.argtypes = [ctypes.POINTER(_TmGeom), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L._tm_ready = True
    return L


def _tm_geom(geometry):
    from synth import default_geometry
    g = geometry or default_geometry()
    rx = np.ascontiguousarray(g.row_x, dtype=np.float64)
    return _TmGeom(g.n_rows, rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), rx, g.n_rows


def tm_encode(ev, tr_offset, tr_ncl, tr_ids, geometry=None) -> TmStream:
    """Track-model encoding of an Event's clusters given its tracks (cluster
    positions, rows ascending): see compress_oracle.c for the format."""
    L = _tm_lib()
    g, rx, nr = _tm_geom(geometry)
    y = np.ascontiguousarray(ev.y, dtype=np.float32)
    z = np.ascontiguousarray(ev.z, dtype=np.float32)
    q = np.ascontiguousarray(ev.charge, dtype=np.uint16) if ev.charge is not None else None
    row = np.ascontiguousarray(ev.row, dtype=np.uint8)
    io = np.ascontiguousarray(ev.sector_offsets, dtype=np.int64)
    off = np.ascontiguousarray(tr_offset, dtype=np.int32)
    ncl = np.ascontiguousarray(tr_ncl, dtype=np.int32)
    ids = np.ascontiguousarray(tr_ids, dtype=np.int32)
    nt = int(ncl.shape[0])
    h = L.orc_tm_encode(ctypes.byref(g), int(ev.n), int(io.shape[0] - 1), _ptr(io), _ptr(y), _ptr(z), _ptr(q),
                        _ptr(row), nt, _ptr(off), _ptr(ncl), _ptr(ids))
    if not h:
        raise MemoryError("oracle encoding failed")
    try:
        nb = int(L.orc_tm_bytes(h))
        nblk = (io.shape[0] - 1) * nr
        cp = lambda p, n, dt: np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                                    shape=(n,)).copy()
        data = cp(L.orc_tm_data(h), nb, np.uint8) if nb else np.zeros(0, np.uint8)
        return TmStream(data, cp(L.orc_tm_track_offsets(h), nt + 1, np.int64),
                        cp(L.orc_tm_row_offsets(h), nblk + 1, np.int64))
    finally:
        L.orc_tm_free(h)


def tm_decode(stream: TmStream, n_max, geometry=None):
    """Decode a stream: dict of x, y, z (float32), charge (uint16), row (uint8)."""
    L = _tm_lib()
    g, rx, nr = _tm_geom(geometry)
    out = {"x": np.zeros(n_max, np.float32), "y": np.zeros(n_max, np.float32), "z": np.zeros(n_max, np.float32),
           "charge": np.zeros(n_max, np.uint16), "row": np.zeros(n_max, np.uint8)}
    data = np.ascontiguousarray(stream.data) if stream.nbytes else np.zeros(1, np.uint8)
    n = L.orc_tm_decode(ctypes.byref(g), _ptr(data), int(stream.track_off.shape[0] - 1), _ptr(stream.track_off),
                        int(stream.row_off.shape[0] - 1), _ptr(stream.row_off), int(n_max), _ptr(out["x"]),
                        _ptr(out["y"]), _ptr(out["z"]), _ptr(out["charge"]), _ptr(out["row"]))
    if n < 0:
        raise ValueError("decoded more clusters than n_max")
    return {k: v[:n] for k, v in out.items()}
