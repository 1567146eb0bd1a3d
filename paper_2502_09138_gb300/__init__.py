"""GB300 TPC sector track finding (arxiv 2502.09138, the "TPC Processing
(Tracking)" step of its Tables 1-3): Python front end of libtpct.so.

    trk = Tracker(precision="mixed")
    trk.reserve(max_clusters, max_instances)
    res = trk.track(DeviceClusters.from_event(ev))      # plain form
    res = trk.track(..., batched=True)                  # graph-captured form

Device buffers are torch tensors; every step runs in the library's kernels.
"""
import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B

N_ROWS_TPC = 152


def default_cuts(**over) -> B.Cuts:
    c = B.Cuts()
    B.load().tpct_default_cuts(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def default_geometry():
    """(row_x, tan_half_sector, z_max) of the TPC readout built into the library
    (152 pad rows, 20-degree sectors, 250 cm drift)."""
    g = B.Geometry()
    B.load().tpct_default_geometry(ctypes.byref(g))
    return np.array(g.row_x[:g.n_rows], dtype=np.float64), float(g.tan_half_sector), float(g.z_max)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


@dataclass
class DeviceClusters:
    """Clusters resident on the device (SoA).  Tracking reads y, z, row and the
    offsets; x only when row is None (nearest row), charge never (it is
    carried for compression): both may be None for a tracking-only caller."""
    x: torch.Tensor               # or None when row is given
    y: torch.Tensor
    z: torch.Tensor
    charge: torch.Tensor          # or None
    row: torch.Tensor            # uint8, or None (row from x)
    sector_offsets: torch.Tensor  # int64 [n_instances + 1]

    @property
    def n(self):
        return int(self.y.shape[0])

    @property
    def n_instances(self):
        return int(self.sector_offsets.shape[0] - 1)

    @classmethod
    def from_event(cls, ev, device="cuda", with_row=True, non_blocking=False, tracking_only=False):
        """tracking_only: leave out x and charge (needs the row)."""
        if tracking_only and not with_row:
            raise ValueError("tracking_only needs the row (x is read only when the row is absent)")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device, non_blocking=non_blocking)
        return cls(None if tracking_only else t(ev.x), t(ev.y), t(ev.z), None if tracking_only else t(ev.charge),
                   t(ev.row) if with_row else None, t(ev.sector_offsets.astype(np.int64)))

    def as_struct(self) -> B.Clusters:
        return B.Clusters(_ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.charge), _ptr(self.row),
                          _ptr(self.sector_offsets), self.n_instances)


class Tracks:
    """Output buffers of one tracking call (device tensors)."""

    def __init__(self, cap_tracks, cap_ids, device):
        kw = dict(device=device)
        self.capacity_tracks, self.capacity_ids = int(cap_tracks), int(cap_ids)
        self.counts = torch.zeros(2, dtype=torch.int32, **kw)
        self.instance = torch.empty(cap_tracks, dtype=torch.int32, **kw)
        self.n_cl = torch.empty(cap_tracks, dtype=torch.int32, **kw)
        self.offset = torch.empty(cap_tracks, dtype=torch.int32, **kw)
        self.ndf = torch.empty(cap_tracks, dtype=torch.int32, **kw)
        self.status = torch.empty(cap_tracks, dtype=torch.int32, **kw)
        self.x_ref = torch.empty(cap_tracks, dtype=torch.float64, **kw)
        self.param = torch.empty(cap_tracks, 5, dtype=torch.float64, **kw)
        self.cov = torch.empty(cap_tracks, 15, dtype=torch.float64, **kw)
        self.chi2 = torch.empty(cap_tracks, dtype=torch.float64, **kw)
        self.cluster_ids = torch.empty(max(1, cap_ids), dtype=torch.int32, **kw)

    def as_struct(self) -> B.TracksOut:
        c = self.counts
        return B.TracksOut(self.capacity_tracks, self.capacity_ids, ctypes.c_void_p(c.data_ptr()),
                           ctypes.c_void_p(c.data_ptr() + 4), _ptr(self.instance), _ptr(self.n_cl),
                           _ptr(self.offset), _ptr(self.ndf), _ptr(self.status), _ptr(self.x_ref),
                           _ptr(self.param), _ptr(self.cov), _ptr(self.chi2), _ptr(self.cluster_ids))

    def to_host(self):
        """Copy the filled part to numpy (synchronises)."""
        nt, ni = (int(v) for v in self.counts.cpu())
        nt_, ni_ = min(nt, self.capacity_tracks), min(ni, self.capacity_ids)
        g = lambda t, k: t[:k].cpu().numpy()
        return dict(n_tracks=nt, n_ids=ni, instance=g(self.instance, nt_), n_cl=g(self.n_cl, nt_),
                    offset=g(self.offset, nt_), ndf=g(self.ndf, nt_), status=g(self.status, nt_),
                    x_ref=g(self.x_ref, nt_), param=g(self.param, nt_), cov=g(self.cov, nt_),
                    chi2=g(self.chi2, nt_), cluster_ids=g(self.cluster_ids, ni_))


def default_merge_cuts(**over) -> B.MergeCuts:
    c = B.MergeCuts()
    B.load().tpct_default_merge_cuts(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


class Chains:
    """Output buffers of tpct_merge (device tensors)."""

    def __init__(self, cap_chains, cap_ids, cap_segs, cap_tracks, device):
        i32 = dict(dtype=torch.int32, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        self.cap = (int(cap_chains), int(cap_ids), int(cap_segs))
        self.counts = torch.zeros(3, **i32)
        c = max(1, cap_chains)
        self.head = torch.empty(c, **i32)
        self.n_seg = torch.empty(c, **i32)
        self.seg_offset = torch.empty(c, **i32)
        self.segs = torch.empty(max(1, cap_segs), **i32)
        self.instance = torch.empty(c, **i32)
        self.n_cl = torch.empty(c, **i32)
        self.offset = torch.empty(c, **i32)
        self.ndf = torch.empty(c, **i32)
        self.status = torch.empty(c, **i32)
        self.x_ref = torch.empty(c, **f64)
        self.param = torch.empty(c, 5, **f64)
        self.cov = torch.empty(c, 15, **f64)
        self.chi2 = torch.empty(c, **f64)
        self.cluster_ids = torch.empty(max(1, cap_ids), **i32)
        self.link_out = torch.full((max(1, cap_tracks),), -1, **i32)
        self.link_in = torch.full((max(1, cap_tracks),), -1, **i32)

    def as_struct(self) -> B.ChainsOut:
        p = self.counts.data_ptr()
        return B.ChainsOut(self.cap[0], self.cap[1], self.cap[2], ctypes.c_void_p(p), ctypes.c_void_p(p + 4),
                           ctypes.c_void_p(p + 8), _ptr(self.head), _ptr(self.n_seg), _ptr(self.seg_offset),
                           _ptr(self.segs), _ptr(self.instance), _ptr(self.n_cl), _ptr(self.offset), _ptr(self.ndf),
                           _ptr(self.status), _ptr(self.x_ref), _ptr(self.param), _ptr(self.cov), _ptr(self.chi2),
                           _ptr(self.cluster_ids), _ptr(self.link_out), _ptr(self.link_in))

    def to_host(self, n_tracks):
        nc, ni, ns = (int(v) for v in self.counts.cpu())
        a, b, c = min(nc, self.cap[0]), min(ni, self.cap[1]), min(ns, self.cap[2])
        g = lambda t, k: t[:k].cpu().numpy()
        return dict(n_chains=nc, n_ids=ni, n_segs=ns, head=g(self.head, a), n_seg=g(self.n_seg, a),
                    seg_offset=g(self.seg_offset, a), segs=g(self.segs, c), instance=g(self.instance, a),
                    n_cl=g(self.n_cl, a), offset=g(self.offset, a), ndf=g(self.ndf, a), status=g(self.status, a),
                    x_ref=g(self.x_ref, a), param=g(self.param, a), cov=g(self.cov, a), chi2=g(self.chi2, a),
                    cluster_ids=g(self.cluster_ids, b), link_out=g(self.link_out, n_tracks),
                    link_in=g(self.link_in, n_tracks))


def default_cf_params(**over) -> B.CfParams:
    p = B.CfParams()
    B.load().tpct_default_cf_params(ctypes.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


class DeviceDigits:
    """Digits on the device (SoA uint16 pad, time, adc; int64 row offsets per
    (instance, row); int32 sector of each instance)."""

    def __init__(self, pad, time, adc, row_offsets, inst_sector):
        self.pad, self.time, self.adc = pad, time, adc
        self.row_offsets, self.inst_sector = row_offsets, inst_sector

    @property
    def n(self):
        return int(self.adc.shape[0])

    @property
    def n_instances(self):
        return int(self.inst_sector.shape[0])

    @classmethod
    def from_digits(cls, dg, device="cuda"):
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(device)
        # uint16 arrays travel as int16 bit patterns (torch has no uint16 arithmetic)
        u16 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(device)
        return cls(u16(dg.pad), u16(dg.time), u16(dg.adc), t(dg.row_offsets, np.int64), t(dg.sectors, np.int32))

    def as_struct(self) -> B.Digits:
        return B.Digits(_ptr(self.pad), _ptr(self.time), _ptr(self.adc), _ptr(self.row_offsets),
                        _ptr(self.inst_sector), self.n_instances)


class ClusterOut:
    """Cluster-finding output buffers (device)."""
    FIELDS = (("x", torch.float32), ("y", torch.float32), ("z", torch.float32), ("pad", torch.float32),
              ("time", torch.float32), ("sigma_pad", torch.float32), ("sigma_time", torch.float32),
              ("q_tot", torch.int32), ("q_max", torch.int16), ("row", torch.uint8), ("flags", torch.uint8))

    def __init__(self, capacity, n_instances, device):
        self.capacity = int(capacity)
        self.counts = torch.zeros(2, dtype=torch.int32, device=device)   # n_clusters, status
        c = max(1, self.capacity)
        for name, dt in self.FIELDS:
            setattr(self, name, torch.empty(c, dtype=dt, device=device))
        self.inst_offsets = torch.zeros(n_instances + 1, dtype=torch.int64, device=device)

    def as_struct(self) -> B.CfOut:
        base = self.counts.data_ptr()
        return B.CfOut(self.capacity, ctypes.c_void_p(base), ctypes.c_void_p(base + 4),
                       *[_ptr(getattr(self, n)) for n, _ in self.FIELDS], _ptr(self.inst_offsets))

    def to_host(self):
        counts = self.counts.cpu().numpy()
        n = int(min(counts[0], self.capacity))
        out = {"n_clusters": int(counts[0]), "status": int(counts[1]) & 0xffffffff,
               "inst_offsets": self.inst_offsets.cpu().numpy()}
        for name, _ in self.FIELDS:
            a = getattr(self, name)[:n].cpu().numpy()
            if name == "q_tot":
                a = a.view(np.uint32)
            elif name == "q_max":
                a = a.view(np.uint16)
            out[name] = a
        return out


class Debug:
    """Intermediate arrays for parity checks (device tensors)."""

    def __init__(self, n, cap_tracklets, n_rows, device):
        i32 = dict(dtype=torch.int32, device=device)
        self.n_rows = n_rows
        self.up = torch.empty(max(1, n), **i32)
        self.down = torch.empty(max(1, n), **i32)
        self.upc = torch.empty(max(1, n), **i32)
        self.downc = torch.empty(max(1, n), **i32)
        self.weight = torch.empty(max(1, n), dtype=torch.int32, device=device)
        self.cap = int(cap_tracklets)
        self.n_tracklets = torch.zeros(1, **i32)
        self.tl_start = torch.empty(max(1, cap_tracklets), **i32)
        self.tl_nhits = torch.empty(max(1, cap_tracklets), **i32)
        self.tl_hits = torch.empty(max(1, cap_tracklets) * n_rows, **i32)
        self.tl_param = torch.empty(max(1, cap_tracklets) * 5, dtype=torch.float64, device=device)
        self.tl_row_ref = torch.empty(max(1, cap_tracklets), **i32)
        self.tr_tracklet = torch.full((max(1, cap_tracklets),), -1, **i32)
        self.counters = torch.zeros(4, dtype=torch.int64, device=device)
        self._n = n

    def as_struct(self) -> B.DebugOut:
        return B.DebugOut(_ptr(self.up), _ptr(self.down), _ptr(self.upc), _ptr(self.downc),
                          _ptr(self.weight), self.cap, _ptr(self.n_tracklets), _ptr(self.tl_start),
                          _ptr(self.tl_nhits), _ptr(self.tl_hits), _ptr(self.tl_param), _ptr(self.tl_row_ref),
                          _ptr(self.tr_tracklet), _ptr(self.counters))

    def to_host(self):
        n = self._n
        T = int(self.n_tracklets.cpu()[0])
        Tc = min(T, self.cap)
        g = lambda t, k: t[:k].cpu().numpy()
        return dict(up=g(self.up, n), down=g(self.down, n), upc=g(self.upc, n), downc=g(self.downc, n),
                    weight=g(self.weight, n).view(np.uint32), n_tracklets=T, tl_start=g(self.tl_start, Tc),
                    tl_nhits=g(self.tl_nhits, Tc), tl_hits=g(self.tl_hits, Tc * self.n_rows).reshape(Tc, self.n_rows),
                    tl_param=g(self.tl_param, Tc * 5).reshape(Tc, 5), tl_row_ref=g(self.tl_row_ref, Tc),
                    tr_tracklet=self.tr_tracklet.cpu().numpy(), counters=self.counters.cpu().numpy())


class Tracker:
    """One context of the CUDA library (one geometry, field, cut set, precision)."""

    def __init__(self, row_x=None, tan_half_sector=None, z_max=250.0, bz=0.5, cuts=None,
                 precision="mixed", device="cuda"):
        L = B.load()
        d_rows, d_tan, _ = default_geometry()
        self.row_x = np.ascontiguousarray(d_rows if row_x is None else row_x, dtype=np.float64)
        self.n_rows = int(self.row_x.shape[0])
        tan_half_sector = d_tan if tan_half_sector is None else tan_half_sector
        g = B.Geometry(self.n_rows, self.row_x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       float(tan_half_sector), float(z_max))
        self.cuts = cuts if cuts is not None else default_cuts()
        self.precision = precision
        h = ctypes.c_void_p()
        B.check(L.tpct_create(ctypes.byref(g), float(bz), ctypes.byref(self.cuts), B.PRECISION[precision],
                              ctypes.byref(h)), "tpct_create")
        self._h = h
        self.device = torch.device(device)
        self._ws = None
        self._plan = (0, 0)

    def close(self):
        if getattr(self, "_h", None):
            B.load().tpct_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, clusters_per_bin=0, tracklet_block=0, refit_block=0):
        B.check(B.load().tpct_set_tuning(self._h, clusters_per_bin, tracklet_block, refit_block),
                "tpct_set_tuning")

    def tuning(self):
        t = B.Tuning()
        B.check(B.load().tpct_get_tuning(self._h, ctypes.byref(t)), "tpct_get_tuning")
        return {f: getattr(t, f) for f, _ in B.Tuning._fields_}

    def autotune(self, clusters: "DeviceClusters", out: "Tracks" = None, cache_path=None, stream=None):
        """Time candidate launch shapes on this workload, keep the fastest (cached in cache_path)."""
        n, ni = clusters.n, clusters.n_instances
        if self._ws is None or n > self._plan[0] or ni > self._plan[1]:
            self.reserve(max(n, self._plan[0]), max(ni, self._plan[1]))
        out = out if out is not None else self.make_output(n)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        t = B.Tuning()
        cs, os_ = clusters.as_struct(), out.as_struct()
        B.check(B.load().tpct_autotune(self._h, ctypes.byref(cs), n, ctypes.byref(os_), ctypes.c_void_p(s.cuda_stream),
                                       cache_path.encode() if cache_path else None, ctypes.byref(t)),
                "tpct_autotune", self._h)
        return {f: getattr(t, f) for f, _ in B.Tuning._fields_}

    def workspace_bytes(self, max_clusters, max_instances):
        return int(B.load().tpct_workspace_bytes(self._h, int(max_clusters), int(max_instances)))

    def reserve(self, max_clusters, max_instances):
        nb = self.workspace_bytes(max_clusters, max_instances)
        if nb == 0:
            raise ValueError("invalid workspace plan")
        self._ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        B.check(B.load().tpct_set_workspace(self._h, ctypes.c_void_p(aligned), nb, int(max_clusters),
                                            int(max_instances)), "tpct_set_workspace")
        self._plan = (int(max_clusters), int(max_instances))

    def make_output(self, n, cap_tracks=None, cap_ids=None):
        cap_tracks = n // 3 + 1 if cap_tracks is None else cap_tracks
        cap_ids = n if cap_ids is None else cap_ids
        return Tracks(cap_tracks, cap_ids, self.device)

    def track(self, clusters: DeviceClusters, out: Tracks = None, batched=False, stream=None):
        n, ni = clusters.n, clusters.n_instances
        if self._ws is None or n > self._plan[0] or ni > self._plan[1]:
            self.reserve(max(n, self._plan[0]), max(ni, self._plan[1]))
        if out is None:
            out = self.make_output(n)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = (clusters, out)
        cs, os_ = clusters.as_struct(), out.as_struct()
        fn = B.load().tpct_track_batch if batched else B.load().tpct_track
        B.check(fn(self._h, ctypes.byref(cs), n, ctypes.byref(os_), ctypes.c_void_p(s.cuda_stream)),
                "tpct_track_batch" if batched else "tpct_track", self._h)
        return out

    def merge(self, clusters: "DeviceClusters", tracks: "Tracks", inst_sector, inst_event, n_events,
              cuts=None, out: "Chains" = None, stream=None):
        """Cross-sector merging of the output of track() on the same clusters."""
        cuts = cuts or default_merge_cuts()
        cap = tracks.capacity_tracks
        nb = int(B.load().tpct_merge_workspace_bytes(cap, clusters.n_instances, int(n_events)))
        if getattr(self, "_mws", None) is None or self._mws.numel() < nb + 256:
            self._mws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        base = (self._mws.data_ptr() + 255) // 256 * 256
        if out is None:
            out = Chains(cap // 2 + 16, clusters.n, cap + 16, cap, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        sec = torch.as_tensor(np.asarray(inst_sector, np.int32), device=self.device)
        evi = torch.as_tensor(np.asarray(inst_event, np.int32), device=self.device)
        self._keep_m = (sec, evi, out, clusters, tracks)
        cs, ts, os_ = clusters.as_struct(), tracks.as_struct(), out.as_struct()
        B.check(B.load().tpct_merge(self._h, ctypes.byref(cs), _ptr(sec), _ptr(evi), int(n_events), ctypes.byref(ts),
                                    ctypes.byref(cuts), ctypes.c_void_p(base), nb, ctypes.byref(os_),
                                    ctypes.c_void_p(s.cuda_stream)), "tpct_merge", self._h)
        return out

    def find_clusters(self, digits: "DeviceDigits", params=None, out: "ClusterOut" = None, capacity=None,
                      stream=None):
        """Cluster finding on device digits (rows of this tracker's geometry)."""
        params = params or default_cf_params()
        lib = B.load()
        if out is None:
            out = ClusterOut(capacity if capacity is not None else digits.n // 4 + 1024, digits.n_instances,
                             self.device)
        nb = int(lib.tpct_cf_workspace_bytes(digits.n, digits.n_instances, self.n_rows, out.capacity))
        if getattr(self, "_cfws", None) is None or self._cfws.numel() < nb + 256:
            self._cfws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        base = (self._cfws.data_ptr() + 255) // 256 * 256
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep_cf = (digits, out)
        ds, os_ = digits.as_struct(), out.as_struct()
        B.check(lib.tpct_find_clusters(self._h, ctypes.byref(ds), ctypes.byref(params), ctypes.c_void_p(base), nb,
                                       ctypes.byref(os_), ctypes.c_void_p(s.cuda_stream)),
                "tpct_find_clusters", self._h)
        return out

    def _scratch(self, name, nbytes):
        buf = getattr(self, name, None)
        if buf is None or buf.numel() < nbytes + 256:
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            setattr(self, name, buf)
        return (buf.data_ptr() + 255) // 256 * 256

    def tm_encode(self, clusters: "DeviceClusters", tracks: "Tracks", capacity_bytes=None, stream=None):
        """Track-model encoding of the clusters with the tracks found on them:
        dict of device tensors data (uint8), n_bytes, track_offsets, row_offsets."""
        lib = B.load()
        ni = clusters.n_instances
        nb = int(lib.tpct_tm_encode_workspace_bytes(clusters.n, tracks.capacity_tracks, ni, self.n_rows))
        base = self._scratch("_tmws", nb)
        cap = int(capacity_bytes if capacity_bytes is not None else 16 * clusters.n + 4 * ni * self.n_rows + 1024)
        st = {"data": torch.empty(max(1, cap), dtype=torch.uint8, device=self.device),
              "n_bytes": torch.zeros(1, dtype=torch.int64, device=self.device),
              "track_offsets": torch.zeros(tracks.capacity_tracks + 1, dtype=torch.int64, device=self.device),
              "row_offsets": torch.zeros(ni * self.n_rows + 1, dtype=torch.int64, device=self.device)}
        ts = B.TmStream(cap, _ptr(st["data"]), _ptr(st["n_bytes"]), _ptr(st["track_offsets"]), _ptr(st["row_offsets"]))
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        cs, os_ = clusters.as_struct(), tracks.as_struct()
        self._keep_tm = (clusters, tracks, st)
        B.check(lib.tpct_tm_encode(self._h, ctypes.byref(cs), clusters.n, ctypes.byref(os_), ctypes.c_void_p(base), nb,
                                   ctypes.byref(ts), ctypes.c_void_p(s.cuda_stream)), "tpct_tm_encode", self._h)
        return st

    def tm_decode(self, data, track_offsets, n_tracks, row_offsets, n_instances, capacity, stream=None,
                  n_bytes=None):
        """Decode a stream (device tensors): dict of x, y, z, charge, row tensors, n and
        status (TD_BAD_STREAM, TD_CAPACITY bits).  n_bytes: the stream's size (default:
        the whole data tensor)."""
        lib = B.load()
        nb = int(lib.tpct_tm_decode_workspace_bytes(int(n_tracks), int(n_instances), self.n_rows))
        base = self._scratch("_tdws", nb)
        c = max(1, int(capacity))
        d = {"n": torch.zeros(1, dtype=torch.int64, device=self.device),
             "x": torch.empty(c, dtype=torch.float32, device=self.device),
             "y": torch.empty(c, dtype=torch.float32, device=self.device),
             "z": torch.empty(c, dtype=torch.float32, device=self.device),
             "charge": torch.empty(c, dtype=torch.int16, device=self.device),
             "row": torch.empty(c, dtype=torch.uint8, device=self.device),
             "status": torch.zeros(1, dtype=torch.int32, device=self.device)}
        ds = B.TmDecoded(int(capacity), _ptr(d["n"]), _ptr(d["x"]), _ptr(d["y"]), _ptr(d["z"]), _ptr(d["charge"]),
                         _ptr(d["row"]), _ptr(d["status"]))
        n_bytes = int(data.numel() * data.element_size()) if n_bytes is None else int(n_bytes)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep_td = (data, track_offsets, row_offsets, d)
        B.check(lib.tpct_tm_decode(self._h, _ptr(data), n_bytes, _ptr(track_offsets), int(n_tracks), _ptr(row_offsets),
                                   int(n_instances), ctypes.c_void_p(base), nb, ctypes.byref(ds),
                                   ctypes.c_void_p(s.cuda_stream)), "tpct_tm_decode", self._h)
        return d

    def set_stage_events(self, events):
        """events: 7 torch.cuda.Event (created with enable_timing) or None to disable."""
        if events is None:
            B.check(B.load().tpct_set_stage_events(self._h, None, 0), "tpct_set_stage_events")
            self._stage_events = None
            return
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        self._stage_events = (events, arr)
        B.check(B.load().tpct_set_stage_events(self._h, arr, len(events)), "tpct_set_stage_events")

    def debug(self, n, cap_tracklets=None, stream=None):
        cap_tracklets = n // 3 + 1 if cap_tracklets is None else cap_tracklets
        d = Debug(n, cap_tracklets, self.n_rows, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        ds = d.as_struct()
        B.check(B.load().tpct_debug_export(self._h, ctypes.byref(ds), ctypes.c_void_p(s.cuda_stream)),
                "tpct_debug_export")
        return d

    def device_status(self):
        return int(B.load().tpct_last_device_status(self._h))

    def kernel_launches(self):
        return int(B.load().tpct_kernel_launches(self._h))


class Pacer:
    """Publishing-rate control of an offline source (native, host-side):
    policy "naive" (in-flight limit only) or "smooth" (adaptive delay)."""

    def __init__(self, policy="smooth", **over):
        lib = B.load()
        c = B.PacerConfig()
        lib.tpct_default_pacer_config(ctypes.byref(c))
        c.policy = {"naive": B.TPCT_PUBLISH_NAIVE, "smooth": B.TPCT_PUBLISH_SMOOTH}[policy]
        for k, v in over.items():
            setattr(c, k, v)
        h = ctypes.c_void_p()
        B.check(lib.tpct_pacer_create(ctypes.byref(c), ctypes.byref(h)), "tpct_pacer_create")
        self._h, self._lib = h, lib

    def try_publish(self, now, in_flight, backlog):
        w = ctypes.c_double(0.0)
        ok = self._lib.tpct_pacer_try_publish(self._h, float(now), int(in_flight), int(backlog), ctypes.byref(w))
        return bool(ok), w.value

    def on_consumed(self, now, in_flight, backlog):
        self._lib.tpct_pacer_on_consumed(self._h, float(now), int(in_flight), int(backlog))

    @property
    def delay(self):
        return self._lib.tpct_pacer_delay(self._h)

    @property
    def pressure_events(self):
        return int(self._lib.tpct_pacer_pressure_events(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.tpct_pacer_destroy(self._h)
            self._h = None


def diag_convert(f_in=None, d_in=None, stream=None):
    """Apply the library's float->double (widen) and double->float (narrow)
    conversions to device tensors; returns (widened, narrowed)."""
    s = stream if stream is not None else torch.cuda.current_stream()
    d_out = torch.empty_like(f_in, dtype=torch.float64) if f_in is not None else None
    f_out = torch.empty_like(d_in, dtype=torch.float32) if d_in is not None else None
    n = int((f_in if f_in is not None else d_in).numel())
    if f_in is not None and d_in is not None and f_in.numel() != d_in.numel():
        raise ValueError("f_in and d_in must have the same length")
    B.check(B.load().tpct_diag_convert(_ptr(f_in), _ptr(d_out), _ptr(d_in), _ptr(f_out), n,
                                       ctypes.c_void_p(s.cuda_stream)), "tpct_diag_convert")
    return d_out, f_out


def probe_fma(use_fp64, blocks, iters, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    ms = ctypes.c_float()
    B.check(B.load().tpct_probe_fma(int(use_fp64), int(blocks), int(iters), ctypes.c_void_p(s.cuda_stream),
                                    ctypes.byref(ms)), "tpct_probe_fma")
    return float(ms.value)


class Server:
    """Serving runtime of the library (continuous batching of time frames
    under a device-memory budget).  Frames are host arrays; the arena is one
    torch allocation of ``budget_bytes``."""

    def __init__(self, n_slots=3, budget_bytes=8 << 30, precision="mixed", bz=0.5, cuts=None, row_x=None,
                 tan_half_sector=None, z_max=250.0, device="cuda"):
        L = B.load()
        d_rows, d_tan, _ = default_geometry()
        self.row_x = np.ascontiguousarray(d_rows if row_x is None else row_x, dtype=np.float64)
        tan_half_sector = d_tan if tan_half_sector is None else tan_half_sector
        g = B.Geometry(int(self.row_x.shape[0]), self.row_x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       float(tan_half_sector), float(z_max))
        self.cuts = cuts if cuts is not None else default_cuts()
        self.device = torch.device(device)
        self.arena = torch.empty(int(budget_bytes) + 256, dtype=torch.uint8, device=self.device)
        base = (self.arena.data_ptr() + 255) // 256 * 256
        cfg = B.ServerConfig(int(n_slots), ctypes.c_void_p(base), int(budget_bytes))
        h = ctypes.c_void_p()
        B.check(L.tpct_server_create(ctypes.byref(g), float(bz), ctypes.byref(self.cuts), B.PRECISION[precision],
                                     ctypes.byref(cfg), ctypes.byref(h)), "tpct_server_create")
        self._h = h
        self._frames = {}

    def close(self):
        if getattr(self, "_h", None):
            B.load().tpct_server_destroy(self._h)
            self._h = None
            self._frames.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def host_frame(x, y, z, charge, row, sector_offsets):
        """Pinned host copies of one frame's arrays (numpy in, torch pinned out)."""
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return dict(x=pin(x), y=pin(y), z=pin(z), charge=None if charge is None else pin(charge),
                    row=None if row is None else pin(row), sector_offsets=pin(np.asarray(sector_offsets, np.int64)))

    def submit(self, frame):
        """frame: dict of host tensors/arrays (x, y, z, charge, row, sector_offsets); kept alive until release."""
        p = lambda t: ctypes.c_void_p(0) if t is None else ctypes.c_void_p(
            t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data)
        n = int(frame["y"].shape[0])
        ni = int(frame["sector_offsets"].shape[0] - 1)
        hf = B.HostFrame(p(frame["x"]), p(frame["y"]), p(frame["z"]), p(frame.get("charge")), p(frame.get("row")),
                         p(frame["sector_offsets"]), ni, n)
        tk = ctypes.c_uint64()
        B.check(B.load().tpct_server_submit(self._h, ctypes.byref(hf), ctypes.byref(tk)), "tpct_server_submit")
        self._frames[tk.value] = frame
        return tk.value

    def poll(self, ticket):
        info = B.FrameInfo()
        B.check(B.load().tpct_server_poll(self._h, ticket, ctypes.byref(info)), "tpct_server_poll")
        return dict(state=info.state, status=info.status, n_tracks=info.n_tracks, n_ids=info.n_ids,
                    queue_us=info.queue_us, latency_us=info.latency_us)

    def wait(self, ticket, timeout_s=600.0):
        B.check(B.load().tpct_server_wait(self._h, ticket, float(timeout_s)), "tpct_server_wait")

    def fetch(self, ticket):
        info = self.poll(ticket)
        nt, ni = max(1, info["n_tracks"]), max(1, info["n_ids"])
        arr = dict(instance=np.empty(nt, np.int32), n_cl=np.empty(nt, np.int32), offset=np.empty(nt, np.int32),
                   ndf=np.empty(nt, np.int32), status=np.empty(nt, np.int32), x_ref=np.empty(nt),
                   param=np.empty((nt, 5)), cov=np.empty((nt, 15)), chi2=np.empty(nt),
                   cluster_ids=np.empty(ni, np.int32))
        q = lambda a: ctypes.c_void_p(a.ctypes.data)
        ht = B.HostTracks(nt, ni, 0, 0, q(arr["instance"]), q(arr["n_cl"]), q(arr["offset"]), q(arr["ndf"]),
                          q(arr["status"]), q(arr["x_ref"]), q(arr["param"]), q(arr["cov"]), q(arr["chi2"]),
                          q(arr["cluster_ids"]))
        B.check(B.load().tpct_server_fetch(self._h, ticket, ctypes.byref(ht)), "tpct_server_fetch")
        out = {k: v[:ht.n_tracks] for k, v in arr.items() if k != "cluster_ids"}
        out["cluster_ids"] = arr["cluster_ids"][:ht.n_ids]
        out["n_tracks"], out["n_ids"] = ht.n_tracks, ht.n_ids
        return out

    def release(self, ticket):
        B.check(B.load().tpct_server_release(self._h, ticket), "tpct_server_release")
        self._frames.pop(ticket, None)

    def stats(self):
        st = B.ServerStats()
        B.check(B.load().tpct_server_get_stats(self._h, ctypes.byref(st)), "tpct_server_get_stats")
        return {f: getattr(st, f) for f, _ in B.ServerStats._fields_}
