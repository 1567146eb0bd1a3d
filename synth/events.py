"""Seeded synthetic TPC events.

Particles start at the origin and move on helices in a solenoidal field Bz
along +z.  In the transverse plane a particle of charge q and transverse
momentum pT moves on a circle of radius R = pT / (k_B) with
k_B = 0.299792458e-2 * Bz [1/cm per GeV/c]; a positive particle turns
clockwise (towards -y of its initial direction).  For every sector whose
wedge the circle passes through, the generator intersects the circle with the
plane of each pad row (local x = row radius) on the outward branch, computes
the swept arc length from the circle-centre angle, and records a hit if the
point lies inside the sector (|y| <= x tan 10deg, |z| <= 250 cm, z on the
sector's side).

This module holds only event simulation; no step of the track finder.

Random numbers: ``synth.rng`` (SplitMix64 addressed by counters).  Streams:
  0 track parameters, 1 y smearing, 2 z smearing, 3 row efficiency,
  4 charge, 5 noise positions, 6 shuffle keys, 7 impact parameter.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from . import rng
from .geometry import Geometry, default_geometry, N_ROWS

BASE_SEED = 250209138
K_B_PER_TESLA = 0.299792458e-2

S_TRACK, S_SMEAR_Y, S_SMEAR_Z, S_EFF, S_CHARGE, S_NOISE, S_SHUFFLE, S_IMPACT = range(8)


def seed_for(config_index: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of workload ``config_index``."""
    return BASE_SEED + 1000 * config_index + instance


@dataclass
class SigmaModel:
    """Cluster resolution: sigma rises linearly with drift length
    d = clamp(z_max - |z|, 0, z_max) from ``at_readout`` (d = 0) to
    ``at_cathode`` (d = z_max), identical for y and z."""
    at_readout: float = 0.1
    at_cathode: float = 0.1
    z_max: float = 250.0

    def __call__(self, z):
        d = np.clip(self.z_max - np.abs(z), 0.0, self.z_max)
        return self.at_readout + (self.at_cathode - self.at_readout) * d / self.z_max


@dataclass
class Event:
    """One batch of collisions in the tracker's input layout.

    Clusters are grouped by sector instance (event-major, then sector);
    ``sector_offsets`` has n_instances + 1 entries.  Cluster ids are positions
    in these arrays.  ``mc`` is the generating particle (-1 for noise),
    offset so that labels are unique across the batch.
    """
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    charge: np.ndarray
    row: np.ndarray
    sector_offsets: np.ndarray
    sectors: np.ndarray            # sector number of each instance
    mc: np.ndarray
    n_events: int = 1
    sectors_per_event: int = 36
    bz: float = 0.5
    sigma: SigmaModel = field(default_factory=SigmaModel)
    y64: np.ndarray = None         # exact (unsmeared, unrounded) positions, if kept
    z64: np.ndarray = None
    truth: dict = field(default_factory=dict)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_instances(self) -> int:
        return int(self.sector_offsets.shape[0] - 1)

    def instance_of_cluster(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_instances, dtype=np.int64),
                         np.diff(self.sector_offsets))

    def nbytes_soa(self) -> int:
        return self.n * (4 * 3 + 2 + 1)

    def select_instances(self, idx):
        """A new Event holding only the given sector instances (same order)."""
        idx = np.asarray(idx, dtype=np.int64)
        parts = [np.arange(self.sector_offsets[i], self.sector_offsets[i + 1]) for i in idx]
        sel = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        counts = np.array([p.shape[0] for p in parts], dtype=np.int64)
        offs = np.zeros(len(idx) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(counts)
        return Event(self.x[sel], self.y[sel], self.z[sel], self.charge[sel], self.row[sel],
                     offs, self.sectors[idx], self.mc[sel], n_events=len(idx),
                     sectors_per_event=1, bz=self.bz, sigma=self.sigma,
                     y64=None if self.y64 is None else self.y64[sel],
                     z64=None if self.z64 is None else self.z64[sel],
                     meta=dict(self.meta, selected_instances=idx.tolist()))


def _sample_tracks(seed, n, pt_mode, eta_lo, eta_hi, eta_fold, phi_lo, phi_hi):
    c = np.arange(n, dtype=np.uint64) * np.uint64(4)
    u_pt = rng.uniform(seed, S_TRACK, c)
    u_eta = rng.uniform(seed, S_TRACK, c + np.uint64(1))
    u_phi = rng.uniform(seed, S_TRACK, c + np.uint64(2))
    u_q = rng.uniform(seed, S_TRACK, c + np.uint64(3))
    kind = pt_mode[0]
    if kind == "loguniform":
        lo, hi = pt_mode[1], pt_mode[2]
        pt = lo * (hi / lo) ** u_pt
    elif kind == "exp":
        scale, lo, hi = pt_mode[1], pt_mode[2], pt_mode[3]
        a, b = math.exp(-lo / scale), math.exp(-hi / scale)
        pt = -scale * np.log(a - u_pt * (a - b))
    elif kind == "fixed":
        pt = np.full(n, float(pt_mode[1]))
    else:
        raise ValueError(pt_mode)
    if eta_fold:
        eta = eta_hi * u_eta          # |eta| in [0, eta_hi): A side only
    else:
        eta = eta_lo + (eta_hi - eta_lo) * u_eta
    phi = phi_lo + (phi_hi - phi_lo) * u_phi
    q = np.where(u_q < 0.5, -1.0, 1.0)
    return pt, eta, phi, q


def _moyal_charge(u):
    from scipy.special import erfcinv
    m = -2.0 * np.log(math.sqrt(2.0) * erfcinv(u))
    return np.clip(np.rint(40.0 + 12.0 * m), 1, 65535).astype(np.uint16)


def _crossings(geom, qpt, phi0, tanl, sector, bz):
    """Hit positions of (track, sector) pairs on all rows.

    Returns (y, z, ok) of shape [pairs, rows]: exact circle/plane
    intersections on the outward branch, in the sector's local frame."""
    x = geom.row_x[None, :]
    alpha = np.radians(geom.alpha0_deg + (sector % 18) * geom.dalpha_deg)[:, None]
    phl = (phi0[:, None] - alpha)
    sphl, cphl = np.sin(phl), np.cos(phl)
    rho = (-K_B_PER_TESLA * bz * qpt)[:, None]
    tl = tanl[:, None]
    straight = rho == 0.0
    rsafe = np.where(straight, 1.0, rho)
    cx = -sphl / rsafe
    cy = cphl / rsafe
    radius = 1.0 / np.abs(rsafe)
    dxc = x - cx
    disc = radius * radius - dxc * dxc
    ok_c = disc >= 0.0
    yc = cy - np.sign(rsafe) * np.sqrt(np.where(ok_c, disc, 0.0))
    ax, ay = -cx, -cy
    bx, by = dxc, yc - cy
    th = np.arctan2(ax * by - ay * bx, ax * bx + ay * by)
    th = np.where((rsafe > 0) & (th < 0), th + 2.0 * np.pi, th)
    th = np.where((rsafe < 0) & (th > 0), th - 2.0 * np.pi, th)
    s_c = th / rsafe
    # straight line (infinite momentum)
    ok_l = cphl > 0.0
    cl = np.where(ok_l, cphl, 1.0)
    y_l = x * sphl / cl
    s_l = x / cl
    y = np.where(straight, y_l, yc)
    s = np.where(straight, s_l, s_c)
    ok = np.where(straight, ok_l, ok_c)
    z = s * tl
    side_c = sector >= 18
    ok &= np.abs(y) <= x * geom.tan_half_sector
    ok &= np.abs(z) <= geom.z_max
    ok &= np.where(side_c[:, None], z < 0.0, z >= 0.0)
    return y, z, ok


def _candidate_sectors(geom, qpt, phi0, tanl, bz, sector_subset):
    """(track, sector) pairs that can hold hits: the wedges spanned by the
    track's azimuth between 80 and 245 cm from the origin, plus one on each side."""
    n = qpt.shape[0]
    if sector_subset is not None:
        tr = np.repeat(np.arange(n), len(sector_subset))
        sec = np.tile(np.asarray(sector_subset, dtype=np.int64), n)
        keep = (sec >= 18) == (tanl[tr] < 0.0)
        return tr[keep], sec[keep]
    rho = -K_B_PER_TESLA * bz * qpt
    def azim(d):
        a = np.clip(rho * d / 2.0, -1.0, 1.0)
        return phi0 + np.arcsin(a)
    ta, tb = azim(80.0), azim(245.0)
    w = math.radians(geom.dalpha_deg)
    lo = np.floor(np.minimum(ta, tb) / w).astype(np.int64) - 1
    hi = np.floor(np.maximum(ta, tb) / w).astype(np.int64) + 1
    cnt = np.minimum(hi - lo + 1, 18)
    tr = np.repeat(np.arange(n), cnt)
    start = np.repeat(lo, cnt)
    k = np.arange(tr.shape[0]) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    sec = np.mod(start + k, 18)
    sec = np.where(tanl[tr] < 0.0, sec + 18, sec)
    return tr, sec


def generate_event(seed, *, n_tracks, sectors=None, n_sectors=36, pt_mode=("exp", 0.3, 0.1, 20.0),
                   eta_range=(-0.9, 0.9), eta_fold=False, phi_range=(0.0, 2.0 * math.pi),
                   efficiency=0.95, sigma=None, noise_fraction=0.1, smear=True, bz=0.5,
                   qpt=None, keep_exact=False, geometry=None, shuffle=True) -> Event:
    """Generate one collision.

    sectors: restrict hits to these sector numbers (the event then has one
    instance per listed sector); default all ``n_sectors``.
    qpt: optional array overriding q/pT of each track (0 = straight line).
    keep_exact: also return unrounded, unsmeared FP64 positions (y64, z64).
    """
    geom = geometry or default_geometry()
    sigma = sigma or SigmaModel()
    inst_sectors = np.arange(n_sectors, dtype=np.int64) if sectors is None else np.asarray(sectors, np.int64)
    pt, eta, phi, q = _sample_tracks(seed, n_tracks, pt_mode, eta_range[0], eta_range[1], eta_fold,
                                     phi_range[0], phi_range[1])
    qpt_arr = q / pt if qpt is None else np.asarray(qpt, dtype=np.float64)
    tanl = np.sinh(eta)
    tr, sec = _candidate_sectors(geom, qpt_arr, phi, tanl, bz, None if sectors is None else inst_sectors)
    keep_sec = np.isin(sec, inst_sectors)
    tr, sec = tr[keep_sec], sec[keep_sec]

    ys, zs, rows, secs, mcs, cnts, y64s, z64s = [], [], [], [], [], [], [], []
    chunk = 8192
    for b in range(0, tr.shape[0], chunk):
        t, s = tr[b:b + chunk], sec[b:b + chunk]
        y, z, ok = _crossings(geom, qpt_arr[t], phi[t], tanl[t], s, bz)
        pi, ri = np.nonzero(ok)
        yt, zt = y[pi, ri], z[pi, ri]
        cnt = ((t[pi].astype(np.uint64) * np.uint64(36) + s[pi].astype(np.uint64)) * np.uint64(N_ROWS)
               + ri.astype(np.uint64))
        if efficiency < 1.0:
            keep = rng.uniform(seed, S_EFF, cnt) < efficiency
            pi, ri, yt, zt, cnt = pi[keep], ri[keep], yt[keep], zt[keep], cnt[keep]
        if smear:
            sg = sigma(zt)
            ym = yt + sg * rng.normal(seed, S_SMEAR_Y, cnt)
            zm = zt + sg * rng.normal(seed, S_SMEAR_Z, cnt)
        else:
            ym, zm = yt, zt
        ys.append(ym); zs.append(zm); rows.append(ri); secs.append(s[pi]); mcs.append(t[pi]); cnts.append(cnt)
        if keep_exact:
            y64s.append(ym.copy()); z64s.append(zm.copy())
    cat = lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt)
    y_sig, z_sig = cat(ys, np.float64), cat(zs, np.float64)
    row_sig, sec_sig = cat(rows, np.int64), cat(secs, np.int64)
    mc_sig, cnt_sig = cat(mcs, np.int64), cat(cnts, np.uint64)

    # noise: round(f * signal count) clusters per (sector, row), uniform in the row
    y_n, z_n, row_n, sec_n, cnt_n = [np.zeros(0)] * 2 + [np.zeros(0, np.int64)] * 2 + [np.zeros(0, np.uint64)]
    if noise_fraction > 0.0:
        key = sec_sig * N_ROWS + row_sig
        counts = np.bincount(key, minlength=n_sectors * N_ROWS if sectors is None else 36 * N_ROWS)
        n_noise = np.floor(noise_fraction * counts + 0.5).astype(np.int64)
        keys = np.nonzero(n_noise)[0]
        if keys.shape[0]:
            reps = n_noise[keys]
            k_rep = np.repeat(keys, reps)
            j = np.arange(k_rep.shape[0]) - np.repeat(np.cumsum(reps) - reps, reps)
            cnt_n = (k_rep.astype(np.uint64) << np.uint64(20)) + j.astype(np.uint64)
            sec_n, row_n = k_rep // N_ROWS, k_rep % N_ROWS
            xr = geom.row_x[row_n]
            half = xr * geom.tan_half_sector
            y_n = -half + 2.0 * half * rng.uniform(seed, S_NOISE, cnt_n * np.uint64(2))
            zu = geom.z_max * rng.uniform(seed, S_NOISE, cnt_n * np.uint64(2) + np.uint64(1))
            z_n = np.where(sec_n >= 18, -zu, zu)
    y_all = np.concatenate([y_sig, y_n])
    z_all = np.concatenate([z_sig, z_n])
    row_all = np.concatenate([row_sig, row_n]).astype(np.int64)
    sec_all = np.concatenate([sec_sig, sec_n]).astype(np.int64)
    mc_all = np.concatenate([mc_sig, -np.ones(row_n.shape[0], np.int64)])
    uid = np.concatenate([cnt_sig, cnt_n | np.uint64(1 << 62)])
    charge = _moyal_charge(rng.uniform(seed, S_CHARGE, uid))

    # group by instance (listed sector order), random order inside a sector
    inst_of_sector = -np.ones(36, np.int64)
    inst_of_sector[inst_sectors] = np.arange(inst_sectors.shape[0])
    inst = inst_of_sector[sec_all]
    shuf = rng.bits(seed, S_SHUFFLE, uid) if shuffle else uid
    order = np.lexsort((shuf, inst))
    inst = inst[order]
    counts = np.bincount(inst, minlength=inst_sectors.shape[0])
    offs = np.zeros(inst_sectors.shape[0] + 1, np.int64)
    offs[1:] = np.cumsum(counts)
    ev = Event(
        x=geom.row_x[row_all[order]].astype(np.float32),
        y=y_all[order].astype(np.float32),
        z=z_all[order].astype(np.float32),
        charge=charge[order],
        row=row_all[order].astype(np.uint8),
        sector_offsets=offs,
        sectors=inst_sectors.copy(),
        mc=mc_all[order].astype(np.int32),
        n_events=1,
        sectors_per_event=int(inst_sectors.shape[0]),
        bz=bz,
        sigma=sigma,
        truth=dict(pt=pt, eta=eta, phi=phi, q=q, qpt=qpt_arr, tanl=tanl),
        meta=dict(seed=int(seed), n_tracks=int(n_tracks)),
    )
    if keep_exact:
        ev.y64 = y_all[order].copy()
        ev.z64 = z_all[order].copy()
    return ev


def concat_events(events) -> Event:
    """Concatenate collisions into one batch (event-major instance order)."""
    offs = [np.zeros(1, np.int64)]
    base, mc_base = 0, 0
    mcs = []
    tracks = []
    for e in events:
        offs.append(e.sector_offsets[1:] + base)
        base += e.n
        m = e.mc.astype(np.int64)
        mcs.append(np.where(m >= 0, m + mc_base, -1).astype(np.int32))
        nt = e.meta.get("n_tracks", int(m.max() + 1) if m.size else 0)
        nt = list(nt) if isinstance(nt, (list, tuple)) else [int(nt)]   # a batch lists its collisions
        tracks += nt
        mc_base += int(sum(nt))
    cat = lambda name: np.concatenate([getattr(e, name) for e in events])
    ev0 = events[0]
    return Event(cat("x"), cat("y"), cat("z"), cat("charge"), cat("row"), np.concatenate(offs),
                 np.concatenate([e.sectors for e in events]), np.concatenate(mcs),
                 n_events=sum(e.n_events for e in events), sectors_per_event=ev0.sectors_per_event, bz=ev0.bz,
                 sigma=ev0.sigma, meta=dict(n_collisions=sum(e.n_events for e in events), n_tracks=tracks))


def _collision(seed, over):
    kw = dict(n_tracks=impact_tracks(seed), sigma=SigmaModel(0.08, 0.15))
    kw.update(over)
    return generate_event(seed, **kw)


def impact_tracks(seed: int) -> int:
    """Multiplicity of a collision of the uneven-multiplicity workloads:
    b uniform in [0, 15] fm, N = max(10, 9000 (1 - b/15)^2)."""
    b = 15.0 * float(rng.uniform(seed, S_IMPACT, np.array([0], np.uint64))[0])
    return max(10, int(9000.0 * (1.0 - b / 15.0) ** 2))


def generate_config(index: int, instance: int = 0, *, n_collisions=None, **over) -> Event:
    """The workloads.

    0: one 20-degree sector (sector 0), 200 tracks, pT log-uniform 0.2-5 GeV/c,
       |eta| < 0.9 folded onto the A side, phi in the sector, sigma 0.1 cm,
       every row crossed gives a cluster, no noise.
    1: central Pb-Pb-like event: 36 sectors, 9000 tracks, pT ~ exp(-pT/0.3)
       on [0.1, 20] GeV/c, |eta| < 0.9, 95 % row efficiency, sigma 0.08 -> 0.15 cm
       with drift length, 10 % noise per row.
    2: the event of workload 1 (the precision comparison runs on it).
    3: a batch of collisions (default 128) with N = max(10, 9000 (1 - b/15)^2),
       b uniform in [0, 15] fm, otherwise as workload 1.
    """
    if index == 0:
        kw = dict(n_tracks=200, sectors=[0], pt_mode=("loguniform", 0.2, 5.0),
                  eta_range=(0.0, 0.9), eta_fold=True, phi_range=(0.0, math.radians(20.0)),
                  efficiency=1.0, sigma=SigmaModel(0.1, 0.1), noise_fraction=0.0)
        kw.update(over)
        ev = generate_event(seed_for(0, instance), **kw)
        ev.meta["workload"] = "single sector, 200 tracks"
        return ev
    if index in (1, 2):
        kw = dict(n_tracks=9000, sigma=SigmaModel(0.08, 0.15))
        kw.update(over)
        ev = generate_event(seed_for(1, instance), **kw)
        ev.meta["workload"] = "central Pb-Pb-like event, 9000 tracks, 36 sectors"
        return ev
    if index == 3:
        nc = 128 if n_collisions is None else n_collisions
        seeds = [seed_for(3, instance * 100000 + c) for c in range(nc)]
        workers = over.pop("workers", 1)
        if workers and workers > 1 and nc > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
                evs = list(ex.map(_collision, seeds, [over] * nc))
        else:
            evs = [_collision(s, over) for s in seeds]
        ev = concat_events(evs)
        ev.meta["workload"] = f"{nc} collisions, b uniform 0-15 fm"
        return ev
    raise ValueError(index)


def truth_state(ev: Event, label: int, sector: int, x: float, event_index: int = 0):
    """Generator truth of particle ``label`` where its circle crosses local
    x = ``x`` of ``sector``: (y, z, sin phi, tan lambda, q/pT), from the circle
    centre and radius (outward branch, first crossing)."""
    geom = default_geometry()
    t = ev.truth
    qpt, phi0, tanl = t["qpt"][label], t["phi"][label], t["tanl"][label]
    y, z, ok = _crossings(_single_row_geometry(geom, x), np.array([qpt]), np.array([phi0]),
                          np.array([tanl]), np.array([sector]), ev.bz)
    alpha = math.radians(geom.alpha0_deg + (sector % 18) * geom.dalpha_deg)
    phl0 = phi0 - alpha
    rho = -K_B_PER_TESLA * ev.bz * qpt
    if rho == 0.0:
        sphi = math.sin(phl0)
    else:
        cx = -math.sin(phl0) / rho
        sphi = rho * (x - cx)   # (P - centre)_x = sin(phi) / rho on the circle
    return np.array([y[0, 0], z[0, 0], sphi, tanl, qpt]), bool(ok[0, 0])


def _single_row_geometry(geom, x):
    from .geometry import Geometry
    return Geometry(n_sectors=geom.n_sectors, row_x=np.array([float(x)]),
                    tan_half_sector=geom.tan_half_sector, z_max=geom.z_max,
                    alpha0_deg=geom.alpha0_deg, dalpha_deg=geom.dalpha_deg)
