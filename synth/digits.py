"""Seeded synthetic TPC digits: the input of cluster finding.

A digit is the zero-suppressed ADC value of one (pad, time bin) cell of a
pad row.  The charge of every particle crossing of a synthetic event (the
exact, unsmeared crossing points of ``synth.events``) is spread over the
cells around it as a two-dimensional Gaussian whose widths grow with the
drift length (pad response plus transverse diffusion across pads,
shaping plus longitudinal diffusion along time), summed over crossings,
digitised with Gaussian electronic noise and rounding, clamped to 10 bits
and zero-suppressed.  Isolated noise digits are added per pad row.

Readout model (a stand-in: the paper gives no detector numbers):
  pads    0.4 cm pitch on rows 0-62, 0.6 cm on rows 63-151; row r has
          n_pad = 2 ceil(x_r tan(10 deg) / pitch) pads, pad p centred at
          y = (p + 0.5 - n_pad / 2) * pitch
  time    bins of 0.5 cm of drift length d = z_max - |z|, 500 bins; bin t
          centred at d = (t + 0.5) * 0.5 cm
  widths  sigma_pad = sqrt(0.25^2 + 0.0209^2 d) cm,
          sigma_time = sqrt(0.20^2 + 0.0220^2 d) cm
  charge  the crossing's Landau-like charge times a gain of 10 ADC counts,
          spread over the 5 x 5 cells around the crossing
  noise   sigma 1 ADC per signal cell; zero suppression keeps ADC >= 3;
          isolated noise digits: round(0.05 x signal digits) per row, ADC 3-6

This module holds no step of the cluster finder.  Random numbers come from
``synth.rng`` (stream 8: digit noise, stream 9: noise digits).
"""
from dataclasses import dataclass
import math
import numpy as np

from . import rng
from .geometry import default_geometry, N_ROWS

S_DIGIT_NOISE, S_NOISE_DIGIT = 8, 9
WINDOW = 2            # cells on each side of the crossing that receive charge


@dataclass
class Readout:
    pad_pitch_inner: float = 0.4
    pad_pitch_outer: float = 0.6
    n_inner_rows: int = 63
    time_bin: float = 0.5
    n_time: int = 500
    z_max: float = 250.0
    gain: float = 10.0
    noise_sigma: float = 1.0
    threshold: int = 3
    adc_max: int = 1023
    noise_digit_fraction: float = 0.05

    def pitch(self, row):
        row = np.asarray(row)
        return np.where(row < self.n_inner_rows, self.pad_pitch_inner, self.pad_pitch_outer)

    def n_pad(self, row_x, tan_half, row):
        row = np.asarray(row)
        return (2 * np.ceil(np.asarray(row_x)[row] * tan_half / self.pitch(row) - 1e-9)).astype(np.int64)

    @staticmethod
    def sigma_pad(d):
        return np.sqrt(0.25 ** 2 + 0.0209 ** 2 * d)

    @staticmethod
    def sigma_time(d):
        return np.sqrt(0.20 ** 2 + 0.0220 ** 2 * d)


@dataclass
class Digits:
    """Digits grouped by (sector instance, pad row); any order inside a row.
    ``row_offsets`` has n_instances * 152 + 1 entries."""
    pad: np.ndarray          # uint16
    time: np.ndarray         # uint16
    adc: np.ndarray          # uint16
    row_offsets: np.ndarray  # int64
    sectors: np.ndarray      # sector number of each instance
    readout: Readout
    n_pad: np.ndarray        # [152] pads per row
    truth: dict

    @property
    def n(self) -> int:
        return int(self.adc.shape[0])

    @property
    def n_instances(self) -> int:
        return int(self.sectors.shape[0])


def _phi(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0)))


def _instance_digits(args):
    """Digit cells (local key (row * 256 + pad) * 512 + time) and ADC values
    of one sector instance."""
    i, seed, ro, n_pad_row, row, u, v, su, sv, amp, shuffle = args
    cells_per_inst = N_ROWS * 256 * 512
    if row.shape[0] == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    p0 = np.rint(u).astype(np.int64)
    t0 = np.rint(v).astype(np.int64)
    offs = np.arange(-WINDOW, WINDOW + 1)
    pc = p0[:, None] + offs[None, :]                      # [hits, 5]
    tc = t0[:, None] + offs[None, :]
    fu = _phi((pc + 0.5 - u[:, None]) / su[:, None]) - _phi((pc - 0.5 - u[:, None]) / su[:, None])
    fv = _phi((tc + 0.5 - v[:, None]) / sv[:, None]) - _phi((tc - 0.5 - v[:, None]) / sv[:, None])
    okp = (pc >= 0) & (pc < n_pad_row[row][:, None])
    okt = (tc >= 0) & (tc < ro.n_time)
    val = amp[:, None, None] * (fu * okp)[:, :, None] * (fv * okt)[:, None, :]
    m = okp[:, :, None] & okt[:, None, :]
    local = ((row[:, None, None] * 256 + np.clip(pc, 0, 255)[:, :, None]) * 512
             + np.clip(tc, 0, 511)[:, None, :])
    grid = np.bincount(local[m], weights=val[m], minlength=cells_per_inst)
    cell = np.nonzero(grid)[0]
    noise = ro.noise_sigma * rng.normal(seed, S_DIGIT_NOISE, (cell + i * cells_per_inst).astype(np.uint64))
    adc = np.clip(np.floor(grid[cell] + noise + 0.5), 0, ro.adc_max).astype(np.int64)
    keep = adc >= ro.threshold
    cell, adc = cell[keep], adc[keep]
    # isolated noise digits: round(f * signal digits) per row, dropped on occupied cells
    cnt = np.bincount(cell // (256 * 512), minlength=N_ROWS)
    n_noise = np.floor(ro.noise_digit_fraction * cnt + 0.5).astype(np.int64)
    rws = np.nonzero(n_noise)[0]
    if rws.shape[0]:
        reps = n_noise[rws]
        r_rep = np.repeat(rws, reps)
        j = np.arange(r_rep.shape[0]) - np.repeat(np.cumsum(reps) - reps, reps)
        c = ((np.uint64(i * N_ROWS) + r_rep.astype(np.uint64)) << np.uint64(20)) + j.astype(np.uint64)
        up = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3))
        ut = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3) + np.uint64(1))
        ua = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3) + np.uint64(2))
        ncell = (r_rep * 256 + np.floor(up * n_pad_row[r_rep]).astype(np.int64)) * 512 \
            + np.floor(ut * ro.n_time).astype(np.int64)
        nadc = ro.threshold + np.floor(ua * 4).astype(np.int64)
        occupied = np.zeros(cells_per_inst, bool)
        occupied[cell] = True
        ncell, first = np.unique(ncell, return_index=True)
        nadc = nadc[first]
        fresh = ~occupied[ncell]
        cell = np.concatenate([cell, ncell[fresh]])
        adc = np.concatenate([adc, nadc[fresh]])
    gkey = cell + i * cells_per_inst
    # grouped by row, in a seeded random order inside each row
    tie = rng.bits(seed, S_NOISE_DIGIT + 1, gkey.astype(np.uint64)) if shuffle else gkey.astype(np.uint64)
    order = np.argsort((cell // (256 * 512)).astype(np.uint64) << np.uint64(48)
                       | (tie & np.uint64((1 << 48) - 1)), kind="stable")
    return gkey[order], adc[order]


def digitize(ev, readout: Readout = None, seed: int = None, shuffle: bool = True, workers: int = 1) -> Digits:
    """Digits of a synthetic event's crossings (use an event generated with
    smear=False and noise_fraction=0: its clusters are the exact crossings).
    Truth: the crossing positions per instance/row, their continuous pad and
    time coordinates and their amplitudes.  ``workers`` > 1 digitises the
    sector instances in a spawn process pool (same result)."""
    ro = readout or Readout()
    geom = default_geometry()
    seed = int(ev.meta.get("seed", 0)) if seed is None else int(seed)
    n_pad_row = ro.n_pad(geom.row_x, geom.tan_half_sector, np.arange(N_ROWS))
    inst = ev.instance_of_cluster()
    row = ev.row.astype(np.int64)
    y = ev.y64 if ev.y64 is not None else ev.y.astype(np.float64)
    z = ev.z64 if ev.z64 is not None else ev.z.astype(np.float64)
    pitch = ro.pitch(row)
    npad = n_pad_row[row]
    d = np.clip(ro.z_max - np.abs(z), 0.0, ro.z_max)
    u = y / pitch + npad / 2.0 - 0.5                      # continuous pad coordinate (pad p centred at p)
    v = d / ro.time_bin - 0.5                             # continuous time coordinate
    su = ro.sigma_pad(d) / pitch
    sv = ro.sigma_time(d) / ro.time_bin
    amp = ro.gain * ev.charge.astype(np.float64)
    n_rk = ev.n_instances * N_ROWS
    order_h = np.argsort(inst, kind="stable")
    bounds = np.searchsorted(inst[order_h], np.arange(ev.n_instances + 1))
    jobs = []
    for i in range(ev.n_instances):
        h = order_h[bounds[i]:bounds[i + 1]]
        jobs.append((i, seed, ro, n_pad_row, row[h], u[h], v[h], su[h], sv[h], amp[h], shuffle))
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_instance_digits, jobs, chunksize=1))
    else:
        parts = [_instance_digits(j) for j in jobs]
    skey = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, np.int64)
    sadc = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.int64)
    rk_all = skey // (256 * 512)
    pad = (skey // 512) % 256
    tim = skey % 512
    offsets = np.zeros(n_rk + 1, np.int64)
    offsets[1:] = np.cumsum(np.bincount(rk_all, minlength=n_rk))
    truth = dict(inst=inst, row=row, y=y, z=z, u=u, v=v, amp=amp, mc=ev.mc.copy())
    return Digits(pad=pad.astype(np.uint16), time=tim.astype(np.uint16),
                  adc=sadc.astype(np.uint16), row_offsets=offsets, sectors=ev.sectors.copy(),
                  readout=ro, n_pad=n_pad_row, truth=truth)


def generate_digits(config_index: int = 1, instance: int = 0, workers: int = 1, **kw) -> Digits:
    """Digits of the exact crossings of a workload's event (the single
    sector or the central Pb-Pb-like event), without cluster noise."""
    from .events import generate_config
    ev = generate_config(config_index, instance=instance, smear=False, noise_fraction=0.0,
                         keep_exact=True, **kw)
    return digitize(ev, workers=workers)
