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


def digitize(ev, readout: Readout = None, seed: int = None, shuffle: bool = True) -> Digits:
    """Digits of a synthetic event's crossings (use an event generated with
    smear=False and noise_fraction=0: its clusters are the exact crossings).
    Truth: the crossing positions per instance/row, their continuous pad and
    time coordinates and their amplitudes."""
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
    p0 = np.rint(u).astype(np.int64)
    t0 = np.rint(v).astype(np.int64)
    offs = np.arange(-WINDOW, WINDOW + 1)
    pc = p0[:, None] + offs[None, :]                      # [hits, 5]
    tc = t0[:, None] + offs[None, :]
    fu = _phi((pc + 0.5 - u[:, None]) / su[:, None]) - _phi((pc - 0.5 - u[:, None]) / su[:, None])
    fv = _phi((tc + 0.5 - v[:, None]) / sv[:, None]) - _phi((tc - 0.5 - v[:, None]) / sv[:, None])
    okp = (pc >= 0) & (pc < npad[:, None])
    okt = (tc >= 0) & (tc < ro.n_time)
    val = amp[:, None, None] * (fu * okp)[:, :, None] * (fv * okt)[:, None, :]
    # cell key: ((instance * 152 + row) * 256 + pad) * 512 + time
    rk = (inst * N_ROWS + row)
    key = ((rk[:, None, None] * 256 + np.clip(pc, 0, 255)[:, :, None]) * 512
           + np.clip(tc, 0, 511)[:, None, :])
    m = (okp[:, :, None] & okt[:, None, :]).ravel()
    key = key.ravel()[m]
    val = val.ravel()[m]
    ukey, inv = np.unique(key, return_inverse=True)
    sval = np.bincount(inv, weights=val, minlength=ukey.shape[0])
    noise = ro.noise_sigma * rng.normal(seed, S_DIGIT_NOISE, ukey.astype(np.uint64))
    adc = np.clip(np.floor(sval + noise + 0.5), 0, ro.adc_max).astype(np.int64)
    keep = adc >= ro.threshold
    skey, sadc = ukey[keep], adc[keep]

    # isolated noise digits: round(f * signal digits) per (instance, row)
    n_rk = ev.n_instances * N_ROWS
    cnt = np.bincount(skey // (256 * 512), minlength=n_rk)
    n_noise = np.floor(ro.noise_digit_fraction * cnt + 0.5).astype(np.int64)
    rks = np.nonzero(n_noise)[0]
    if rks.shape[0]:
        reps = n_noise[rks]
        rk_rep = np.repeat(rks, reps)
        j = np.arange(rk_rep.shape[0]) - np.repeat(np.cumsum(reps) - reps, reps)
        c = (rk_rep.astype(np.uint64) << np.uint64(20)) + j.astype(np.uint64)
        up = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3))
        ut = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3) + np.uint64(1))
        ua = rng.uniform(seed, S_NOISE_DIGIT, c * np.uint64(3) + np.uint64(2))
        np_row = n_pad_row[rk_rep % N_ROWS]
        nkey = (rk_rep * 256 + np.floor(up * np_row).astype(np.int64)) * 512 + np.floor(ut * ro.n_time).astype(np.int64)
        nadc = ro.threshold + np.floor(ua * 4).astype(np.int64)
        # a noise digit on an occupied cell (or a repeated one) is dropped
        fresh = ~np.isin(nkey, skey)
        nkey, nadc = nkey[fresh], nadc[fresh]
        nkey, first = np.unique(nkey, return_index=True)
        nadc = nadc[first]
        skey = np.concatenate([skey, nkey])
        sadc = np.concatenate([sadc, nadc])
    rk_all = skey // (256 * 512)
    pad = (skey // 512) % 256
    tim = skey % 512
    tie = rng.bits(seed, S_NOISE_DIGIT + 1, skey.astype(np.uint64)) if shuffle else skey.astype(np.uint64)
    order = np.lexsort((tie, rk_all))                    # grouped by (instance, row), shuffled inside
    rk_all = rk_all[order]
    offsets = np.zeros(n_rk + 1, np.int64)
    offsets[1:] = np.cumsum(np.bincount(rk_all, minlength=n_rk))
    truth = dict(inst=inst, row=row, y=y, z=z, u=u, v=v, amp=amp, mc=ev.mc.copy())
    return Digits(pad=pad[order].astype(np.uint16), time=tim[order].astype(np.uint16),
                  adc=sadc[order].astype(np.uint16), row_offsets=offsets, sectors=ev.sectors.copy(),
                  readout=ro, n_pad=n_pad_row, truth=truth)


def generate_digits(config_index: int = 1, instance: int = 0, **kw) -> Digits:
    """Digits of the exact crossings of a workload's event (the single
    sector or the central Pb-Pb-like event), without cluster noise."""
    from .events import generate_config
    ev = generate_config(config_index, instance=instance, smear=False, noise_fraction=0.0,
                         keep_exact=True, **kw)
    return digitize(ev)
