"""The integer-only arithmetic the GPU track-model coder relies on, checked on
the CPU against its plain definition (numpy float64 / Python integers):

- Y = rint(200 y) of a float y formed from its IEEE-754 fields (200 y =
  25 m 2^(E-147) exactly; a right shift rounding half to even);
- the decoder's y = (float)(Y / 200.0) formed as one correctly rounded float
  division (Y / 200 is dyadic or has a binary expansion of period 20, so the
  double-then-float rounding never differs from one rounding);
- floor(a / b) from a float quotient estimate corrected by the remainder.

Each function restates the bit-level steps of the kernel in Python, so a
mistake in the reasoning behind them (not only a typo) fails here."""
import numpy as np


def qpos_fields(v):
    bits = int(np.float32(v).view(np.uint32))
    sign, e, frac = bits >> 31, (bits >> 23) & 0xFF, bits & 0x7FFFFF
    if e == 0:
        return 0
    sh = e - 147
    if e == 255 or sh > 34:
        return None                      # the kernel takes the double expression here
    p = 25 * (frac | 0x800000)
    if sh >= 0:
        q = p << sh
    else:
        s = -sh
        if s >= 31:
            return 0
        q, rem, half = p >> s, p & ((1 << s) - 1), 1 << (s - 1)
        if rem > half or (rem == half and q & 1):
            q += 1
    return -q if sign else q


def test_quantisation_from_ieee_fields():
    rng = np.random.default_rng(11)
    vals = np.concatenate([
        rng.uniform(-260, 260, 40000).astype(np.float32),
        (rng.integers(-52000, 52000, 20000) / 200.0).astype(np.float32),          # on the grid
        ((rng.integers(-52000, 52000, 20000) + 0.5) / 200.0).astype(np.float32),  # halfway cases
        (rng.standard_normal(10000) * 1e-3).astype(np.float32),
        np.array([0.0, -0.0, 0.0025, -0.0025, 0.0075, -0.0125, 1e-30, 3e5, -3e5], np.float32)])
    ref = np.rint(vals.astype(np.float64) * 200.0).astype(np.int64)
    got = np.array([qpos_fields(v) for v in vals], dtype=object)
    assert all(g is not None for g in got)
    assert np.array_equal(got.astype(np.int64), ref)


def test_grid_to_cm_single_rounding():
    ys = np.concatenate([np.arange(-60000, 60001, 3), np.random.default_rng(2).integers(-2**23, 2**23, 100000)])
    double_round = (ys.astype(np.float64) / 200.0).astype(np.float32)
    single = ys.astype(np.float32) / np.float32(200.0)      # IEEE float division, correctly rounded
    assert np.array_equal(double_round, single)


def udiv(a, b):
    if a < (1 << 62) and b < (1 << 40):
        fa = np.float32(np.float64(np.float32(a >> 32)) * 4294967296.0 + np.float64(np.float32(a & 0xFFFFFFFF)))
        fb = np.float32(np.float64(np.float32(b >> 32)) * 4294967296.0 + np.float64(np.float32(b & 0xFFFFFFFF)))
        qf = np.float32(fa / fb)
        if qf < np.float32(1048576.0):
            q = int(qf)
            r = a - q * b
            for _ in range(4):
                if r >= 0:
                    break
                q, r = q - 1, r + b
            for _ in range(4):
                if r < b:
                    break
                q, r = q + 1, r - b
            if 0 <= r < b:
                return q
    return a // b


def test_division_estimate_and_correction():
    rng = np.random.default_rng(5)
    for _ in range(60000):
        b = int(rng.integers(1, 1 << int(rng.integers(1, 41))))
        q = int(rng.integers(0, 1 << 21))
        a = q * b + int(rng.integers(0, b))
        if a >= 1 << 62:
            continue
        assert udiv(a, b) == a // b
