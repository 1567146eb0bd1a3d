"""Pins of the oracle's sector-frame rotation (used by cross-sector merging):
the generator's circle geometry seen from two sector frames, the round trip,
and central finite differences of the exact rotate-then-return-to-plane map."""
import math

import numpy as np

import oracle
import synth
from synth.events import truth_state

BZ, SMAX = 0.5, 0.999
G = synth.default_geometry()
D20 = math.radians(20.0)


def _boundary_event(n=40, seed=5):
    # tracks heading close to the 20-degree boundary between sectors 0 and 1
    r = np.random.default_rng(seed)
    ev = synth.generate_config(0, n_tracks=1)
    pt = np.exp(r.uniform(np.log(0.3), np.log(10.0), n))
    q = r.choice([-1.0, 1.0], n)
    ev.truth = dict(qpt=q / pt, tanl=np.sinh(r.uniform(0.0, 0.9, n)), phi=np.radians(r.uniform(17.0, 23.0, n)))
    return ev


def test_rotation_matches_circle_geometry_across_sectors():
    ev = _boundary_event()
    checked = 0
    for m in range(len(ev.truth["qpt"])):
        for r_a, r_b in ((20, 60), (60, 100), (100, 140), (40, 41)):
            sa, ok_a = truth_state(ev, m, 0, G.row_x[r_a])
            sb, ok_b = truth_state(ev, m, 1, G.row_x[r_b])
            if abs(sa[2]) > 0.95 or abs(sb[2]) > 0.95:
                continue
            rc, x1, p1, _ = oracle.rotate(BZ, SMAX, D20, G.row_x[r_a], sa, want_jacobian=False)
            if rc:
                continue
            rc, p2, _ = oracle.propagate(BZ, SMAX, x1, G.row_x[r_b], p1, want_jacobian=False)
            if rc:
                continue
            assert abs(p2[0] - sb[0]) < 1e-9 and abs(p2[1] - sb[1]) < 1e-9, (m, r_a, r_b, p2, sb)
            assert abs(p2[2] - sb[2]) < 1e-12
            checked += 1
    assert checked > 60


def test_rotation_round_trip_and_jacobian_inverse():
    r = np.random.default_rng(2)
    for _ in range(200):
        p0 = np.array([r.uniform(-20, 20), r.uniform(-200, 200), r.uniform(-0.6, 0.6), r.uniform(-1, 1),
                       r.uniform(-5, 5)])
        x0 = r.uniform(85, 235)
        d = r.choice([-1, 1]) * D20
        rc, x1, p1, F1 = oracle.rotate(BZ, SMAX, d, x0, p0)
        if rc:
            continue
        rc, x2, p2, F2 = oracle.rotate(BZ, SMAX, -d, x1, p1)
        assert rc == 0
        assert abs(x2 - x0) < 1e-11 and np.allclose(p2, p0, rtol=0, atol=1e-12)
        assert np.allclose(F2 @ F1, np.eye(5), atol=1e-9)


def test_rotation_jacobian_central_differences():
    r = np.random.default_rng(4)
    for _ in range(60):
        p0 = np.array([r.uniform(-15, 15), r.uniform(-100, 100), r.uniform(-0.5, 0.5), r.uniform(-1, 1),
                       r.uniform(-4, 4)])
        x0 = r.uniform(85, 235)
        d = r.choice([-1, 1]) * D20
        rc, x1, p1, F = oracle.rotate(BZ, SMAX, d, x0, p0)
        if rc:
            continue

        def f(p):
            rc_, xa, pa, _ = oracle.rotate(BZ, SMAX, d, x0, p, want_jacobian=False)
            assert rc_ == 0
            rc_, pb, _ = oracle.propagate(BZ, SMAX, xa, x1, pa, want_jacobian=False)
            assert rc_ == 0
            return pb

        num = np.zeros((5, 5))
        for j in range(5):
            h = 1e-6 * max(1.0, abs(p0[j]))
            a, b = p0.copy(), p0.copy()
            a[j] += h
            b[j] -= h
            num[:, j] = (f(a) - f(b)) / (2 * h)
        assert np.all(np.abs(F - num) <= 1e-6 * np.maximum(np.abs(num), 1e-3)), (F, num)
