"""Pins of the oracle's helix transport and Jacobian against closed forms:
the generator's exact circle geometry, straight lines, round trips, mirror
symmetry and central finite differences."""
import math
import numpy as np
import pytest

import oracle
import synth
from synth.events import truth_state

BZ, SMAX = 0.5, 0.999
G = synth.default_geometry()


def _tracks(n=60, seed=7):
    r = np.random.default_rng(seed)
    pt = np.exp(r.uniform(np.log(0.12), np.log(20.0), n))
    q = r.choice([-1.0, 1.0], n)
    eta = r.uniform(0.0, 0.9, n)
    phi = np.radians(r.uniform(2.0, 18.0, n))
    return q / pt, np.sinh(eta), phi


def _event_with(qpt, tanl, phi):
    ev = synth.generate_config(0, n_tracks=1)
    ev.truth = dict(qpt=np.asarray(qpt), tanl=np.asarray(tanl), phi=np.asarray(phi))
    return ev


def test_transport_matches_circle_geometry():
    qpt, tanl, phi = _tracks()
    ev = _event_with(qpt, tanl, phi)
    checked = 0
    for m in range(len(qpt)):
        rows = [r for r in (0, 17, 63, 90, 127, 151) if truth_state(ev, m, 0, G.row_x[r])[1]]
        for a, b in zip(rows[:-1], rows[1:]):
            sa, _ = truth_state(ev, m, 0, G.row_x[a])
            sb, _ = truth_state(ev, m, 0, G.row_x[b])
            if max(abs(sa[2]), abs(sb[2])) >= SMAX:
                continue
            for x0, x1, s0, s1 in ((G.row_x[a], G.row_x[b], sa, sb), (G.row_x[b], G.row_x[a], sb, sa)):
                rc, p1, _ = oracle.propagate(BZ, SMAX, x0, x1, s0)
                assert rc == 0
                assert abs(p1[0] - s1[0]) < 1e-9 and abs(p1[1] - s1[1]) < 1e-9, (m, a, b)
                assert abs(p1[2] - s1[2]) < 1e-12
                assert p1[3] == s0[3] and p1[4] == s0[4]
                checked += 1
    assert checked > 100


def test_straight_line_closed_form():
    r = np.random.default_rng(3)
    for _ in range(200):
        s, t = r.uniform(-0.9, 0.9), r.uniform(-1.0, 1.0)
        x0, x1 = r.uniform(85, 240, 2)
        p0 = np.array([r.uniform(-20, 20), r.uniform(-200, 200), s, t, 0.0])
        rc, p1, _ = oracle.propagate(BZ, SMAX, x0, x1, p0)
        c = math.sqrt(1 - s * s)
        assert rc == 0
        assert abs(p1[0] - (p0[0] + (x1 - x0) * s / c)) < 1e-11
        assert abs(p1[1] - (p0[1] + t * (x1 - x0) / c)) < 1e-11
        assert p1[2] == s


def test_round_trip_and_jacobian_composition():
    r = np.random.default_rng(4)
    for _ in range(200):
        p0 = np.array([r.uniform(-20, 20), r.uniform(-200, 200), r.uniform(-0.6, 0.6),
                       r.uniform(-1, 1), r.uniform(-5, 5)])
        x0, x1 = r.uniform(85, 140), r.uniform(140, 235)
        rc, p1, F01 = oracle.propagate(BZ, SMAX, x0, x1, p0)
        if rc:
            continue
        rc, p2, F10 = oracle.propagate(BZ, SMAX, x1, x0, p1)
        assert rc == 0
        assert np.allclose(p2, p0, rtol=0, atol=1e-10)
        assert np.allclose(F10 @ F01, np.eye(5), atol=1e-9)


def test_sinphi_limit():
    # s1 = s0 + rho dx beyond s_max fails
    p0 = np.array([0.0, 0.0, 0.9, 0.1, 5.0])   # rho = -k_B * 5: s decreases outward
    rc, _, _ = oracle.propagate(BZ, SMAX, 100.0, 50.0, p0)   # inward: s increases
    assert rc == 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jacobian_central_differences(seed):
    r = np.random.default_rng(seed)
    for _ in range(40):
        # F does not depend on y0, z0 (translation invariance); zero offsets keep
        # the differences free of cancellation
        p0 = np.array([0.0, 0.0, r.uniform(-0.7, 0.7), r.uniform(-1, 1), r.uniform(-8, 8)])
        x0 = r.uniform(85, 235)
        x1 = x0 + r.choice([-1, 1]) * r.uniform(0.5, 30)
        rc, _, F = oracle.propagate(BZ, SMAX, x0, x1, p0)
        if rc:
            continue
        num = np.zeros((5, 5))
        for j in range(5):
            h = 1e-5 * max(1.0, abs(p0[j]))
            pp, pm = p0.copy(), p0.copy()
            pp[j] += h
            pm[j] -= h
            rp, a, _ = oracle.propagate(BZ, SMAX, x0, x1, pp, want_jacobian=False)
            rm, b, _ = oracle.propagate(BZ, SMAX, x0, x1, pm, want_jacobian=False)
            assert rp == 0 and rm == 0
            num[:, j] = (a - b) / (2 * h)
        scale = np.maximum(np.abs(num), 1e-3)
        assert np.all(np.abs(F - num) / scale < 1e-6), (F, num)


def test_mirror_symmetry():
    r = np.random.default_rng(5)
    for _ in range(200):
        p0 = np.array([r.uniform(-20, 20), r.uniform(-200, 200), r.uniform(-0.7, 0.7),
                       r.uniform(-1, 1), r.uniform(-8, 8)])
        x0, x1 = r.uniform(85, 235, 2)
        m0 = p0 * np.array([-1, 1, -1, 1, -1])
        ra, a, Fa = oracle.propagate(BZ, SMAX, x0, x1, p0)
        rb, b, Fb = oracle.propagate(BZ, SMAX, x0, x1, m0)
        assert ra == rb
        if ra:
            continue
        assert np.array_equal(b, a * np.array([-1, 1, -1, 1, -1]))
        S = np.diag([-1.0, 1, -1, 1, -1])
        assert np.allclose(Fb, S @ Fa @ S, rtol=1e-15, atol=0)
