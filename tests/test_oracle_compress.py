"""Pins of the oracle's track-model compression: a hand-encoded frame (byte
for byte); exact round trip of the quantised clusters on the single sector
and the central event; parabola residuals of noiseless helices within one
grid unit; the compressed size."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixture_event():
    fx = json.load(open(os.path.join(HERE, "golden", "tm_hand_fixture.json")))
    c = fx["clusters"]
    g = synth.default_geometry()
    row = np.array([k["row"] for k in c], np.uint8)
    ev = synth.Event(x=g.row_x[row].astype(np.float32), y=np.array([k["y"] for k in c], np.float32),
                     z=np.array([k["z"] for k in c], np.float32), charge=np.array([k["charge"] for k in c], np.uint16),
                     row=row, sector_offsets=np.array([0, len(c)], np.int64), sectors=np.array([0]),
                     mc=np.zeros(len(c), np.int32), sectors_per_event=1)
    tr = np.array(fx["track"], np.int32)
    return fx, ev, np.array([0], np.int32), np.array([tr.shape[0]], np.int32), tr


def test_hand_encoded_frame():
    fx, ev, off, ncl, ids = _fixture_event()
    s = oracle.tm_encode(ev, off, ncl, ids)
    assert s.nbytes == fx["total_bytes"]
    assert list(s.data[:len(fx["track_bytes"])]) == fx["track_bytes"]
    assert list(s.track_off) == [0, len(fx["track_bytes"])]
    assert s.row_off[20] == fx["row20_offset"]
    assert list(s.data[s.row_off[20]:s.row_off[21]]) == fx["row20_bytes"]
    # every other row holds a single zero (no clusters)
    others = [r for r in range(152) if r != 20]
    assert all(s.row_off[r + 1] - s.row_off[r] == 1 and s.data[s.row_off[r]] == 0 for r in others)
    d = oracle.tm_decode(s, 16)
    assert list(d["row"]) == [10, 11, 12, 14, 20, 20]
    assert list(d["charge"]) == [50, 60, 300, 45, 41, 40]
    assert np.array_equal(d["y"], np.float32([1.0, 1.1, 1.2, 1.43, -2.0, -0.5]))
    assert np.array_equal(d["z"], np.float32([10.0, 10.05, 10.1, 10.2, 31.0, 30.0]))


def _expected_decode(ev, res):
    """The quantised clusters in decode order (tracks, then rows sorted by Y, Z, charge)."""
    g = synth.default_geometry()
    Y = np.rint(ev.y.astype(np.float64) * 200.0).astype(np.int64)
    Z = np.rint(ev.z.astype(np.float64) * 200.0).astype(np.int64)
    q = ev.charge.astype(np.int64)
    used = np.zeros(ev.n, bool)
    order = []
    for k in range(res.n_tracks):
        ids = res.track_ids(k)
        used[ids] = True
        order.extend(ids.tolist())
    inst = ev.instance_of_cluster()
    free = np.nonzero(~used)[0]
    key = np.lexsort((q[free], Z[free], Y[free], ev.row[free], inst[free]))
    order.extend(free[key].tolist())
    order = np.array(order, np.int64)
    return dict(row=ev.row[order], charge=ev.charge[order],
                y=(Y[order] / 200.0).astype(np.float32), z=(Z[order] / 200.0).astype(np.float32),
                x=g.row_x[ev.row[order]].astype(np.float32))


@pytest.mark.parametrize("which", [0, 1])
def test_round_trip(which):
    ev = synth.generate_config(which)
    res = oracle.track_event(ev)
    s = oracle.tm_encode(ev, res.tr_offset, res.tr_ncl, res.tr_ids)
    d = oracle.tm_decode(s, ev.n)
    e = _expected_decode(ev, res)
    for k in ("row", "charge", "x", "y", "z"):
        assert np.array_equal(d[k], e[k]), k
    # quantisation error of a position is at most half a grid step (25 um)
    assert np.max(np.abs(np.sort(d["y"]) - np.sort(np.rint(ev.y.astype(np.float64) * 200) / 200))) < 1e-5
    per_cluster = s.nbytes / ev.n
    assert per_cluster < (5.5 if which == 0 else 7.0), per_cluster     # raw: 4 + 4 + 4 + 2 B


def _varints(buf, pos, n):
    out = []
    for _ in range(n):
        v, sh = 0, 0
        while True:
            b = int(buf[pos]); pos += 1
            v |= (b & 127) << sh
            if not b & 128:
                break
            sh += 7
        out.append(v)
    return out, pos


def test_parabola_residuals_of_noiseless_helices():
    # Exact helix crossings: (a) every stored residual equals the quantised
    # value minus the parabola through the three previous quantised points,
    # evaluated here in the Lagrange form in floating point (the oracle uses
    # the Newton form in integers), rounded half away from zero; (b) on the
    # unquantised crossings that parabola predicts the next crossing of a
    # helix to far below the 50 um grid (the model, not the code, is pinned).
    ev = synth.generate_config(0, smear=False, keep_exact=True)
    res = oracle.track_event(ev)
    s = oracle.tm_encode(ev, res.tr_offset, res.tr_ncl, res.tr_ids)
    X = np.rint(synth.default_geometry().row_x * 200.0)
    unz = lambda u: -((u + 1) >> 1) if u & 1 else u >> 1
    rhaf = lambda v: np.sign(v) * np.floor(np.abs(v) + 0.5)
    checked, trunc = 0, []
    for k in range(res.n_tracks):
        ids = res.track_ids(k)
        pos = int(s.track_off[k])
        (m,), pos = _varints(s.data, pos, 1)
        _, pos = _varints(s.data, pos, 4)                  # row, Y0, Z0, charge
        for j in range(1, m):
            (gap, ry, rz, _q), pos = _varints(s.data, pos, 4)
            if j < 3:
                continue
            c = ids[j - 3:j + 1]
            xs, x = X[ev.row[c[:3]]], X[ev.row[c[3]]]
            w = np.array([(x - xs[1]) * (x - xs[2]) / ((xs[0] - xs[1]) * (xs[0] - xs[2])),
                          (x - xs[0]) * (x - xs[2]) / ((xs[1] - xs[0]) * (xs[1] - xs[2])),
                          (x - xs[0]) * (x - xs[1]) / ((xs[2] - xs[0]) * (xs[2] - xs[1]))])
            for r, exact in ((unz(ry), ev.y64), (unz(rz), ev.z64)):
                vq = np.rint(200.0 * exact[c].astype(np.float32).astype(np.float64))
                pq = float(w @ vq[:3])
                if abs(abs(pq - np.trunc(pq)) - 0.5) > 1e-6:
                    assert r == vq[3] - rhaf(pq), (k, j, r, vq, pq)
                    checked += 1
                ve = 200.0 * exact[c]
                trunc.append(abs(ve[3] - w @ ve[:3]))
    trunc = np.array(trunc)
    assert checked > 10000
    assert np.quantile(trunc, 0.999) < 0.1, np.quantile(trunc, 0.999)
