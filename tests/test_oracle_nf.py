"""Pins of the oracle's neighbour finder, link cleaning, start hits and
selection: a hand-computed fixture, an all-pairs scan, and the set
definitions checked by independent (sorting / chain-walking) methods."""
import json
import os

import numpy as np

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixture():
    with open(os.path.join(HERE, "golden", "nf_hand_fixture.json")) as f:
        return json.load(f)


def test_hand_fixture():
    fx = _fixture()
    cl = sorted(fx["clusters"], key=lambda c: c["id"])
    n = len(cl)
    geom = synth.Geometry(row_x=np.array(fx["row_x"]), tan_half_sector=10.0, z_max=500.0)
    cuts = oracle.Cuts(**fx["cuts"])
    y = np.array([c["y"] for c in cl])
    z = np.array([c["z"] for c in cl])
    row = np.array([c["row"] for c in cl], np.int32)
    res = oracle.track(geom, cuts, np.array([0, n]), y, z, row=row)
    exp = fx["expected"]
    for name in ("up", "down", "upc", "downc"):
        want = -np.ones(n, np.int32)
        for k, v in exp[name].items():
            want[int(k)] = v
        assert np.array_equal(getattr(res, name), want), (name, getattr(res, name), want)
    assert sorted(res.tl_start.tolist()) == exp["start"]


def test_window_scan_equals_all_pairs(event0):
    a = oracle.track_event(event0)
    b = oracle.track_event(event0, brute_force_nf=True)
    for f in ("up", "down", "upc", "downc", "tl_start", "tl_nhits", "tr_ids", "tr_ncl"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert np.array_equal(a.nf_margin, b.nf_margin)


def test_window_scan_equals_all_pairs_dense():
    ev = synth.generate_config(1, sectors=[3], n_sectors=36)
    a = oracle.track_event(ev)
    b = oracle.track_event(ev, brute_force_nf=True)
    for f in ("up", "down", "tl_start", "tr_ids"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def _check_links_and_starts(res, ev):
    up, down, upc, downc = res.up, res.down, res.upc, res.downc
    n = up.shape[0]
    idx = np.arange(n)
    # cleaned links are reciprocal, a subset of the raw links, and maximal
    m = upc >= 0
    assert np.array_equal(downc[upc[m]], idx[m])
    m = downc >= 0
    assert np.array_equal(upc[downc[m]], idx[m])
    assert np.all((upc < 0) | (upc == up)) and np.all((downc < 0) | (downc == down))
    recip = (up >= 0) & (down[np.maximum(up, 0)] == idx)
    assert np.array_equal(upc >= 0, recip)
    # links join adjacent rows only
    row = ev.row.astype(np.int64)
    assert np.all(row[up[up >= 0]] == row[up >= 0] + 1)
    assert np.all(row[down[down >= 0]] == row[down >= 0] - 1)
    # start hits = bottoms of cleaned chains with at least three hits (walk the chains)
    starts = []
    for h in np.nonzero((downc < 0) & (upc >= 0))[0]:
        length, k = 1, h
        while upc[k] >= 0:
            k = upc[k]
            length += 1
        if length >= 3:
            starts.append(h)
    assert sorted(starts) == sorted(res.tl_start.tolist())
    # start order: by (instance, row, id)
    key = list(zip(res.tl_inst.tolist(), row[res.tl_start].tolist(), res.tl_start.tolist()))
    assert key == sorted(key)


def test_clean_and_start_definitions(event0, oracle0):
    _check_links_and_starts(oracle0, event0)


def test_selection_definitions(event0, oracle0):
    res = oracle0
    T = res.n_tracklets
    rank = np.zeros(T, np.int64)
    for i in np.unique(res.tl_inst):
        sel = np.nonzero(res.tl_inst == i)[0]
        rank[sel] = np.arange(sel.shape[0])
    w = (res.tl_nhits.astype(np.int64) << 20) | ((1 << 20) - 1 - rank)
    # W by sorting (cluster, weight) pairs and taking the last of each cluster
    t_idx, r_idx = np.nonzero(res.tl_hits >= 0)
    cl = res.tl_hits[t_idx, r_idx].astype(np.int64)
    order = np.lexsort((w[t_idx], cl))
    cl_s, w_s = cl[order], w[t_idx][order]
    last = np.r_[cl_s[1:] != cl_s[:-1], True]
    W = np.zeros(event0.n, np.int64)
    W[cl_s[last]] = w_s[last]
    assert np.array_equal(W, res.weight.astype(np.int64))
    # accepted tracks: owned clusters, cuts, order
    nh = (res.tl_hits >= 0).sum(1)
    assert np.array_equal(nh, res.tl_nhits)
    expect = []
    for t in range(T):
        hits = res.tl_hits[t][res.tl_hits[t] >= 0]
        own = hits[W[hits] == w[t]]
        shared = hits.shape[0] - own.shape[0]
        if own.shape[0] >= 20 and shared <= 0.1 * hits.shape[0]:
            expect.append((t, own.tolist()))
    assert [e[0] for e in expect] == res.tr_tracklet.tolist()
    for k, (t, own) in enumerate(expect):
        assert res.track_ids(k).tolist() == own
    # the tracks partition the clusters they use
    assert np.unique(res.tr_ids).shape[0] == res.tr_ids.shape[0]
