"""Whole-oracle checks against generator truth and symmetries: infinite-pT
lines are found with all their clusters, efficiency and fake rate on the
single sector, mirror invariance, determinism."""
import numpy as np

import oracle
import synth
from synth.truth import evaluate


def test_straight_lines_found_noiseless():
    ev = synth.generate_config(0, qpt=np.zeros(200), smear=False, keep_exact=True)
    res = oracle.track_event(ev, exact=True)
    lab = ev.mc
    n_per = np.bincount(lab[lab >= 0])
    findable = np.nonzero(n_per >= 20)[0]
    assert findable.shape[0] == 200           # straight tracks stay inside the sector
    got = {}
    for k in range(res.n_tracks):
        ids = res.track_ids(k)
        u = np.unique(lab[ids])
        assert u.shape[0] == 1                # pure
        got[int(u[0])] = ids.shape[0]
    for m in findable:
        assert got.get(int(m)) == n_per[m], m  # every cluster of every line
    assert np.allclose(res.tr_param[:, 4], 0.0, atol=1e-9)


def test_straight_lines_found_smeared():
    # 40 lines: with 200 lines from one vertex, a few pairs overlap within sigma
    ev = synth.generate_config(0, n_tracks=40, qpt=np.zeros(40))
    res = oracle.track_event(ev)
    q = evaluate(ev, res.tr_inst, res.tr_offset, res.tr_ncl, res.tr_ids)
    assert q["efficiency"] == 1.0 and q["fake_rate"] == 0.0
    assert res.tr_ids.shape[0] >= 0.995 * ev.n


def test_efficiency_single_sector(event0, oracle0):
    q = evaluate(event0, oracle0.tr_inst, oracle0.tr_offset, oracle0.tr_ncl, oracle0.tr_ids)
    assert q["findable"] > 100
    assert q["efficiency"] >= 0.95 and q["fake_rate"] <= 0.02 and q["clone_rate"] <= 0.02, q


def test_mirror_invariance(event0, oracle0):
    ev = event0
    res_m = oracle.track(synth.default_geometry(), oracle.Cuts.for_event(ev), ev.sector_offsets,
                         -ev.y.astype(np.float64), ev.z, row=ev.row)
    for f in ("up", "down", "upc", "downc", "tl_start", "tl_hits", "weight", "tr_ids", "tr_ncl", "tr_ndf"):
        assert np.array_equal(getattr(oracle0, f), getattr(res_m, f)), f
    sgn = np.array([-1.0, 1.0, -1.0, 1.0, -1.0])
    assert np.allclose(res_m.tr_param, oracle0.tr_param * sgn, rtol=1e-12, atol=1e-12)
    assert np.allclose(res_m.tr_chi2, oracle0.tr_chi2, rtol=1e-10)


def test_deterministic(event0, oracle0):
    again = oracle.track_event(event0)
    assert np.array_equal(again.tr_ids, oracle0.tr_ids)
    assert np.array_equal(again.tr_param, oracle0.tr_param)


def test_empty_and_tiny_inputs():
    g = synth.default_geometry()
    c = oracle.Cuts()
    res = oracle.track(g, c, np.array([0, 0, 0]), np.zeros(0), np.zeros(0), row=np.zeros(0, np.int32))
    assert res.n_tracks == 0 and res.up.shape[0] == 0
    # two clusters: no links, no tracks
    res = oracle.track(g, c, np.array([0, 2]), np.array([0.0, 0.1]), np.array([10.0, 10.1]),
                       row=np.array([5, 6], np.int32))
    assert res.n_tracklets == 0 and np.all(res.up == -1)
    # row from x when no row array is given
    ev = synth.generate_config(0)
    a = oracle.track_event(ev)
    b = oracle.track(g, oracle.Cuts.for_event(ev), ev.sector_offsets, ev.y, ev.z, x=ev.x)
    assert np.array_equal(a.tr_ids, b.tr_ids)
