"""Pins of the oracle's cross-sector merging and chain refit: noiseless
multi-sector particles are linked and refit to generator truth within 1e-9;
chi2 of true pairs follows chi2(5); links are the mutual best pairs of the
tested-pair list (re-derived by sorting); purity and efficiency vs truth."""
import numpy as np
import pytest

import oracle
import synth
from synth.events import truth_state


def _labels(ev, res):
    lab = np.empty(res.n_tracks, np.int64)
    for k in range(res.n_tracks):
        v, c = np.unique(ev.mc[res.track_ids(k)], return_counts=True)
        lab[k] = v[np.argmax(c)]
    return lab


@pytest.fixture(scope="module")
def noiseless():
    ev = synth.generate_event(synth.seed_for(1, 91), n_tracks=400, efficiency=1.0, noise_fraction=0.0,
                              smear=False, keep_exact=True)
    return ev, oracle.track_merge_event(ev, exact=True)


@pytest.fixture(scope="module")
def clean():
    ev = synth.generate_config(1, n_tracks=1500, noise_fraction=0.0)
    return ev, oracle.track_merge_event(ev)


def test_noiseless_chains_refit_to_truth(noiseless):
    ev, (res, mrg) = noiseless
    assert mrg.n_chains > 20
    assert np.all(mrg.ch_status == 0)
    worst = np.zeros(5)
    n = 0
    for k in range(mrg.n_chains):
        ids = mrg.chain_ids(k)
        u = np.unique(ev.mc[ids])
        assert u.shape[0] == 1
        head = int(mrg.ch_head[k])
        sec = int(ev.sectors[res.tr_inst[head]])
        ts, _ = truth_state(ev, int(u[0]), sec, mrg.ch_x_ref[k])
        worst = np.maximum(worst, np.abs(mrg.ch_param[k] - ts) / np.abs(ts))
        n += 1
    assert n > 20 and np.all(worst < 1e-9), worst


def test_noiseless_segments_all_linked(noiseless):
    ev, (res, mrg) = noiseless
    lab = _labels(ev, res)
    sec = ev.sectors[res.tr_inst]
    # segments of one particle in adjacent sectors of the same side
    missing = 0
    total = 0
    for a in range(res.n_tracks):
        for b in range(a + 1, res.n_tracks):
            if lab[a] != lab[b]:
                continue
            sa, sb = int(sec[a]), int(sec[b])
            if sa // 18 != sb // 18 or (sa % 18 - sb % 18) % 18 not in (1, 17):
                continue
            total += 1
            if not (mrg.link_out[a] == b or mrg.link_out[b] == a):
                missing += 1
    assert total > 20 and missing == 0, (missing, total)


def test_true_pair_chi2_distribution(clean):
    ev, (res, mrg) = clean
    lab = _labels(ev, res)
    I = mrg.pairs[:, 0].astype(int)
    O = mrg.pairs[:, 1].astype(int)
    true = (lab[I] == lab[O]) & (lab[I] >= 0)
    chi = mrg.pairs[true, 2]
    assert chi.shape[0] > 150
    # median of chi2 with 5 degrees of freedom is 4.351
    assert abs(np.median(chi) - 4.351) < 0.6, np.median(chi)
    assert (chi < 11.07).mean() > 0.85          # 95 % quantile of chi2(5)


def test_links_are_mutual_best(clean):
    ev, (res, mrg) = clean
    c = oracle.MergeCuts()
    P = mrg.pairs[mrg.pairs[:, 2] <= c.chi2_max]
    K = res.n_tracks
    best_out = -np.ones(K, np.int64)
    best_in = -np.ones(K, np.int64)
    # sort by (inner, chi2, outer) and keep the first of each inner; likewise for outer
    o = np.lexsort((P[:, 1], P[:, 2], P[:, 0]))
    first = np.r_[True, P[o[1:], 0] != P[o[:-1], 0]]
    best_out[P[o[first], 0].astype(int)] = P[o[first], 1].astype(int)
    o = np.lexsort((P[:, 0], P[:, 2], P[:, 1]))
    first = np.r_[True, P[o[1:], 1] != P[o[:-1], 1]]
    best_in[P[o[first], 1].astype(int)] = P[o[first], 0].astype(int)
    want = np.where((best_out >= 0) & (best_in[np.maximum(best_out, 0)] == np.arange(K)), best_out, -1)
    assert np.array_equal(want, mrg.link_out)


def test_purity_and_efficiency_central_event():
    ev = synth.generate_config(1)
    res, mrg = oracle.track_merge_event(ev)
    lab = _labels(ev, res)
    k = np.nonzero(mrg.link_out >= 0)[0]
    assert k.shape[0] > 3000
    assert (lab[k] == lab[mrg.link_out[k]]).mean() > 0.99
    # efficiency over pairs of good segments of one particle in adjacent sectors
    sec = ev.sectors[res.tr_inst]
    by = {}
    for t in range(res.n_tracks):
        if lab[t] >= 0:
            by.setdefault(int(lab[t]), []).append(t)
    total = linked = 0
    for ts in by.values():
        for i in range(len(ts)):
            for j in range(i + 1, len(ts)):
                a, b = ts[i], ts[j]
                sa, sb = int(sec[a]), int(sec[b])
                if sa // 18 == sb // 18 and (sa % 18 - sb % 18) % 18 in (1, 17):
                    total += 1
                    linked += mrg.link_out[a] == b or mrg.link_out[b] == a
    assert total > 3000 and linked / total > 0.9, (linked, total)
    assert np.all(mrg.ch_status == 0)
