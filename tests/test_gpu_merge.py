"""Cross-sector merging on the GPU against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_09138_gb300.build as b
    b.build()
    import paper_2502_09138_gb300 as G
    return G


def _run(G, ev, precision="mixed"):
    import torch
    trk = G.Tracker(precision=precision, bz=ev.bz,
                    cuts=G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode))
    dc = G.DeviceClusters.from_event(ev)
    tracks = trk.track(dc)
    sec, evi = oracle.event_instances(ev)
    ch = trk.merge(dc, tracks, sec, evi, int(evi.max()) + 1)
    torch.cuda.synchronize()
    th = tracks.to_host()
    return th, ch.to_host(th["n_tracks"])


def _compare(ev, ores, mres, gtr, gch, tol=1e-5):
    # sector tracks identical -> same track indices on both sides
    assert gtr["n_tracks"] == ores.n_tracks
    assert np.array_equal(gtr["cluster_ids"], ores.tr_ids)
    mis = np.nonzero(gch["link_out"] != mres.link_out)[0]
    excused = [k for k in mis if mres.margin[k] < tol or
               (mres.link_out[k] >= 0 and mres.margin[mres.link_out[k]] < tol) or
               (gch["link_out"][k] >= 0 and mres.margin[gch["link_out"][k]] < tol)]
    assert len(mis) == len(excused), (len(mis), len(excused))
    assert len(excused) <= 1e-3 * max(1, ores.n_tracks)
    if len(mis):
        return
    assert gch["n_chains"] == mres.n_chains
    assert np.array_equal(gch["head"], mres.ch_head)
    assert np.array_equal(gch["n_seg"], mres.ch_nseg)
    assert np.array_equal(gch["segs"], mres.ch_segs)
    assert np.array_equal(gch["cluster_ids"], mres.ch_ids)
    assert np.array_equal(gch["status"], mres.ch_status)
    ok = mres.ch_status == 0
    di = [0, 2, 5, 9, 14]
    sig = np.sqrt(np.abs(mres.ch_cov[:, di]))
    scale = np.maximum(np.abs(mres.ch_param), sig)
    assert np.all((np.abs(gch["param"] - mres.ch_param) / scale)[ok] <= 1e-4)
    ii, jj = np.tril_indices(5)
    cs = np.sqrt(np.abs(mres.ch_cov[:, [di[i] for i in ii]] * mres.ch_cov[:, [di[j] for j in jj]]))
    assert np.all((np.abs(gch["cov"] - mres.ch_cov) / np.where(cs > 0, cs, 1))[ok] <= 1e-3)
    assert np.all(np.abs(gch["chi2"] - mres.ch_chi2)[ok] <= 1e-4 * np.maximum(mres.ch_chi2[ok], 1.0))


def test_merge_central_event(G):
    ev = synth.generate_config(1)
    ores, mres = oracle.track_merge_event(ev)
    gtr, gch = _run(G, ev)
    assert mres.n_chains > 3000
    _compare(ev, ores, mres, gtr, gch)


def test_merge_collision_batch(G):
    ev = synth.generate_config(3, n_collisions=4)
    ores, mres = oracle.track_merge_event(ev)
    gtr, gch = _run(G, ev)
    assert mres.n_chains > 100
    _compare(ev, ores, mres, gtr, gch)


def test_merge_single_sector_has_no_chains(G):
    ev = synth.generate_config(0)
    gtr, gch = _run(G, ev)
    assert gch["n_chains"] == 0 and np.all(gch["link_out"] == -1)
