"""The hand-worked tracklet-growth fixture (tests/golden/tracklet_hand_fixture.json)
through the CUDA library: links, start hits, the row-indexed hit list of every
tracklet and the selected tracks must equal the hand-worked values element by
element, in the plain and the graph-captured form and in every precision that
meets the parity bar (the fixture's decisions are all far from their cuts,
except two exact search ties that both sides break by the smaller id)."""
import numpy as np
import pytest

from test_oracle_tracklets import fixture_arrays, load_fixture

pytestmark = pytest.mark.gpu


def _run(fx, precision, batched):
    import torch
    import paper_2502_09138_gb300 as G
    offs, y, z, row = fixture_arrays(fx)
    g = fx["geometry"]
    rx = np.array(g["row_x"])
    trk = G.Tracker(row_x=rx, tan_half_sector=g["tan_half_sector"], z_max=g["z_max"], bz=0.5,
                    cuts=G.default_cuts(**fx["cuts"]), precision=precision)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dc = G.DeviceClusters(t(rx[row].astype(np.float32)), t(y), t(z), t(np.ones(y.shape, np.uint16)),
                          t(row.astype(np.uint8)), t(offs))
    out = trk.make_output(dc.n)
    trk.track(dc, out, batched=batched)
    if batched:                      # second replay of the captured graph
        trk.track(dc, out, batched=True)
    dbg = trk.debug(dc.n)
    torch.cuda.synchronize()
    assert trk.device_status() == 0
    return out.to_host(), dbg.to_host(), offs


@pytest.mark.parametrize("precision", ["mixed", "mixed_df", "fp64"])
@pytest.mark.parametrize("batched", [False, True])
def test_tracklet_fixture_on_gpu(precision, batched):
    fx = load_fixture()
    tr, dbg, offs = _run(fx, precision, batched)
    n_rows = len(fx["geometry"]["row_x"])
    inst_of = np.searchsorted(offs, np.arange(offs[-1]), side="right") - 1
    tl_inst = inst_of[dbg["tl_start"]]
    bad = []
    for i, inst in enumerate(fx["instances"]):
        base = int(offs[i])
        loc = lambda a: int(a) - base if a >= 0 else -1
        for k, want in inst.get("links", {}).items():
            c = base + int(k)
            got = [loc(dbg["up"][c]), loc(dbg["down"][c]), loc(dbg["upc"][c]), loc(dbg["downc"][c])]
            if got != want:
                bad.append((inst["name"], "links", k, got, want))
        tl = np.nonzero(tl_inst == i)[0]
        starts = [loc(dbg["tl_start"][t]) for t in tl]
        if starts != inst["starts"]:
            bad.append((inst["name"], "starts", starts, inst["starts"]))
            continue
        for t, want in zip(tl, inst["tracklets"]):
            hits = [loc(dbg["tl_hits"][t, r]) for r in range(n_rows) if dbg["tl_hits"][t, r] >= 0]
            if hits != want["hits"]:
                bad.append((inst["name"], "hits of tracklet", want["start"], hits, want["hits"]))
        tracks = []
        for k in range(int(tr["n_tracks"])):
            if int(tr["instance"][k]) == i:
                a = int(tr["offset"][k])
                tracks.append([loc(c) for c in tr["cluster_ids"][a:a + int(tr["n_cl"][k])]])
        if tracks != inst["tracks"]:
            bad.append((inst["name"], "tracks", tracks, inst["tracks"]))
    assert bad == []
