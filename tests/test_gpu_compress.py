"""Track-model compression on the GPU through the C ABI: the encoded bytes
and block offsets identical to the oracle's, and the GPU decoding of them
identical to the oracle's decoding (the format is integer-exact)."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_compress import _fixture_event

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


def _tracks_from(G, off, ncl, ids, cap=None):
    import torch
    nt = int(ncl.shape[0])
    t = G.Tracks(cap or nt + 4, max(1, ids.shape[0]), "cuda")
    t.counts.copy_(torch.tensor([nt, ids.shape[0]], dtype=torch.int32))
    if nt:
        t.offset[:nt] = torch.from_numpy(np.ascontiguousarray(off, np.int32)).cuda()
        t.n_cl[:nt] = torch.from_numpy(np.ascontiguousarray(ncl, np.int32)).cuda()
        t.cluster_ids[:ids.shape[0]] = torch.from_numpy(np.ascontiguousarray(ids, np.int32)).cuda()
    return t


def _check(G, ev, off, ncl, ids, trk=None, tracks=None):
    import torch
    trk = trk or G.Tracker(precision="mixed", bz=ev.bz)
    dc = G.DeviceClusters.from_event(ev)
    tracks = tracks or _tracks_from(G, off, ncl, ids)
    st = trk.tm_encode(dc, tracks)
    torch.cuda.synchronize()
    ref = oracle.tm_encode(ev, off, ncl, ids)
    nb = int(st["n_bytes"].item())
    assert nb == ref.nbytes
    assert np.array_equal(st["data"][:nb].cpu().numpy(), ref.data)
    nt = int(ncl.shape[0])
    assert np.array_equal(st["track_offsets"][:nt + 1].cpu().numpy(), ref.track_off)
    assert np.array_equal(st["row_offsets"].cpu().numpy(), ref.row_off)
    d = trk.tm_decode(st["data"], st["track_offsets"], nt, st["row_offsets"], ev.n_instances, ev.n)
    torch.cuda.synchronize()
    od = oracle.tm_decode(ref, ev.n)
    assert int(d["n"].item()) == ev.n
    for k in ("x", "y", "z", "row"):
        assert np.array_equal(d[k][:ev.n].cpu().numpy(), od[k]), k
    assert np.array_equal(d["charge"][:ev.n].cpu().numpy().view(np.uint16), od["charge"])
    return st, ref


def test_hand_encoded_frame(G):
    fx, ev, off, ncl, ids = _fixture_event()
    _check(G, ev, off, ncl, ids)


def test_central_event_with_its_gpu_tracks(G):
    ev = synth.generate_config(1)
    res = oracle.track_event(ev)
    trk = G.Tracker(precision="mixed", bz=ev.bz,
                    cuts=G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode))
    dc = G.DeviceClusters.from_event(ev)
    tracks = trk.track(dc)
    gt = tracks.to_host()
    assert np.array_equal(gt["cluster_ids"], res.tr_ids)        # the tracks are the oracle's
    st, ref = _check(G, ev, res.tr_offset, res.tr_ncl, res.tr_ids, trk=trk, tracks=tracks)
    assert ref.nbytes < 7.0 * ev.n                               # raw: 14 B per cluster


def test_collision_batch(G):
    ev = synth.generate_config(3, n_collisions=4)
    res = oracle.track_event(ev)
    _check(G, ev, res.tr_offset, res.tr_ncl, res.tr_ids)


def test_no_tracks_and_capacity(G):
    import torch
    ev = synth.generate_config(0)
    _check(G, ev, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    # a stream larger than the buffer: the size is reported, nothing is written
    trk = G.Tracker(precision="mixed")
    dc = G.DeviceClusters.from_event(ev)
    tracks = _tracks_from(G, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    st = trk.tm_encode(dc, tracks, capacity_bytes=64)
    torch.cuda.synchronize()
    ref = oracle.tm_encode(ev, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert int(st["n_bytes"].item()) == ref.nbytes > 64
