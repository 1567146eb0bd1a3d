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
    assert int(d["status"].item()) == 0
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


def _decode(trk, data, toff, roff, nt, ni, cap, n_bytes=None):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = trk.tm_decode(t(np.asarray(data, np.uint8)), t(np.asarray(toff, np.int64)), nt,
                      t(np.asarray(roff, np.int64)), ni, cap, n_bytes=n_bytes)
    torch.cuda.synchronize()
    return int(d["status"].item()), int(d["n"].item())


def test_decoder_rejects_malformed_streams(G):
    """The decoder takes caller data: every malformed item is reported by a
    status bit, and no read leaves the stream or its item (the kernel's own
    bounds checks, on inputs built here on the CPU)."""
    from paper_2502_09138_gb300.binding import TPCT_TD_BAD_STREAM, TPCT_TD_CAPACITY
    from synth.geometry import row_radii
    fx, ev, off, ncl, ids = _fixture_event()
    ref = oracle.tm_encode(ev, off, ncl, ids)
    nt, ni = int(ncl.shape[0]), ev.n_instances
    trk = G.Tracker(precision="mixed", bz=ev.bz)
    assert _decode(trk, ref.data, ref.track_off, ref.row_off, nt, ni, ev.n) == (0, ev.n)
    # output capacity too small: the count is reported, the bit set
    assert _decode(trk, ref.data, ref.track_off, ref.row_off, nt, ni, 1) == (TPCT_TD_CAPACITY, ev.n)
    # truncated stream (the last bytes missing, or none at all)
    st, _ = _decode(trk, ref.data, ref.track_off, ref.row_off, nt, ni, ev.n, n_bytes=ref.nbytes - 3)
    assert st & TPCT_TD_BAD_STREAM
    st, _ = _decode(trk, ref.data, ref.track_off, ref.row_off, nt, ni, ev.n, n_bytes=0)
    assert st & TPCT_TD_BAD_STREAM
    # an item offset beyond the stream, and offsets running backwards
    toff = np.array(ref.track_off, np.int64)
    toff[0] = ref.nbytes + 100
    st, _ = _decode(trk, ref.data, toff, ref.row_off, nt, ni, ev.n)
    assert st & TPCT_TD_BAD_STREAM
    toff = np.array(ref.track_off, np.int64)
    toff[1] = toff[0] - 1
    st, _ = _decode(trk, ref.data, toff, ref.row_off, nt, ni, ev.n)
    assert st & TPCT_TD_BAD_STREAM
    # a varint of 11 bytes, and a count larger than its item's bytes allow
    nb0 = ni * 152
    for data in ([0x80] * 11 + [0], [0xE8, 0x07]):   # continuation bytes only; the count 1000
        st, n = _decode(trk, data, [0, len(data)], [len(data)] * (nb0 + 1), 1, ni, 16)
        assert st == TPCT_TD_BAD_STREAM and n == 0
    # rows outside the geometry: the same stream decoded with a 12-row geometry
    # (the track's third cluster lies on row 12)
    few = G.Tracker(row_x=row_radii()[:12], precision="mixed", bz=ev.bz)
    assert int(ev.row[ids].max()) >= 12
    st, _ = _decode(few, ref.data, ref.track_off, ref.row_off, nt, ni, ev.n)
    assert st & TPCT_TD_BAD_STREAM
