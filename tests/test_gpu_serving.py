"""Serving runtime (continuous batching under a device-memory budget),
through the C ABI: each frame's result is the same alone and in a mix whose
work overlaps on the device; admission waits for memory; oversize frames are
refused."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def collisions():
    return [synth.generate_config(3, instance=7, n_collisions=1, n_tracks=n) for n in (3000, 800, 5000, 1500)]


def _frame(G, ev):
    return G.Server.host_frame(ev.x, ev.y, ev.z, ev.charge, ev.row, ev.sector_offsets)


def _server(G, ev, **kw):
    return G.Server(bz=ev.bz, cuts=G.default_cuts(sig_readout=ev.sigma.at_readout,
                                                  sig_cathode=ev.sigma.at_cathode), **kw)


def test_alone_equals_in_mix(G, collisions):
    ev = collisions
    alone = {}
    srv = _server(G, ev[0], n_slots=1, budget_bytes=4 << 30)
    for i, e in enumerate(ev):
        tk = srv.submit(_frame(G, e))
        srv.wait(tk)
        alone[i] = srv.fetch(tk)
        srv.release(tk)
    srv.close()
    srv = _server(G, ev[0], n_slots=3, budget_bytes=8 << 30)
    tks = [srv.submit(_frame(G, e)) for e in ev * 2]
    for tk in tks:
        srv.wait(tk)
    st = srv.stats()
    assert st["peak_in_flight"] >= 2, st          # frames overlapped on the device
    for j, tk in enumerate(tks):
        got = srv.fetch(tk)
        ref = alone[j % len(ev)]
        assert got["n_tracks"] == ref["n_tracks"] > 0
        for k in ("instance", "n_cl", "offset", "cluster_ids", "param", "cov", "chi2"):
            assert np.array_equal(got[k], ref[k]), (j, k)
        srv.release(tk)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_admission_waits_for_memory(G, collisions):
    ev = collisions[2]
    per_frame = G.Tracker(device="cpu").workspace_bytes(ev.n, ev.n_instances)
    srv = _server(G, ev, n_slots=4, budget_bytes=int(per_frame * 1.8) + (64 << 20))
    tks = [srv.submit(_frame(G, ev)) for _ in range(4)]
    for tk in tks:
        srv.wait(tk)
    st = srv.stats()
    assert st["completed"] == 4 and st["peak_in_flight"] == 1, st   # one frame fits at a time
    assert st["peak_bytes"] <= st["budget_bytes"]
    first = srv.fetch(tks[0])
    for tk in tks[1:]:
        assert np.array_equal(srv.fetch(tk)["cluster_ids"], first["cluster_ids"])
    for tk in tks:
        srv.release(tk)
    srv.close()


def test_oversize_frame_refused(G, collisions):
    ev = collisions[0]
    srv = _server(G, ev, n_slots=1, budget_bytes=16 << 20)
    with pytest.raises(G.B.TpctError) as e:
        srv.submit(_frame(G, ev))
    assert e.value.code == G.B.TPCT_E_BUDGET
    srv.close()


def test_wait_times_out_on_the_host_then_completes(G, collisions):
    """tpct_server_wait gives up after its host timeout with TPCT_E_TIMEOUT
    while the frame is still queued or running (no kernel waits for anything:
    the timeout is the host's); a later wait returns the finished frame, equal
    to the frame tracked alone."""
    ev = collisions[2]
    srv = _server(G, ev, n_slots=1, budget_bytes=4 << 30)
    tk = srv.submit(_frame(G, ev))
    with pytest.raises(G.B.TpctError) as e:
        srv.wait(tk, timeout_s=1e-6)
    assert e.value.code == G.B.TPCT_E_TIMEOUT
    srv.wait(tk, timeout_s=600.0)
    got = srv.fetch(tk)
    srv.release(tk)
    tk2 = srv.submit(_frame(G, ev))
    srv.wait(tk2)
    ref = srv.fetch(tk2)
    srv.release(tk2)
    srv.close()
    assert got["n_tracks"] == ref["n_tracks"] > 0
    assert np.array_equal(got["cluster_ids"], ref["cluster_ids"])
