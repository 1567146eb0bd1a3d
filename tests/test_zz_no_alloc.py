"""The allocation-free entry point tpct_track_static, called through the C ABI.

Some callers cannot allocate device memory (a plug-in handed only its input
and output buffers, a process with all device memory planned at start-up, a
latency-critical path where cudaMalloc would synchronise the device), so they
cannot attach a workspace.  tpct_track_static runs the same tracking chain
with its scratch in a fixed array inside the library.  This test checks that
two calls in a row give what the workspace entry point tpct_track gives on the
same inputs, and that a request beyond the array's limit is refused.  It lives
in its own file, collected last, and builds everything it needs itself."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX_CLUSTERS = 65536


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_09138_gb300.build as b
    b.build()
    import paper_2502_09138_gb300 as G
    return torch, G


def _largest_central_sector():
    ev = synth.generate_config(1)
    sizes = np.diff(ev.sector_offsets)
    i = int(np.argmax(sizes))
    return ev.select_instances([i])


def _check_same(a, b):
    # same kernels on the same inputs: integer results identical, floats within
    # the parity tolerances (1e-4 relative for parameters, 1e-3 for covariances)
    assert a["n_tracks"] == b["n_tracks"] and a["n_ids"] == b["n_ids"]
    for k in ("instance", "n_cl", "offset", "ndf", "status", "cluster_ids"):
        assert np.array_equal(a[k], b[k]), k
    assert np.allclose(a["param"], b["param"], rtol=1e-4, atol=1e-12)
    assert np.allclose(a["cov"], b["cov"], rtol=1e-3, atol=1e-15)
    assert np.allclose(a["chi2"], b["chi2"], rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("which", ["single_sector", "largest_central_sector"])
def test_static_matches_workspace_entry_twice(env, which):
    torch, G = env
    ev = synth.generate_config(0) if which == "single_sector" else _largest_central_sector()
    assert ev.n <= MAX_CLUSTERS and ev.n_instances == 1
    trk = G.Tracker(precision="mixed", bz=ev.bz,
                    cuts=G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode))
    dc = G.DeviceClusters.from_event(ev)
    ref = trk.track(dc).to_host()
    torch.cuda.synchronize()
    assert ref["n_tracks"] > 0
    lib = G.B.load()
    stream = torch.cuda.current_stream()
    outs = [trk.make_output(ev.n) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs:
        cs, os_ = dc.as_struct(), out.as_struct()
        rc = lib.tpct_track_static(trk._h, ctypes.byref(cs), ev.n, ctypes.byref(os_),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == G.B.TPCT_OK, lib.tpct_last_cuda_error(trk._h)
        torch.cuda.synchronize()
    # the two calls took no device memory (the device's free memory is unchanged)
    assert torch.cuda.mem_get_info()[0] == free0
    for out in outs:
        _check_same(out.to_host(), ref)


def test_static_rejects_oversize(env):
    torch, G = env
    trk = G.Tracker(precision="mixed")
    n = MAX_CLUSTERS + 1
    f = torch.zeros(n, dtype=torch.float32, device="cuda")
    row = torch.zeros(n, dtype=torch.uint8, device="cuda")
    offs = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    dc = G.DeviceClusters(f, f, f, None, row, offs)
    out = trk.make_output(16, 16, 16)
    cs, os_ = dc.as_struct(), out.as_struct()
    rc = G.B.load().tpct_track_static(trk._h, ctypes.byref(cs), n, ctypes.byref(os_), None)
    assert rc == G.B.TPCT_E_NOMEM
    # two instances are refused as well
    offs2 = torch.tensor([0, 5, 10], dtype=torch.int64, device="cuda")
    dc2 = G.DeviceClusters(f[:10], f[:10], f[:10], None, row[:10], offs2)
    cs2 = dc2.as_struct()
    assert G.B.load().tpct_track_static(trk._h, ctypes.byref(cs2), 10, ctypes.byref(os_), None) == G.B.TPCT_E_NOMEM
