"""The C ABI library loads and exports every declared entry point; host-side
argument checks work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2502_09138_gb300.build as b
    b.build()
    import paper_2502_09138_gb300.binding as B
    return B.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tpct_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_create_and_workspace_without_gpu(lib):
    import paper_2502_09138_gb300 as G
    trk = G.Tracker(device="cpu")
    nb = trk.workspace_bytes(1_400_000, 36)
    assert 100e6 < nb < 2e9
    assert trk.workspace_bytes(0, 1) > 0
    assert trk.workspace_bytes(-1, 1) == 0


def test_invalid_arguments(lib):
    import paper_2502_09138_gb300 as G
    B = G.B
    c = G.default_cuts()
    rx = np.array([1.0, 2.0, 1.5])      # not ascending
    g = B.Geometry(3, rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.17, 250.0)
    h = ctypes.c_void_p()
    assert lib.tpct_create(ctypes.byref(g), 0.5, ctypes.byref(c), 1, ctypes.byref(h)) == B.TPCT_E_INVALID
    bad = G.default_cuts(s_max=1.5)
    rx = np.arange(10, dtype=np.float64) + 80
    g = B.Geometry(10, rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.17, 250.0)
    assert lib.tpct_create(ctypes.byref(g), 0.5, ctypes.byref(bad), 1, ctypes.byref(h)) == B.TPCT_E_INVALID
    assert lib.tpct_create(ctypes.byref(g), 0.5, ctypes.byref(c), 7, ctypes.byref(h)) == B.TPCT_E_INVALID
    assert lib.tpct_create(ctypes.byref(g), 0.5, ctypes.byref(c), 1, ctypes.byref(h)) == B.TPCT_OK
    # tracking without a workspace is a state error, detected on the host
    cl = B.Clusters()
    cl.n_instances = 1
    out = B.TracksOut()
    assert lib.tpct_track(h, ctypes.byref(cl), 10, ctypes.byref(out), None) == B.TPCT_E_STATE
    assert lib.tpct_set_tuning(h, 0, 33, 0) == B.TPCT_E_INVALID
    lib.tpct_destroy(h)
    assert lib.tpct_status_str(B.TPCT_E_CAPACITY) == b"output capacity exceeded"


def test_static_scratch_fits_one_sector(lib):
    # tpct_track_static carries a 24 MiB scratch array sized for one sector
    # instance of 65536 clusters at 152 rows; the workspace plan must fit it
    import paper_2502_09138_gb300 as G
    assert G.Tracker(device="cpu").workspace_bytes(65536, 1) <= 24 << 20


def test_auxiliary_workspace_sizes_without_gpu(lib):
    """Host-only size queries of cluster finding and track-model coding: zero
    for invalid arguments, growing with the digits / clusters and the output
    capacity."""
    cf = lib.tpct_cf_workspace_bytes
    a = cf(1_000_000, 36, 152, 100_000)
    assert a > 4 * 1_000_000 and cf(2_000_000, 36, 152, 100_000) > a and cf(1_000_000, 36, 152, 200_000) > a
    assert cf(-1, 36, 152, 10) == 0 and cf(10, -1, 152, 10) == 0 and cf(10, 36, 0, 10) == 0 and cf(10, 36, 152, -1) == 0
    assert cf(0, 0, 152, 0) > 0
    tm = lib.tpct_tm_encode_workspace_bytes
    b = tm(1_000_000, 20_000, 36, 152)
    assert b > 16 * 1_000_000 and tm(2_000_000, 20_000, 36, 152) > b
    assert tm(-1, 1, 1, 152) == 0 and tm(1, -1, 1, 152) == 0


def test_default_geometry_is_the_tpc_readout(lib):
    """The library's built-in geometry equals the synthetic events' readout
    (152 rows in three pitch regions, tan 10 deg, 250 cm)."""
    import paper_2502_09138_gb300 as G
    import synth
    rx, tan_half, z_max = G.default_geometry()
    g = synth.default_geometry()
    assert np.array_equal(rx, g.row_x)
    assert tan_half == g.tan_half_sector and z_max == g.z_max
    assert rx.shape == (152,) and rx[0] == 85.2 and rx[63] == 135.1 and rx[127] == 199.4


def test_package_does_not_import_test_data():
    """The library package takes its default geometry from the library, not
    from the synthetic-event package."""
    import subprocess
    import sys
    code = ("import sys, paper_2502_09138_gb300 as G; G.Tracker(device='cpu'); "
            "sys.exit(1 if 'synth' in sys.modules else 0)")
    assert subprocess.run([sys.executable, "-c", code], cwd=ROOT).returncode == 0


def test_tracking_only_clusters_need_the_row():
    import paper_2502_09138_gb300 as G
    with pytest.raises(ValueError):
        G.DeviceClusters.from_event(None, device="cpu", with_row=False, tracking_only=True)
