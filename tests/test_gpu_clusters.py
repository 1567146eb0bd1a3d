"""Cluster finding on the GPU against the oracle, through the C ABI: integer
results (cluster count and order, total and peak charge, row, flags,
instance offsets) exactly; positions and widths within float rounding."""
import numpy as np
import pytest

import oracle
import synth.digits as D
from test_oracle_clusters import _fixture_digits, _params

pytestmark = pytest.mark.gpu

# the GPU forms the means in float from the same integer sums
RTOL_POS, ATOL_POS, ATOL_SIGMA = 2e-6, 2e-5, 2e-5


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_09138_gb300.build as b
    b.build()
    import paper_2502_09138_gb300 as G
    return G


def _run(G, dg, params=None, capacity=None):
    import torch
    trk = G.Tracker(precision="mixed")
    dd = G.DeviceDigits.from_digits(dg)
    prm = G.default_cf_params() if params is None else G.default_cf_params(
        q_peak_min=params.q_peak_min, valley_delta=params.valley_delta)
    out = trk.find_clusters(dd, prm, capacity=capacity)
    torch.cuda.synchronize()
    return out.to_host()


def _compare(dg, g, o):
    assert g["status"] == 0, g["status"]
    assert g["n_clusters"] == o.n
    for f in ("q_tot", "q_max", "row", "flags"):
        assert np.array_equal(g[f].astype(np.int64), getattr(o, f).astype(np.int64)), f
    offs = np.searchsorted(o.instance, np.arange(dg.n_instances + 1))
    assert np.array_equal(g["inst_offsets"], offs)
    for f in ("pad", "time", "x", "y", "z"):
        ref = getattr(o, f)
        assert np.all(np.abs(g[f] - ref) <= ATOL_POS + RTOL_POS * np.abs(ref)), (f, np.max(np.abs(g[f] - ref)))
    for f in ("sigma_pad", "sigma_time"):
        assert np.max(np.abs(g[f] - getattr(o, f))) <= ATOL_SIGMA, f


def test_hand_fixture(G):
    fx, dg = _fixture_digits()
    prm = _params(fx)
    _compare(dg, _run(G, dg, prm), oracle.find_clusters(dg, prm))


@pytest.fixture(scope="module")
def sector_digits():
    return D.generate_digits(0)


def test_single_sector(G, sector_digits):
    g = _run(G, sector_digits)
    _compare(sector_digits, g, oracle.find_clusters(sector_digits))


def test_central_event(G):
    dg = D.generate_digits(1, workers=8)
    o = oracle.find_clusters(dg)
    assert o.n > 1_000_000
    _compare(dg, _run(G, dg), o)


def test_repeatable_and_row_order_invariant(G, sector_digits):
    dg = sector_digits
    a, b = _run(G, dg), _run(G, dg)
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    rng = np.random.default_rng(9)
    perm = np.arange(dg.n)
    for k in range(dg.row_offsets.shape[0] - 1):
        lo, hi = dg.row_offsets[k], dg.row_offsets[k + 1]
        perm[lo:hi] = lo + rng.permutation(hi - lo)
    dg2 = D.Digits(pad=dg.pad[perm], time=dg.time[perm], adc=dg.adc[perm], row_offsets=dg.row_offsets,
                   sectors=dg.sectors, readout=dg.readout, n_pad=dg.n_pad, truth=dg.truth)
    c = _run(G, dg2)
    for k in a:   # the output order is (instance, row, peak time, peak pad)
        assert np.array_equal(np.asarray(a[k]), np.asarray(c[k])), k


def test_empty_and_single_digit_rows(G):
    n_inst = 2
    offs = np.zeros(n_inst * 152 + 1, np.int64)
    empty = D.Digits(pad=np.zeros(0, np.uint16), time=np.zeros(0, np.uint16), adc=np.zeros(0, np.uint16),
                     row_offsets=offs, sectors=np.array([3, 30]), readout=D.Readout(), n_pad=None, truth={})
    g = _run(G, empty)
    assert g["n_clusters"] == 0 and g["status"] == 0 and np.all(g["inst_offsets"] == 0)
    # one digit in the last row of the second instance, one in the first row of the first
    offs1 = np.zeros(n_inst * 152 + 1, np.int64)
    offs1[1:] = 1
    offs1[-1] = 2
    one = D.Digits(pad=np.array([5, 100], np.uint16), time=np.array([499, 0], np.uint16),
                   adc=np.array([9, 1023], np.uint16), row_offsets=offs1, sectors=np.array([3, 30]),
                   readout=D.Readout(), n_pad=None, truth={})
    g = _run(G, one)
    _compare(one, g, oracle.find_clusters(one))
    assert g["n_clusters"] == 2 and list(g["flags"]) == [2, 2]


def test_bad_digits_and_capacity_are_reported(G, sector_digits):
    dg = sector_digits
    o = oracle.find_clusters(dg)
    g = _run(G, dg, capacity=100)
    assert g["status"] == 8 and g["n_clusters"] == o.n            # TPCT_CF_CAPACITY, needed size written
    g = _run(G, dg, capacity=int(g["n_clusters"]))                # exactly the size needed: complete
    _compare(dg, g, o)
    bad = D.Digits(pad=dg.pad.copy(), time=dg.time.copy(), adc=dg.adc.copy(), row_offsets=dg.row_offsets,
                   sectors=dg.sectors, readout=dg.readout, n_pad=dg.n_pad, truth={})
    bad.pad[0] = 250                                              # beyond every row's pads
    g = _run(G, bad)
    assert g["status"] & 1                                        # TPCT_CF_BAD_DIGIT


def test_workspace_sized_for_fewer_digits_skips_rows(G, sector_digits):
    """A workspace sized for fewer digits than the rows hold: the rows that end
    beyond it are skipped and TPCT_CF_WORKSPACE is raised; the rows before
    them give the oracle's clusters."""
    import ctypes
    import torch
    import paper_2502_09138_gb300.binding as B
    dg = sector_digits
    o = oracle.find_clusters(dg)
    trk = G.Tracker(precision="mixed")
    dd = G.DeviceDigits.from_digits(dg)
    out = G.ClusterOut(o.n + 1024, dg.n_instances, trk.device)
    lib = B.load()
    half = int(dg.row_offsets[dg.row_offsets.shape[0] // 2])          # digits of the first half of the rows
    nb = int(lib.tpct_cf_workspace_bytes(half, dg.n_instances, trk.n_rows, out.capacity))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=trk.device)
    base = (ws.data_ptr() + 255) // 256 * 256
    prm = G.default_cf_params()
    ds, os_ = dd.as_struct(), out.as_struct()
    B.check(lib.tpct_find_clusters(trk._h, ctypes.byref(ds), ctypes.byref(prm), ctypes.c_void_p(base), nb,
                                   ctypes.byref(os_), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
            "tpct_find_clusters", trk._h)
    torch.cuda.synchronize()
    g = out.to_host()
    assert g["status"] == B.TPCT_CF_WORKSPACE
    # every row that ends within the requested digits is complete; rows that
    # end beyond them by more than the 256-byte rounding of the area are absent
    ends = dg.row_offsets[1:]
    rows_ok = np.nonzero(ends <= half)[0]
    rows_out = np.nonzero(ends > half + 64)[0]
    ir_o = o.instance.astype(np.int64) * trk.n_rows + o.row
    ir_g = np.repeat(np.arange(dg.n_instances), np.diff(g["inst_offsets"])) * trk.n_rows + g["row"].astype(np.int64)
    keep, sel = np.isin(ir_o, rows_ok), np.isin(ir_g, rows_ok)
    assert sel.sum() == keep.sum() > 0
    assert np.array_equal(g["q_tot"][sel].astype(np.int64), o.q_tot[keep].astype(np.int64))
    assert not np.isin(ir_g, rows_out).any()
