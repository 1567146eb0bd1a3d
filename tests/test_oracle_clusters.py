"""Pins of the oracle's cluster finding: a hand-built fixture whose expected
clusters were worked out by hand from the readings (peak and plateau order,
valley test, outer-ring rule, centroid and width, edge flags, sign of z);
generator truth of isolated crossings (one cluster each, centroid residuals,
collected charge); translation in time and the input order inside a row."""
import json
import os

import numpy as np
import pytest

import oracle
import synth.digits as D

HERE = os.path.dirname(os.path.abspath(__file__))
N_ROWS = 152


def _fixture_digits(shift_t=0):
    fx = json.load(open(os.path.join(HERE, "golden", "cf_hand_fixture.json")))
    n_inst = len(fx["instances"])
    per = {}
    for g in fx["digits"]:
        per.setdefault((g["inst"], g["row"]), []).extend(g["cells"])
    pad, tim, adc, counts = [], [], [], np.zeros(n_inst * N_ROWS, np.int64)
    for k in range(n_inst * N_ROWS):
        cells = per.get((k // N_ROWS, k % N_ROWS), [])
        for p, t, q in cells:
            pad.append(p); tim.append(t + shift_t); adc.append(q)
        counts[k] = len(cells)
    offs = np.zeros(n_inst * N_ROWS + 1, np.int64)
    offs[1:] = np.cumsum(counts)
    dg = D.Digits(pad=np.array(pad, np.uint16), time=np.array(tim, np.uint16), adc=np.array(adc, np.uint16),
                  row_offsets=offs, sectors=np.array([i["sector"] for i in fx["instances"]], np.int64),
                  readout=D.Readout(), n_pad=None, truth={})
    return fx, dg


def _params(fx):
    return oracle.CfParams(q_peak_min=fx["params"]["q_peak_min"], valley_delta=fx["params"]["valley_delta"])


def test_hand_fixture():
    fx, dg = _fixture_digits()
    res = oracle.find_clusters(dg, _params(fx))
    exp = [e for e in fx["expected"] if not e.get("none")]
    assert res.n == len(exp)
    for k, e in enumerate(exp):
        assert res.instance[k] == e["inst"] and res.row[k] == e["row"], (k, e)
        assert (dg.pad[res.peak[k]], dg.time[res.peak[k]]) == tuple(e["peak_cell"]), (k, e)
        assert res.q_tot[k] == e["q_tot"] and res.q_max[k] == e["q_max"] and res.flags[k] == e["flags"], (k, e)
        for f in ("pad", "time", "sigma_pad", "sigma_time", "y", "z"):
            assert abs(getattr(res, f)[k] - e[f]) <= 1e-12 * max(1.0, abs(e[f])), (k, f, getattr(res, f)[k], e[f])


def test_translation_in_time():
    fx, dg = _fixture_digits()
    _, dg13 = _fixture_digits(shift_t=13)
    a = oracle.find_clusters(dg, _params(fx))
    b = oracle.find_clusters(dg13, _params(fx))
    assert a.n == b.n
    for f in ("q_tot", "q_max", "row", "instance", "pad", "sigma_pad", "sigma_time", "y"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert np.allclose(b.time, a.time + 13, rtol=0, atol=1e-9)
    side = np.where(dg.sectors[a.instance] >= 18, -1.0, 1.0)
    assert np.allclose(b.z, a.z - side * 13 * 0.5, rtol=0, atol=1e-9)
    # the time-edge flag moves with the pattern (the corner cluster leaves t = 0)
    assert np.array_equal(b.flags, a.flags & ~np.where(a.time < 1.0, 2, 0).astype(np.uint8))


@pytest.fixture(scope="module")
def sector_digits():
    return D.generate_digits(0)


def test_input_order_inside_a_row(sector_digits):
    dg = sector_digits
    res = oracle.find_clusters(dg)
    rng = np.random.default_rng(5)
    perm = np.arange(dg.n)
    for k in range(dg.row_offsets.shape[0] - 1):
        a, b = dg.row_offsets[k], dg.row_offsets[k + 1]
        perm[a:b] = a + rng.permutation(b - a)
    dg2 = D.Digits(pad=dg.pad[perm], time=dg.time[perm], adc=dg.adc[perm], row_offsets=dg.row_offsets,
                   sectors=dg.sectors, readout=dg.readout, n_pad=dg.n_pad, truth=dg.truth)
    res2 = oracle.find_clusters(dg2)
    # the output order is (instance, row, peak time, peak pad): independent of the input order
    for f in ("q_tot", "q_max", "pad", "time", "y", "z", "sigma_pad", "flags", "row", "instance"):
        assert np.array_equal(getattr(res, f), getattr(res2, f)), f
    key = np.lexsort((dg.pad[res.peak], dg.time[res.peak], res.row, res.instance))
    assert np.array_equal(key, np.arange(res.n))


def test_isolated_crossings_against_truth(sector_digits):
    dg = sector_digits
    res = oracle.find_clusters(dg)
    tr = dg.truth
    rows, u, v = tr["row"], tr["u"], tr["v"]
    # isolated: no other crossing within 4 pads and 4 time bins in the same row
    iso = np.ones(u.shape[0], bool)
    order = np.lexsort((u, rows))
    for a in range(order.shape[0]):
        i = order[a]
        for b in range(a + 1, order.shape[0]):
            j = order[b]
            if rows[j] != rows[i] or u[j] - u[i] > 4:
                break
            if abs(v[j] - v[i]) <= 4:
                iso[i] = iso[j] = False
    iso &= (u > 3) & (u < dg.n_pad[rows] - 4) & (v > 3) & (v < 496)
    assert iso.sum() > 5000
    found, dpad, dtim, ratio = 0, [], [], []
    for i in np.nonzero(iso)[0]:
        sel = np.nonzero((res.row == rows[i]) & (np.abs(res.pad - u[i]) < 1.5) & (np.abs(res.time - v[i]) < 1.5))[0]
        if sel.shape[0] == 1:
            found += 1
            k = sel[0]
            dpad.append(res.pad[k] - u[i]); dtim.append(res.time[k] - v[i])
            ratio.append(res.q_tot[k] / tr["amp"][i])
    eff = found / iso.sum()
    assert eff > 0.995, eff
    dpad, dtim, ratio = np.array(dpad), np.array(dtim), np.array(ratio)
    # the charge-weighted centroid of a Gaussian sampled on unit cells recovers
    # its centre to a small fraction of a cell (noise 1 ADC, rounding)
    assert abs(dpad.mean()) < 0.01 and abs(dtim.mean()) < 0.01, (dpad.mean(), dtim.mean())
    assert dpad.std() < 0.1 and dtim.std() < 0.1, (dpad.std(), dtim.std())
    # the 5x5 window with the outer-ring rule and zero suppression collects
    # almost all of the deposited charge
    assert 0.9 < np.median(ratio) <= 1.01, np.median(ratio)


def test_rejects_duplicates_and_out_of_range():
    fx, dg = _fixture_digits()
    bad = D.Digits(pad=dg.pad.copy(), time=dg.time.copy(), adc=dg.adc.copy(), row_offsets=dg.row_offsets,
                   sectors=dg.sectors, readout=dg.readout, n_pad=None, truth={})
    bad.time[1] = bad.time[0]; bad.pad[1] = bad.pad[0]
    with pytest.raises(ValueError):
        oracle.find_clusters(bad, _params(fx))
    bad2 = D.Digits(pad=dg.pad.copy(), time=dg.time.copy(), adc=dg.adc.copy(), row_offsets=dg.row_offsets,
                    sectors=dg.sectors, readout=dg.readout, n_pad=None, truth={})
    bad2.pad[0] = 200
    with pytest.raises(ValueError):
        oracle.find_clusters(bad2, _params(fx))
