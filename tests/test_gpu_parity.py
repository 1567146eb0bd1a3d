"""CUDA path against the oracle, element by element, through the C ABI."""
import json

import numpy as np
import pytest

import oracle
import synth
from oracle.check import compare
from gpu_util import run_gpu, slice_instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_09138_gb300.build as b
    b.build()


def _assert_pass(rep):
    if not rep["pass"]:
        pytest.fail("parity failed: " + json.dumps(rep, default=str))


@pytest.mark.parametrize("precision", ["mixed", "fp64", "mixed_df"])
def test_single_sector_parity(event0, oracle0, precision):
    gtr, gdbg, st, _ = run_gpu(event0, precision)
    assert st == 0
    rep = compare(event0, oracle0, gdbg, gtr)
    _assert_pass(rep)
    assert rep["nf_mismatch"] == 0 and rep["track_mismatch"] == 0


def test_single_sector_fp32_close(event0, oracle0):
    # all-FP32: integer decisions may drift further; efficiency and most tracks must agree
    gtr, gdbg, st, _ = run_gpu(event0, "fp32")
    rep = compare(event0, oracle0, gdbg, gtr, rtol_par=1e-2, rtol_cov=1e-1)
    assert st == 0
    assert abs(rep["eff_gpu"] - rep["eff_oracle"]) <= 0.005, rep
    assert rep["tracks_identical"] >= 0.98 * rep["tracks_oracle"], rep


@pytest.fixture(scope="module")
def oracle1(event1):
    return oracle.track_event(event1)


@pytest.mark.parametrize("precision", ["mixed", "fp64", "mixed_df"])
def test_central_event_parity(event1, oracle1, precision):
    gtr, gdbg, st, _ = run_gpu(event1, precision)
    assert st == 0
    rep = compare(event1, oracle1, gdbg, gtr)
    _assert_pass(rep)


def test_batched_equals_plain(event1):
    a, da, sa, trk = run_gpu(event1, "mixed")
    b, db, sb, _ = run_gpu(event1, "mixed", batched=True, tracker=trk)
    assert sa == 0 and sb == 0
    for k in ("cluster_ids", "n_cl", "instance", "param", "cov", "chi2"):
        assert np.array_equal(a[k], b[k]), k


def test_grid_invariance(event0):
    ref, _, _, _ = run_gpu(event0, "mixed")
    for cpb in (1, 5, 50, 100000):
        g, _, st, _ = run_gpu(event0, "mixed", tuning=dict(clusters_per_bin=cpb))
        assert st == 0
        for k in ("cluster_ids", "n_cl", "param", "cov", "chi2"):
            assert np.array_equal(ref[k], g[k]), (cpb, k)


def test_block_shape_invariance(event0):
    ref, _, _, _ = run_gpu(event0, "mixed")
    g, _, _, _ = run_gpu(event0, "mixed", tuning=dict(tracklet_block=32, refit_block=256))
    for k in ("cluster_ids", "param", "cov"):
        assert np.array_equal(ref[k], g[k]), k


def test_deterministic(event1):
    a, _, _, trk = run_gpu(event1, "mixed")
    b, _, _, _ = run_gpu(event1, "mixed", tracker=trk)
    for k in ("cluster_ids", "param", "cov", "chi2"):
        assert np.array_equal(a[k], b[k]), k


def test_row_from_x(event0):
    a, _, _, _ = run_gpu(event0, "mixed")
    b, _, _, _ = run_gpu(event0, "mixed", with_row=False)
    assert np.array_equal(a["cluster_ids"], b["cluster_ids"])
    assert np.array_equal(a["param"], b["param"])


def test_capacity_overflow_reports_sizes(event0, oracle0):
    gtr, _, st, _ = run_gpu(event0, "mixed", cap=(10, 100))
    assert st == 3   # TPCT_E_CAPACITY
    assert gtr["n_tracks"] == oracle0.n_tracks


def test_empty_and_sparse_instances():
    ev0 = synth.generate_config(0)
    empty = synth.Event(ev0.x[:0], ev0.y[:0], ev0.z[:0], ev0.charge[:0], ev0.row[:0],
                        np.zeros(3, np.int64), np.array([0, 1]), ev0.mc[:0], sectors_per_event=2)
    gtr, gdbg, st, _ = run_gpu(empty, "mixed")
    assert st == 0 and gtr["n_tracks"] == 0
    # an empty instance between two real ones
    ev = synth.concat_events([ev0, empty, ev0])
    gtr, gdbg, st, _ = run_gpu(ev, "mixed")
    ores = oracle.track_event(ev)
    assert st == 0
    _assert_pass(compare(ev, ores, gdbg, gtr))


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_batch_of_collisions_sampled_parity(precision):
    ev = synth.generate_config(3, n_collisions=12)
    gtr, gdbg, st, _ = run_gpu(ev, precision, batched=True)
    assert st == 0
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(ev.n_instances, 24, replace=False))
    sub = ev.select_instances(idx)
    ores = oracle.track_event(sub)
    tr, dbg = slice_instances(ev, gtr, gdbg, idx)
    _assert_pass(compare(sub, ores, dbg, tr))


def test_autotune_keeps_results_and_caches(event0, tmp_path):
    import paper_2502_09138_gb300 as G
    ref, _, _, trk = run_gpu(event0, "mixed")
    dc = G.DeviceClusters.from_event(event0)
    cache = str(tmp_path / "tuning.cache")
    t1 = trk.autotune(dc, cache_path=cache)
    assert t1["from_cache"] == 0 and t1["ms"] > 0
    assert t1["clusters_per_bin"] in (1, 2, 4, 8) and t1["tracklet_block"] in (64, 128, 256)
    got, _, st, _ = run_gpu(event0, "mixed", tracker=trk)
    assert st == 0
    for k in ("cluster_ids", "param", "cov", "chi2"):
        assert np.array_equal(ref[k], got[k]), k
    t2 = G.Tracker(precision="mixed", bz=event0.bz, cuts=trk.cuts).autotune(dc, cache_path=cache)
    assert t2["from_cache"] == 1
    assert (t2["clusters_per_bin"], t2["tracklet_block"], t2["refit_block"]) == \
        (t1["clusters_per_bin"], t1["tracklet_block"], t1["refit_block"])
