"""Pins of the oracle's Kalman update and refit: the information form of the
Bayesian update, noiseless helices refit to generator truth within 1e-9,
chi2/ndf near 1 and unit pulls on Gaussian-smeared tracks."""
import numpy as np
import pytest

import oracle
import synth
from synth.events import truth_state


def test_update_equals_information_form():
    r = np.random.default_rng(11)
    H = np.zeros((2, 5))
    H[0, 0] = H[1, 1] = 1.0
    for _ in range(100):
        A = r.normal(size=(5, 5))
        C = A @ A.T + 0.1 * np.eye(5)
        p = r.normal(size=5)
        m = r.normal(size=2)
        vy, vz = r.uniform(0.005, 0.05, 2)
        V = np.diag([vy, vz])
        chi2, p1, C1 = oracle.kf_update(p, C.ravel(), m[0], m[1], vy, vz)
        Ci = np.linalg.inv(C)
        Cpost = np.linalg.inv(Ci + H.T @ np.linalg.inv(V) @ H)
        ppost = Cpost @ (Ci @ p + H.T @ np.linalg.inv(V) @ m)
        res = m - p[:2]
        S = C[:2, :2] + V
        assert np.allclose(C1.reshape(5, 5), Cpost, rtol=1e-9, atol=1e-12)
        assert np.allclose(p1, ppost, rtol=1e-9, atol=1e-12)
        assert chi2 == pytest.approx(res @ np.linalg.solve(S, res), rel=1e-10)


def _max_rel_err_vs_truth(ev, res):
    worst = np.zeros(5)
    for k in range(res.n_tracks):
        ids = res.track_ids(k)
        m = int(np.bincount(ev.mc[ids][ev.mc[ids] >= 0]).argmax())
        sec = int(ev.sectors[res.tr_inst[k]])
        ts, ok = truth_state(ev, m, sec, res.tr_x_ref[k])
        assert ok
        worst = np.maximum(worst, np.abs(res.tr_param[k] - ts) / np.abs(ts))
    return worst


def test_noiseless_single_sector_refit_to_truth():
    ev = synth.generate_config(0, smear=False, keep_exact=True)
    res = oracle.track_event(ev, exact=True)
    assert res.n_tracks > 100 and np.all(res.tr_status == 0)
    worst = _max_rel_err_vs_truth(ev, res)
    assert np.all(worst < 1e-9), worst


def test_noiseless_full_tpc_refit_to_truth():
    ev = synth.generate_event(synth.seed_for(1, 77), n_tracks=300, efficiency=1.0, noise_fraction=0.0,
                              smear=False, keep_exact=True)
    res = oracle.track_event(ev, exact=True)
    ok = res.tr_status == 0
    assert res.n_tracks > 200 and ok.mean() > 0.99
    # only clean tracks (all clusters from one particle) have an exact truth
    worst = np.zeros(5)
    for k in np.nonzero(ok)[0]:
        ids = res.track_ids(k)
        if len(np.unique(ev.mc[ids])) != 1:
            continue
        ts, _ = truth_state(ev, int(ev.mc[ids[0]]), int(ev.sectors[res.tr_inst[k]]), res.tr_x_ref[k])
        worst = np.maximum(worst, np.abs(res.tr_param[k] - ts) / np.abs(ts))
    assert np.all(worst < 1e-9), worst


def test_chi2_per_ndf_single_sector(oracle0):
    s = oracle0.tr_chi2.sum() / oracle0.tr_ndf.sum()
    assert abs(s - 1.0) < 3.0 * np.sqrt(2.0 / oracle0.tr_ndf.sum()), s


def test_pulls_and_chi2_clean_events():
    ev = synth.generate_config(1, n_tracks=1500, noise_fraction=0.0)
    res = oracle.track_event(ev)
    s = res.tr_chi2.sum() / res.tr_ndf.sum()
    assert abs(s - 1.0) < 3.0 * np.sqrt(2.0 / res.tr_ndf.sum()), s
    pulls = []
    for k in range(res.n_tracks):
        ids = res.track_ids(k)
        if len(np.unique(ev.mc[ids])) != 1 or res.tr_status[k]:
            continue
        ts, ok = truth_state(ev, int(ev.mc[ids[0]]), int(ev.sectors[res.tr_inst[k]]), res.tr_x_ref[k])
        # truth at the row is unsmeared; the pull of y, z includes nothing else
        cov = res.tr_cov[k]
        diag = np.array([cov[0], cov[2], cov[5], cov[9], cov[14]])
        pulls.append((res.tr_param[k] - ts) / np.sqrt(diag))
    pulls = np.array(pulls)
    K = pulls.shape[0]
    assert K > 1500
    assert np.all(np.abs(pulls.mean(0)) < 3.0 / np.sqrt(K)), pulls.mean(0)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.05), pulls.std(0)


def test_sequential_scalar_updates_equal_the_oracle_update():
    """The tracking kernels update with two scalar measurements, y then z
    (the z residual taken after the y step), where the oracle takes the joint
    2-D update; for the diagonal cluster covariance the two are the same
    posterior and the same chi2 (sequential processing of independent
    measurements).  Written here in plain numpy against the oracle's update,
    including prior covariances far wider than the measurement."""
    r = np.random.default_rng(12)
    for trial in range(200):
        A = r.normal(size=(5, 5))
        scale = np.diag(10.0 ** r.uniform(-3, 3, 5))
        C = scale @ (A @ A.T + 0.1 * np.eye(5)) @ scale
        p = r.normal(size=5)
        m = p[:2] + r.normal(scale=0.1, size=2)
        v = r.uniform(0.005, 0.05)
        chi2, p1, C1 = oracle.kf_update(p, C.ravel(), m[0], m[1], v, v)
        ps, Cs, chi2s = p.copy(), C.copy(), 0.0
        for k in (0, 1):
            res = m[k] - ps[k]                    # residual after the previous scalar step
            S = Cs[k, k] + v
            K = Cs[:, k] / S
            chi2s += res * res / S
            ps = ps + K * res
            Cs = Cs - np.outer(K, Cs[k, :])
        assert np.allclose(Cs, C1.reshape(5, 5), rtol=1e-7, atol=1e-9 * np.abs(C).max())
        assert np.allclose(ps, p1, rtol=1e-9, atol=1e-9)
        assert chi2s == pytest.approx(chi2, rel=1e-9, abs=1e-12)
