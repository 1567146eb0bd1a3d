"""Parity checker: CUDA results against the oracle -- TEST INFRASTRUCTURE.

Integer results (links, start hits, tracklet cluster lists, weights, track
cluster lists) must be identical, except where a decision of the oracle lies
within ``tol`` (relative) of its cut or of the runner-up candidate: there the
FP32 arithmetic of the CUDA path may decide the other way.  Such mismatches
are excused and counted, together with everything downstream of them:
  links        mismatch at a hit whose oracle neighbour margin < tol
  clean/start  mismatches explained by a link mismatch at the hit or a partner
  tracklets    mismatch if the oracle's tracklet margin < tol or the tracklet
               holds a hit tainted above
  selection    weight mismatches only on clusters of mismatched tracklets; a
               track mismatch only if its tracklet is excused or holds a
               cluster of one
Anything else is an unexcused mismatch.  The bar is on links and track
lists: a tracklet-list difference outside the band (the FP32 extrapolation
of the mixed precisions can flip a later decision of a long tracklet) is
counted and passes only while it changes no output track and stays below
0.1 % of the tracklets.  Floating outputs of identical tracks:
|dp_i| <= rtol_par * max(|p_i|, sigma_i) with sigma_i from the oracle
covariance; |dC_ij| <= rtol_cov * sqrt(C_ii C_jj).  The plain element-wise
relative errors (parameters larger than their sigma, diagonal covariance
terms) are reported beside that bar.
"""
import numpy as np

from synth.truth import evaluate


def _key_tracks(ores):
    return {int(ores.tl_start[t]): k for k, t in enumerate(ores.tr_tracklet)}


def compare(ev, ores, gdbg, gtr, tol=1e-5, rtol_par=1e-4, rtol_cov=1e-3, eff_tol=0.005):
    rep = {}
    n = ev.n
    # ---------------------------------------------------------------- links
    nf_mis = (ores.up != gdbg["up"]) | (ores.down != gdbg["down"])
    nf_exc = nf_mis & (ores.nf_margin < tol)
    rep["nf_compared"] = n
    rep["nf_mismatch"] = int(nf_mis.sum())
    rep["nf_excused"] = int(nf_exc.sum())
    rep["nf_unexcused"] = int((nf_mis & ~nf_exc).sum())
    taint = np.zeros(n, bool)
    idx = np.nonzero(nf_mis)[0]
    taint[idx] = True
    for arr in (ores.up, ores.down, gdbg["up"], gdbg["down"]):
        t = arr[idx]
        taint[t[t >= 0]] = True
    c_mis = (ores.upc != gdbg["upc"]) | (ores.downc != gdbg["downc"])
    rep["clean_mismatch"] = int(c_mis.sum())
    rep["clean_unexcused"] = int((c_mis & ~taint).sum())
    idx = np.nonzero(c_mis)[0]
    taint2 = taint.copy()
    taint2[idx] = True
    for arr in (ores.upc, ores.downc, gdbg["upc"], gdbg["downc"]):
        t = arr[idx]
        taint2[t[t >= 0]] = True

    # ---------------------------------------------------------------- start hits / tracklets
    o_start = {int(s): t for t, s in enumerate(ores.tl_start)}
    g_start = {int(s): t for t, s in enumerate(gdbg["tl_start"])}
    only = set(o_start) ^ set(g_start)
    def start_tainted(h):
        if taint2[h]:
            return True
        for arr in (ores.upc, gdbg["upc"]):
            u = arr[h]
            if u >= 0 and taint2[u]:
                return True
        return False
    rep["start_only_one_side"] = len(only)
    rep["start_unexcused"] = sum(1 for h in only if not start_tainted(h))
    # A tracklet-list difference is excused by the near-cut rule (margin < tol
    # or downstream of an excused link / start hit).  One outside the band is
    # counted as unexcused; it fails the comparison only if it changes an
    # output track (the bar is on links and track lists; tracklets are
    # intermediate) or if such differences exceed 0.1 % of the tracklets.
    exc_tl_o = np.zeros(len(ores.tl_start), bool)
    exc_tl_g = np.zeros(len(gdbg["tl_start"]), bool)
    unexc_tl_o = np.zeros(len(ores.tl_start), bool)
    unexc_tl_g = np.zeros(len(gdbg["tl_start"]), bool)
    tl_mis = tl_unexc = 0
    cl_taint = np.zeros(n, bool)
    cl_taint_unexc = np.zeros(n, bool)
    gh, oh = gdbg["tl_hits"], ores.tl_hits
    for h, to in o_start.items():
        tg = g_start.get(h)
        if tg is None:
            exc_tl_o[to] = True
            cl_taint[oh[to][oh[to] >= 0]] = True
            continue
        if np.array_equal(oh[to], gh[tg]):
            continue
        tl_mis += 1
        hits = np.concatenate([oh[to][oh[to] >= 0], gh[tg][gh[tg] >= 0]])
        ok = ores.tl_margin[to] < tol or start_tainted(h) or taint2[hits].any()
        if ok:
            exc_tl_o[to] = exc_tl_g[tg] = True
            cl_taint[hits] = True
        else:
            tl_unexc += 1
            unexc_tl_o[to] = unexc_tl_g[tg] = True
            cl_taint_unexc[hits] = True
    for h, tg in g_start.items():
        if h not in o_start:
            exc_tl_g[tg] = True
            cl_taint[gh[tg][gh[tg] >= 0]] = True
    rep["tracklets_compared"] = len(set(o_start) & set(g_start))
    rep["tracklet_mismatch"] = tl_mis
    rep["tracklet_unexcused"] = tl_unexc

    # ---------------------------------------------------------------- weights
    w_mis = ores.weight != gdbg["weight"]
    rep["weight_mismatch"] = int(w_mis.sum())
    rep["weight_unexcused"] = int((w_mis & ~cl_taint & ~cl_taint_unexc).sum())

    # ---------------------------------------------------------------- tracks
    g_tr_key = {}
    for k in range(gtr["n_tracks"]):
        t = int(gdbg["tr_tracklet"][k])
        g_tr_key[int(gdbg["tl_start"][t])] = k
    o_tr_key = _key_tracks(ores)
    tr_mis = tr_unexc = tr_exc = 0
    same = []
    for h in set(o_tr_key) | set(g_tr_key):
        ko, kg = o_tr_key.get(h), g_tr_key.get(h)
        ids_o = ores.track_ids(ko) if ko is not None else np.zeros(0, np.int32)
        ids_g = (gtr["cluster_ids"][gtr["offset"][kg]:gtr["offset"][kg] + gtr["n_cl"][kg]]
                 if kg is not None else np.zeros(0, np.int32))
        if ko is not None and kg is not None and np.array_equal(ids_o, ids_g):
            same.append((ko, kg))
            continue
        tr_mis += 1
        to = o_start.get(h)
        tg = g_start.get(h)
        both = np.concatenate([ids_o, ids_g])
        excused = ((to is not None and exc_tl_o[to]) or (tg is not None and exc_tl_g[tg]) or
                   cl_taint[both].any())
        if to is not None and not excused:
            excused = excused or cl_taint[oh[to][oh[to] >= 0]].any()
        # a track changed by a tracklet difference outside the band is not excused
        if ((to is not None and unexc_tl_o[to]) or (tg is not None and unexc_tl_g[tg]) or
                cl_taint_unexc[both].any()):
            excused = False
        if excused:
            tr_exc += 1
        else:
            tr_unexc += 1
    rep["tracks_oracle"] = ores.n_tracks
    rep["tracks_gpu"] = int(gtr["n_tracks"])
    rep["track_mismatch"] = tr_mis
    rep["track_excused"] = tr_exc
    rep["track_unexcused"] = tr_unexc
    rep["tracks_identical"] = len(same)

    # ---------------------------------------------------------------- floating outputs
    if same:
        ko = np.array([a for a, _ in same])
        kg = np.array([b for _, b in same])
        op, gp = ores.tr_param[ko], gtr["param"][kg]
        ocov, gcov = ores.tr_cov[ko], gtr["cov"][kg]
        diag_i = [0, 2, 5, 9, 14]
        sig = np.sqrt(np.abs(ocov[:, diag_i]))
        scale = np.maximum(np.abs(op), sig)
        par_err = np.abs(gp - op) / np.where(scale > 0, scale, 1.0)
        ii, jj = np.tril_indices(5)
        cscale = np.sqrt(np.abs(ocov[:, [diag_i[i] for i in ii]] * ocov[:, [diag_i[j] for j in jj]]))
        cov_err = np.abs(gcov - ocov) / np.where(cscale > 0, cscale, 1.0)
        ok_status = gtr["status"][kg] == ores.tr_status[ko]
        good = ok_status & (ores.tr_status[ko] == 0)
        rep["param_max_rel_err"] = [float(v) for v in par_err[good].max(0)] if good.any() else [0.0] * 5
        # the plain element-wise relative error, reported beside the scaled
        # bar above: parameters with |p| > sigma_p, diagonal covariance terms
        big = np.abs(op) > sig
        plain = np.abs(gp - op) / np.where(big, np.abs(op), 1.0)
        rep["param_plain_rel_err"] = [float(plain[good & big[:, i], i].max()) if (good & big[:, i]).any() else 0.0
                                      for i in range(5)]
        dg = np.abs(gcov[:, diag_i] - ocov[:, diag_i]) / np.maximum(np.abs(ocov[:, diag_i]), 1e-300)
        rep["cov_diag_plain_rel_err"] = float(dg[good].max()) if good.any() else 0.0
        rep["cov_max_rel_err"] = float(cov_err[good].max()) if good.any() else 0.0
        chi2_err = np.abs(gtr["chi2"][kg] - ores.tr_chi2[ko]) / np.maximum(ores.tr_chi2[ko], 1.0)
        rep["chi2_max_rel_err"] = float(chi2_err[good].max()) if good.any() else 0.0
        rep["ndf_mismatch"] = int((gtr["ndf"][kg] != ores.tr_ndf[ko]).sum())
        rep["status_mismatch"] = int((~ok_status).sum())
        rep["param_fail"] = int((par_err[good] > rtol_par).any(1).sum())
        rep["cov_fail"] = int((cov_err[good] > rtol_cov).any(1).sum())
        rep["xref_mismatch"] = int((gtr["x_ref"][kg] != ores.tr_x_ref[ko])[good].sum())
    else:
        rep.update(param_max_rel_err=[0.0] * 5, param_plain_rel_err=[0.0] * 5, cov_diag_plain_rel_err=0.0,
                   cov_max_rel_err=0.0, chi2_max_rel_err=0.0, ndf_mismatch=0,
                   status_mismatch=0, param_fail=0, cov_fail=0, xref_mismatch=0)

    # ---------------------------------------------------------------- efficiency
    qo = evaluate(ev, ores.tr_inst, ores.tr_offset, ores.tr_ncl, ores.tr_ids)
    qg = evaluate(ev, gtr["instance"], gtr["offset"], gtr["n_cl"], gtr["cluster_ids"])
    rep["eff_oracle"], rep["eff_gpu"] = qo["efficiency"], qg["efficiency"]
    rep["fake_oracle"], rep["fake_gpu"] = qo["fake_rate"], qg["fake_rate"]
    rep["excused_fraction_nf"] = rep["nf_excused"] / max(1, n)
    rep["excused_fraction_tracks"] = rep["track_excused"] / max(1, ores.n_tracks)
    rep["tracklet_unexcused_fraction"] = rep["tracklet_unexcused"] / max(1, rep["tracklets_compared"])
    rep["pass"] = bool(
        rep["nf_unexcused"] == 0 and rep["clean_unexcused"] == 0 and rep["start_unexcused"] == 0
        and rep["tracklet_unexcused_fraction"] < 1e-3 and rep["weight_unexcused"] == 0
        and rep["track_unexcused"] == 0
        and rep["param_fail"] == 0 and rep["cov_fail"] == 0 and rep["ndf_mismatch"] == 0
        and rep["status_mismatch"] == 0 and rep["xref_mismatch"] == 0
        and rep["excused_fraction_nf"] < 1e-3 and rep["excused_fraction_tracks"] < 1e-3
        and abs(rep["eff_oracle"] - rep["eff_gpu"]) <= eff_tol)
    return rep
