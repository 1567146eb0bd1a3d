"""Helpers of the GPU tests: run the CUDA library on an Event and bring the
results to the host; slice batch results to a subset of instances."""
import numpy as np


def run_gpu(ev, precision="mixed", batched=False, with_row=True, tuning=None, tracker=None, cap=None):
    import torch
    import paper_2502_09138_gb300 as G
    trk = tracker or G.Tracker(precision=precision, bz=ev.bz,
                               cuts=G.default_cuts(sig_readout=ev.sigma.at_readout,
                                                   sig_cathode=ev.sigma.at_cathode))
    if tuning:
        trk.set_tuning(**tuning)
    dc = G.DeviceClusters.from_event(ev, with_row=with_row)
    out = trk.make_output(ev.n, *(cap or (None, None)))
    trk.track(dc, out, batched=batched)
    dbg = trk.debug(ev.n)
    torch.cuda.synchronize()
    status = trk.device_status()
    return out.to_host(), dbg.to_host(), status, trk


def slice_instances(ev, gtr, gdbg, idx):
    """GPU results of instances ``idx`` with ids renumbered as in ev.select_instances(idx)."""
    idx = np.asarray(idx)
    offs = ev.sector_offsets
    old = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in idx])
    remap = -np.ones(ev.n, np.int64)
    remap[old] = np.arange(old.shape[0])
    rm = lambda a: np.where(a >= 0, remap[np.maximum(a, 0)], -1).astype(np.int32)
    dbg = {k: rm(gdbg[k][old]) for k in ("up", "down", "upc", "downc")}
    dbg["weight"] = gdbg["weight"][old]
    # tracklets of the selected instances, in order
    inst_of = ev.instance_of_cluster()
    tl_inst = inst_of[gdbg["tl_start"]]
    pos = {int(i): k for k, i in enumerate(idx)}
    sel_tl = np.array([t for t in range(len(tl_inst)) if int(tl_inst[t]) in pos], np.int64)
    order = sorted(sel_tl, key=lambda t: (pos[int(tl_inst[t])], t))
    new_of_tl = {int(t): k for k, t in enumerate(order)}
    dbg["tl_start"] = rm(gdbg["tl_start"][order]) if order else np.zeros(0, np.int32)
    dbg["tl_hits"] = rm(gdbg["tl_hits"][order]) if order else np.zeros((0, gdbg["tl_hits"].shape[1]), np.int32)
    dbg["tl_nhits"] = gdbg["tl_nhits"][order] if order else np.zeros(0, np.int32)
    # tracks
    ks = [k for k in range(gtr["n_tracks"]) if int(gtr["instance"][k]) in pos]
    ks.sort(key=lambda k: (pos[int(gtr["instance"][k])], k))
    tr = {f: gtr[f][ks] for f in ("n_cl", "ndf", "status", "x_ref", "param", "cov", "chi2")}
    tr["instance"] = np.array([pos[int(gtr["instance"][k])] for k in ks], np.int32)
    offs_new, ids = [], []
    o = 0
    for k in ks:
        a, b = gtr["offset"][k], gtr["offset"][k] + gtr["n_cl"][k]
        ids.append(rm(gtr["cluster_ids"][a:b]))
        offs_new.append(o)
        o += b - a
    tr["offset"] = np.array(offs_new, np.int32)
    tr["cluster_ids"] = np.concatenate(ids) if ids else np.zeros(0, np.int32)
    tr["n_tracks"] = len(ks)
    dbg["tr_tracklet"] = np.array([new_of_tl[int(gdbg["tr_tracklet"][k])] for k in ks], np.int64)
    return tr, dbg
