"""Track-finding quality against generator truth (evaluation only).

A reconstructed track's label is the majority MC particle among its clusters
(ties to the smaller id); it is "good" if at least ``purity`` of its clusters
carry that label.  A findable unit is an (MC particle, sector instance) pair
with at least ``n_min`` clusters.  Efficiency = found findable units / all
findable units, where found means at least one good track with that label in
that instance; fake rate = non-good tracks / all tracks; clone rate = good
tracks beyond the first per unit / found units.
"""
import numpy as np


def evaluate(ev, tr_inst, tr_offset, tr_ncl, tr_ids, n_min=20, purity=0.9):
    mc = ev.mc.astype(np.int64)
    inst_of = ev.instance_of_cluster()
    key_all = inst_of * (1 << 32) + np.where(mc >= 0, mc, (1 << 32) - 1)
    sig = mc >= 0
    uk, uc = np.unique(key_all[sig], return_counts=True)
    findable = set(uk[uc >= n_min].tolist())
    good, labels = 0, []
    found = {}
    n_tracks = int(len(tr_inst))
    for k in range(n_tracks):
        o, n = int(tr_offset[k]), int(tr_ncl[k])
        ids = tr_ids[o:o + n]
        m = mc[ids]
        if n == 0:
            continue
        vals, cnt = np.unique(m, return_counts=True)
        best = vals[np.argmax(cnt)]   # np.unique sorts: argmax picks the smaller id on ties
        frac = cnt.max() / n
        if best >= 0 and frac >= purity:
            good += 1
            key = int(tr_inst[k]) * (1 << 32) + int(best)
            found[key] = found.get(key, 0) + 1
    n_found = sum(1 for k in found if k in findable)
    clones = sum(v - 1 for k, v in found.items() if k in findable)
    return dict(
        findable=len(findable),
        found=n_found,
        efficiency=n_found / max(1, len(findable)),
        tracks=n_tracks,
        fake_rate=(n_tracks - good) / max(1, n_tracks),
        clone_rate=clones / max(1, n_found),
    )
