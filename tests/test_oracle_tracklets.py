"""Pins of the oracle's tracklet growth (S5) on a hand-worked fixture.

tests/golden/tracklet_hand_fixture.json lays out ten sector instances on a
60-row geometry, each built so that one rule of the stated reading decides
its result: a gap of exactly max_miss rows and one of max_miss + 1, a
chi2-rejected reciprocal link (a miss, and its row is not searched), a
downward pass that drops an upward hit without searching its row, the 1 cm
sector-edge margin on the way up and on the way down (and on either side of
the sector), a search-window tie broken by the smaller id, and a smeared
line across an 8-row gap.  Every expected value (links, start hits, the
row-indexed hit lists, stop reasons, selected tracks) was worked out by hand.

The second test plants each plausible mistake in a copy of the oracle and
checks that the fixture then fails: the fixture pins the control flow, not
just the oracle as it happens to be.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
STOP = {0: "END", 1: "PROP", 2: "EDGE", 3: "MISS", 4: "SINPHI"}


def load_fixture():
    with open(os.path.join(HERE, "golden", "tracklet_hand_fixture.json")) as f:
        return json.load(f)


def fixture_arrays(fx):
    """Concatenate the instances: sector offsets, y, z (float32 values) and rows."""
    offs, y, z, row = [0], [], [], []
    for inst in fx["instances"]:
        for r, yy, zz in inst["clusters"]:
            row.append(r)
            y.append(yy)
            z.append(zz)
        offs.append(len(row))
    return (np.array(offs, np.int64), np.array(y, np.float32), np.array(z, np.float32),
            np.array(row, np.int32))


def fixture_geometry(fx):
    g = fx["geometry"]
    return synth.Geometry(row_x=np.array(g["row_x"]), tan_half_sector=g["tan_half_sector"], z_max=g["z_max"])


def run_oracle(fx):
    offs, y, z, row = fixture_arrays(fx)
    cuts = oracle.Cuts(**fx["cuts"])
    return oracle.track(fixture_geometry(fx), cuts, offs, y.astype(np.float64), z.astype(np.float64), row=row)


def compare(fx, res, check_stops=True):
    """List of differences between an oracle result and the fixture (empty = equal)."""
    offs = fixture_arrays(fx)[0]
    bad = []
    n_rows = len(fx["geometry"]["row_x"])
    for i, inst in enumerate(fx["instances"]):
        base = int(offs[i])
        loc = lambda a: int(a) - base if a >= 0 else -1
        for k, want in inst.get("links", {}).items():
            c = base + int(k)
            got = [loc(res.up[c]), loc(res.down[c]), loc(res.upc[c]), loc(res.downc[c])]
            if got != want:
                bad.append((inst["name"], "links", k, got, want))
        tl = [t for t in range(res.n_tracklets) if int(res.tl_inst[t]) == i]
        starts = [loc(res.tl_start[t]) for t in tl]
        if starts != inst["starts"]:
            bad.append((inst["name"], "starts", starts, inst["starts"]))
            continue
        for t, want in zip(tl, inst["tracklets"]):
            hits = [loc(res.tl_hits[t, r]) for r in range(n_rows) if res.tl_hits[t, r] >= 0]
            if hits != want["hits"]:
                bad.append((inst["name"], "hits of tracklet", want["start"], hits, want["hits"]))
            if check_stops:
                got = (STOP[int(res.tl_stop_up[t])], STOP[int(res.tl_stop_down[t])])
                if got != (want["stop_up"], want["stop_down"]):
                    bad.append((inst["name"], "stops of tracklet", want["start"], got))
        tracks = [[loc(c) for c in res.track_ids(k)] for k in range(res.n_tracks) if int(res.tr_inst[k]) == i]
        if tracks != inst["tracks"]:
            bad.append((inst["name"], "tracks", tracks, inst["tracks"]))
    return bad


def test_tracklet_fixture_hand_values():
    fx = load_fixture()
    res = run_oracle(fx)
    assert compare(fx, res) == []


def test_tracklet_fixture_is_far_from_every_cut():
    """Every decision of the fixture lies well away from its cut (the oracle's
    logged relative margins), apart from the two intended exact ties, so the
    hand-worked lists cannot flip under rounding, here or on the GPU."""
    fx = load_fixture()
    res = run_oracle(fx)
    for t in range(res.n_tracklets):
        name = fx["instances"][int(res.tl_inst[t])]["name"]
        if name.startswith("T"):
            assert res.tl_margin[t] == 0.0       # the exact tie
        elif name.startswith("E"):
            assert res.tl_margin[t] > 0.02        # 0.5 cm of ~24 cm at the edge
        else:
            assert res.tl_margin[t] > 0.3, (name, res.tl_margin[t])


# (label, original text, replacement): each is a plausible mistake in S5; the
# fixture must fail with every one of them planted.
_UP_ACCEPT = "    if (cand >= 0 && try_hit(t, cand, p, C, &margin)) {\n      up_hit[r] = cand;"
_DOWN_PICK = ("    int64_t cand = up_hit[r] >= 0 ? up_hit[r] : search_row(t, r, p, C, &margin);\n"
              "    if (cand >= 0 && try_hit(t, cand, p, C, &margin)) {\n      tl->hits[r] = cand;")
MISTAKES = [
    ("stop after max_miss misses instead of more than max_miss",
     "if (++miss > c->max_miss)", "if (++miss >= c->max_miss)"),
    ("stop after more than max_miss + 1 misses",
     "if (++miss > c->max_miss)", "if (++miss > c->max_miss + 1)"),
    ("search the row after a chi2-rejected link",
     _UP_ACCEPT,
     "    int ok_ = cand >= 0 && try_hit(t, cand, p, C, &margin);\n"
     "    if (!ok_ && cand >= 0 && prev_row == r - 1 && res->upc[prev] == cand) {\n"
     "      cand = search_row(t, r, p, C, &margin);\n"
     "      ok_ = cand >= 0 && try_hit(t, cand, p, C, &margin);\n"
     "    }\n"
     "    if (ok_) {\n      up_hit[r] = cand;"),
    ("a chi2-rejected link is not a missed row",
     "    } else {\n      if (++miss > c->max_miss) { stop = STOP_MISS; break; }\n    }\n  }\n  tl->stop_up = stop;",
     "    } else if (!(prev_row == r - 1 && res->upc[prev] >= 0)) {\n"
     "      if (++miss > c->max_miss) { stop = STOP_MISS; break; }\n    }\n  }\n  tl->stop_up = stop;"),
    ("search a row whose upward hit the downward pass rejected",
     _DOWN_PICK,
     "    int64_t cand = up_hit[r] >= 0 ? up_hit[r] : search_row(t, r, p, C, &margin);\n"
     "    int ok_ = cand >= 0 && try_hit(t, cand, p, C, &margin);\n"
     "    if (!ok_ && up_hit[r] >= 0) {\n"
     "      cand = search_row(t, r, p, C, &margin);\n"
     "      ok_ = cand >= 0 && try_hit(t, cand, p, C, &margin);\n"
     "    }\n"
     "    if (ok_) {\n      tl->hits[r] = cand;"),
    ("keep an upward hit the downward pass rejected",
     _DOWN_PICK,
     "    int64_t cand = up_hit[r] >= 0 ? up_hit[r] : search_row(t, r, p, C, &margin);\n"
     "    if (cand >= 0 && (try_hit(t, cand, p, C, &margin) || up_hit[r] >= 0)) {\n      tl->hits[r] = cand;"),
    ("no edge margin",
     "double edge = X[r] * tanh_ + c->edge_margin;", "double edge = X[r] * tanh_;"),
    ("edge test on signed y",
     "if (fabs(p[0]) > edge) { stop = STOP_EDGE; break; }", "if (p[0] > edge) { stop = STOP_EDGE; break; }"),
    ("search tie to the larger id", "(d == d1 && i < best)", "(d == d1 && i > best)"),
    ("search tie to the first candidate in y order", "(d == d1 && i < best)", "(0)"),
    ("no covariance reset at the start of the downward pass",
     "  init_cov(t, C, t->z[up_hit[top_row]]);\n  tl->hits[top_row]", "  tl->hits[top_row]"),
    ("measurement variance dropped from the chi2",
     "  double S00 = C[0] + vy, S01 = C[1], S11 = C[6] + vz;\n  double det = S00 * S11 - S01 * S01;\n  double r0",
     "  double S00 = C[0], S01 = C[1], S11 = C[6];\n  double det = S00 * S11 - S01 * S01;\n  double r0"),
    ("initial direction with the wrong sign in y",
     "double p[5] = {t->y[h0], t->z[h0], dy / L, dz / L, 0.0};",
     "double p[5] = {t->y[h0], t->z[h0], -dy / L, dz / L, 0.0};"),
]


@pytest.mark.parametrize("label,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_tracklet_fixture_catches_planted_mistake(label, old, new, tmp_path):
    with open(os.path.join(os.path.dirname(oracle.__file__), "tpct_oracle.c")) as f:
        src = f.read()
    assert old in src, f"mutation site not found: {label}"
    path = oracle.build_variant(src.replace(old, new), str(tmp_path))
    fx = load_fixture()
    with oracle.using_library(oracle.load_library(path)):
        res = run_oracle(fx)
    assert compare(fx, res, check_stops=False) != [], f"fixture does not catch: {label}"
