"""Synthetic event generator: counter-based RNG and workload shapes."""
import numpy as np

import synth
from synth import rng
from synth.events import truth_state


def test_splitmix64_known_answer():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first two outputs.
    g = rng._GOLDEN
    assert int(rng._mix64(np.uint64(0) + g)) == 0xE220A8397B1DCDAF
    assert int(rng._mix64(g * np.uint64(2))) == 0x6E789E6AA1B965F4


def test_uniform_and_normal_moments():
    u = rng.uniform(1, 0, np.arange(200000))
    assert 0.0 < u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.003
    n = rng.normal(1, 1, np.arange(200000))
    assert abs(n.mean()) < 0.01 and abs(n.std() - 1.0) < 0.01


def test_deterministic(event0):
    e2 = synth.generate_config(0)
    for f in ("x", "y", "z", "charge", "row", "mc", "sector_offsets"):
        assert np.array_equal(getattr(event0, f), getattr(e2, f))


def test_layout(event0, event1):
    g = synth.default_geometry()
    for ev in (event0, event1):
        assert ev.sector_offsets[0] == 0 and ev.sector_offsets[-1] == ev.n
        assert np.all(np.diff(ev.sector_offsets) >= 0)
        assert np.array_equal(ev.x, g.row_x[ev.row].astype(np.float32))
        inst = ev.instance_of_cluster()
        side_c = ev.sectors[inst] >= 18
        assert np.all(ev.z[ev.mc >= 0][~side_c[ev.mc >= 0]] > -1.0)
    assert event0.n_instances == 1 and event0.sectors[0] == 0
    assert event1.n_instances == 36
    assert 1.2e6 < event1.n < 1.45e6          # "about 1.3M clusters"
    noise = (event1.mc < 0).mean()
    assert 0.085 < noise < 0.095                # 10 % of the signal


def test_truth_state_on_generated_hit(event0):
    # a noiseless copy: every hit lies on the truth trajectory at its row
    ev = synth.generate_config(0, smear=False, keep_exact=True)
    g = synth.default_geometry()
    for i in range(0, ev.n, 997):
        st, ok = truth_state(ev, int(ev.mc[i]), 0, g.row_x[ev.row[i]])
        assert ok
        assert abs(st[0] - ev.y64[i]) < 1e-9 and abs(st[1] - ev.z64[i]) < 1e-9
