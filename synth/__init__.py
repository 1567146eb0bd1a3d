"""Seeded synthetic TPC events: the inputs that both the CUDA tracker and the
CPU oracle consume, plus generator truth for efficiency evaluation.

This package holds no tracking arithmetic.  It simulates detector hits of
charged particles (exact circle geometry in the transverse plane), adds
Gaussian smearing, inefficiency and noise, and draws every random number from
a counter-based SplitMix64 generator so that an event depends only on its seed.

The workloads stand in for the ALICE data behind Tables 1-3 of the paper
(50 kHz Pb-Pb Monte Carlo, 650 kHz pp and 47 kHz Pb-Pb real data), which are
not available: a single 20-degree sector with 200 tracks, a central Pb-Pb-like
event of 9000 tracks over 36 sectors, and batches / time frames of collisions
of uneven multiplicity.
"""
from .geometry import Geometry, default_geometry
from .events import Event, generate_event, generate_config, concat_events, seed_for

__all__ = ["Geometry", "default_geometry", "Event", "generate_event",
           "generate_config", "concat_events", "seed_for"]
