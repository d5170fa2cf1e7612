"""Seeded synthetic silicon-tracker events.

This package is the only code shared by the CPU oracle's tests and the CUDA
path's tests and benchmarks.  It simulates detector hits from helix track
parameters (forward simulation) and holds none of the Hough-transform
arithmetic (no voting, binning, peak finding or association).
"""
from .configs import CONFIGS, KAPPA, B_FIELD, LAYER_R, geometry_of, track_geometry, track_of, learned_of
from .events import Event, make_event, make_jet_event, perigee_of, generate, helix_hits, make_stream

__all__ = ["CONFIGS", "KAPPA", "B_FIELD", "LAYER_R", "geometry_of", "track_geometry", "track_of", "learned_of",
           "Event", "make_event", "make_jet_event", "perigee_of", "generate", "helix_hits",
           "make_stream"]
