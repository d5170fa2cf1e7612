"""CPU oracle for the Hough-transform track-finding path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.
"""
from . import oracle
from .oracle import (build, tables, edge_tables, vote, vote_hitmask, vote_swept, peaks,
                     associate, associate_dense, vote_z, atan2, run_event, vote_layers,
                     circle3, confirm, confirm_assign, run_event_tracks, CONFIRM_DEFAULT)

__all__ = ["oracle", "build", "tables", "edge_tables", "vote", "vote_hitmask", "vote_swept",
           "peaks", "associate", "associate_dense", "vote_z", "atan2", "run_event",
           "vote_layers", "circle3", "confirm", "confirm_assign", "run_event_tracks",
           "CONFIRM_DEFAULT"]
