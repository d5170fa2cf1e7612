"""Host-side measures of the second transform (the displaced-jet module):
the vertex cell of a position, the jet-matching rule (a kept peak within one
radius bin and one circular azimuth bin of the true vertex cell), and the fit
residuals of candidates whose hits are mostly one track's.  No GPU."""
import math

import numpy as np

import synth
from paper_1309_6275_gb300 import displaced

VD = dict(r_max=16.0, n_r=16, n_theta=64)


def test_vertex_cell_edges_and_azimuth_wrap():
    dq = 2 * math.pi / 64
    assert displaced.vertex_cell(VD, 0.0, -math.pi) == (0, 0)
    assert displaced.vertex_cell(VD, 15.999, math.pi - 1e-9) == (15, 63)
    assert displaced.vertex_cell(VD, 1.0, math.pi)[1] == 0          # +pi is -pi
    for q in (0, 17, 63):
        assert displaced.vertex_cell(VD, 3.5, -math.pi + (q + 0.5) * dq) == (3, q)
    assert displaced.vertex_cell(VD, 2.0 - 1e-12, 0.0)[0] == 1       # bin edge at 2 cm
    assert displaced.vertex_cell(VD, 2.0, 0.0)[0] == 2


def _event(vr, vth):
    z = np.zeros(0, np.float32)
    return synth.Event(x=z, y=z, z=z, layer=np.zeros(0, np.int8), track=np.zeros(0, np.int32),
                       vr=np.asarray(vr, float), vtheta=np.asarray(vth, float))


def test_match_counts_found_jets_and_fakes_across_the_wrap():
    ev = _event([5.5, 10.2], [0.1, -math.pi + 0.01])
    j0 = displaced.vertex_cell(VD, 5.5, 0.1)
    j1 = displaced.vertex_cell(VD, 10.2, -math.pi + 0.01)
    assert j1[1] == 0
    kept = [np.array([0, j0[0] + 1, j0[1] - 1, 9]),      # diagonal neighbour: found
            np.array([0, j1[0], 63, 9]),                 # azimuth 63 is next to 0: found
            np.array([0, 2, 40, 9])]                     # far from both: a fake
    assert displaced.match(VD, ev, kept) == (2, 2, 1)
    far = [np.array([0, j0[0] + 2, j0[1], 9])]           # two radius bins off
    assert displaced.match(VD, ev, far) == (2, 0, 1)
    assert displaced.match(VD, ev, []) == (2, 0, 0)


def test_fit_quality_keeps_fitted_majority_candidates():
    z = np.zeros(8, np.float32)
    ev = synth.Event(x=z, y=z, z=z, layer=np.zeros(8, np.int8),
                     track=np.array([0, 0, 0, 1, 1, 0, -1, 1], np.int32),
                     rho=np.array([1e-3, -2e-3]), d0=np.array([0.5, -1.0]))
    assign = np.array([0, 0, 0, 1, 1, 1, 0, 1])
    tracks = [dict(status=1, d0=0.52, rho=1.1e-3),       # 3 of 4 hits from track 0
              dict(status=1, d0=-0.9, rho=-2e-3),        # 3 of 4 from track 1 (one is 0's)
              dict(status=0, d0=9.0, rho=0.0)]           # not fitted
    n_fit, rd0, rrho = displaced.fit_quality(ev, assign, tracks)
    assert n_fit == 2
    assert np.allclose(rd0, [0.02, 0.1]) and np.allclose(rrho, [1e-4, 0.0])
    # a candidate whose hits split evenly between two tracks gives no residual
    tie = np.array([0, 0, 1, 1, 1, 1, 0, 0])
    ev2 = synth.Event(x=z, y=z, z=z, layer=np.zeros(8, np.int8),
                      track=np.array([0, 1, 0, 1, 0, 1, 0, 1], np.int32),
                      rho=np.array([1e-3, -2e-3]), d0=np.array([0.5, -1.0]))
    n_fit, rd0, _ = displaced.fit_quality(ev2, tie, tracks[:2])
    assert n_fit == 2 and rd0.size == 0
