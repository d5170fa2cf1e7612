"""Displaced-jet finding (Sections 6-7): the first transform over hits, then
the second transform (ht_vertex_*) over its candidates, through the C ABI.

This module only sequences the library calls and measures the result: a
jet counts as found when a reported vertex peak outside the beam pipe lies
within one radius bin and one azimuth bin (circular) of the cell holding the
jet's true vertex; every other reported peak is a fake.
"""
import math

import numpy as np


def fit_quality(ev, assign, tracks):
    """For fitted candidates (status 1) whose assigned hits are mostly one
    track's: d0 and rho residuals against that track's truth and the number
    of such candidates.  tracks: the event's ht_track records."""
    assign = np.asarray(assign)
    res_d0, res_rho, n_fit = [], [], 0
    for m in range(len(tracks)):
        if tracks[m]["status"] != 1:
            continue
        n_fit += 1
        tr = ev.track[assign == m]
        tr = tr[tr >= 0]
        if tr.size == 0:
            continue
        vals, cnts = np.unique(tr, return_counts=True)
        b = int(np.argmax(cnts))
        if cnts[b] * 2 <= (assign == m).sum():
            continue
        t = vals[b]
        res_d0.append(tracks[m]["d0"] - ev.d0[t])
        res_rho.append(tracks[m]["rho"] - ev.rho[t])
    return n_fit, np.array(res_d0), np.array(res_rho)


def vertex_cell(vd, r, theta):
    """(radius bin, azimuth bin) of a vertex position."""
    dr = vd["r_max"] / vd["n_r"]
    nt = vd["n_theta"]
    q = int(math.floor((theta + math.pi) / (2.0 * math.pi / nt))) % nt
    return int(math.floor(r / dr)), q


def match(vd, ev, kept):
    """(jets, found, fakes) for one event's reported peaks outside r_keep."""
    nt = vd["n_theta"]
    used = set()
    found = 0
    for jt in range(len(ev.vr)):
        jb, qb = vertex_cell(vd, ev.vr[jt], ev.vtheta[jt])
        near = [i for i, p in enumerate(kept)
                if abs(int(p[1]) - jb) <= 1 and min((int(p[2]) - qb) % nt, (qb - int(p[2])) % nt) <= 1]
        found += bool(near)
        used |= set(near)
    return len(ev.vr), found, len(kept) - len(used)


class DisplacedJetPipeline:
    """Batched first transform + second transform for batches of events."""

    def __init__(self, g, vd, max_events, max_hits, cap=1 << 16, vcap=4096):
        from . import ht
        self.ht = ht
        self.g, self.vd, self.cap = g, vd, cap
        self.G = ht.Geometry(g)
        self.B = ht.Batch(self.G, max_events=max_events, max_hits=max_hits, cap=cap)
        self.V = ht.Vertex(self.G, vd, max_events=max_events, cap=vcap)

    def run(self, x, y, z, offsets, stream=None):
        n_ev = len(offsets) - 1
        self.B.run(x, y, z, offsets, stream)
        self.V.run(self.B.peaks, self.B.counts, self.cap, n_ev, stream)

    def kept(self, e):
        r = self.V.event_results(e)
        return r["peaks"][r["first"]:]

    def close(self):
        self.V.close()
        self.B.close()
        self.G.close()
