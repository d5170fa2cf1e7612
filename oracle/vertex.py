"""Oracle of the second Hough transform: displaced-vertex finding.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; it shares no code with the
CUDA path.

Section 6 (Fig. 6) applies a second Hough transform to the candidate
tracks: tracks from one vertex lie on a sinusoid in (phi0, d0), and the
same peak finder locates those sinusoids; Section 7 drops features inside
the 3.0 cm beam pipe.  The paper gives no formulas; the readings here:

* A track is the straight line of its candidate cell centre: perigee
  P = d0 n, n = (-sin phi0, cos phi0), direction (cos phi0, sin phi0),
  d0 = (j - n_d0/2) delta (the straight-line approximation; the curvature is
  not used).  A vertex V = r (cos theta, sin theta) lies on it iff
  d0 = r sin(theta - phi0).
* Vertex space: theta_q = (2q + 1 - N) pi / N over [-pi, pi) (the phi0 axis
  formula, wrapping), radius bins of width r_max / n_r from 0.
* Each candidate votes once in every theta column where its line meets the
  ray at angle theta_q at r >= 0: den = sin theta_q cos phi0 - cos theta_q
  sin phi0 (products, then the difference), r = d0 / den, u = r / dr, a vote
  in bin floor(u) iff 0 <= u < n_r (den = 0 gives no vote; d0 = 0 votes in
  bin 0 of every column with den != 0).
* Peaks: the rule of the first transform on the 1 x n_r x n_theta array
  (r does not wrap, theta does); threshold T2 tracks.
* Interaction-point filter: peaks whose radius-bin centre (j + 1/2) dr is
  below r_keep are dropped; in the peak order (radius bin major) they are a
  prefix of the list.
All arithmetic is float64, one correctly rounded operation at a time.
"""
import math

import numpy as np

from . import oracle as O


def theta_tables(n_theta):
    """(theta, sin theta, cos theta) float64, libm sin/cos like the phi0 axis."""
    th = np.array([(2 * q + 1 - n_theta) * (math.pi / n_theta) for q in range(n_theta)])
    return th, np.array([math.sin(t) for t in th]), np.array([math.cos(t) for t in th])


def _peak_geom(vd):
    return dict(n_rho=1, n_d0=vd["n_r"], n_phi0=vd["n_theta"], n_z0=1, n_cot=1,
                threshold=vd["threshold"], count_bits=32, rho_max=1.0, d0_half=1.0,
                z0_max=1.0, cot_max=1.0)


def vote(g, vd, peaks, chunk=4096):
    """Vertex accumulator int64 [n_r, n_theta] and the number of votes.
    Candidates with count < vd['min_count'] (default 0) do not vote."""
    _, sphi, cphi, _ = O.tables(g)
    _, sth, cth = theta_tables(vd["n_theta"])
    NR, NT = vd["n_r"], vd["n_theta"]
    dr = vd["r_max"] / NR
    delta = 2.0 * g["d0_half"] / g["n_d0"]
    acc = np.zeros((NR, NT), np.int64)
    pk = np.asarray(peaks).reshape(-1, 4)
    pk = pk[pk[:, 3] >= vd.get("min_count", 0)]
    votes = 0
    for a in range(0, pk.shape[0], chunk):
        p = pk[a:a + chunk]
        d0 = (p[:, 1].astype(np.float64) - 0.5 * g["n_d0"]) * delta
        sp, cp = sphi[p[:, 2]][:, None], cphi[p[:, 2]][:, None]
        den = sth[None, :] * cp - cth[None, :] * sp
        with np.errstate(divide="ignore", invalid="ignore"):
            u = (d0[:, None] / den) / dr
        ok = (u >= 0.0) & (u < NR)
        m, q = np.nonzero(ok)
        b = np.floor(u[m, q]).astype(np.int64)
        np.add.at(acc, (b, q), 1)
        votes += int(m.shape[0])
    return acc, votes


def find(vd, acc, cap=None):
    """(peaks int32 [k, 4] = {0, r bin, theta bin, count}, total, first) where
    peaks[first:] are the ones outside r_keep."""
    pk, cnt = O.peaks(_peak_geom(vd), np.asarray(acc).reshape(1, vd["n_r"], vd["n_theta"]), cap)
    first = first_kept(vd, pk)
    return pk, cnt, first


def first_kept(vd, pk):
    dr = vd["r_max"] / vd["n_r"]
    centre = (np.asarray(pk)[:, 1].astype(np.float64) + 0.5) * dr
    return int(np.count_nonzero(centre < vd["r_keep"]))


def run(g, vd, peaks, cap=None):
    acc, votes = vote(g, vd, peaks)
    pk, cnt, first = find(vd, acc, cap)
    return dict(acc=acc, votes=votes, peaks=pk, count=cnt, first=first)
