"""Track-finding quality of one event's results against the generator truth.

Host-side numpy over the library's outputs (candidates and hit assignments);
no Hough arithmetic.  Definitions (Section 7 defines efficiency as the
fraction of the objects present that the algorithm identifies; its peak
finder is tuned for tracks of at least seven hits):

  reconstructable  a true track with at least ``min_track_hits`` hits whose
                   true (rho, d0) lies inside the accumulator's axes;
  track candidate  a candidate with at least ``min_hits`` assigned hits (what
                   the finder reports as a track);
  matched          a track candidate whose assigned hits are more than half
                   from one true track, with at least ``min_hits`` of them:
                   that track is then found;
  efficiency       found reconstructable tracks / reconstructable tracks;
  fake             a track candidate that matches no true track;
  duplicate        a track candidate matched to a track that an earlier
                   (smaller index) candidate already matched.

The candidate-level measure (some candidate inside the 3 x 3 x 3 box of the
cell holding the track's true parameters) is reported beside it: it says
where peaks are, not whether hits were collected, and at high candidate
density a random box holds a candidate by chance (``chance`` gives that
probability, 1 - (1 - density)^27).
"""
import math

import numpy as np


def true_cells(g, ev):
    """(i, j, k) cell of every true track's parameters (i, j may be outside
    the axes) -- the cell the vote bins a circle with those parameters in."""
    NR, ND, NP = g["n_rho"], g["n_d0"], g["n_phi0"]
    delta = 2.0 * g["d0_half"] / ND
    ti = np.floor((np.asarray(ev.rho) + g["rho_max"]) / (2.0 * g["rho_max"] / NR)).astype(np.int64)
    tj = np.floor(np.asarray(ev.d0) / delta + ND / 2.0 + 0.5).astype(np.int64)
    tk = np.floor((np.asarray(ev.phi0) + math.pi) / (2.0 * math.pi / NP)).astype(np.int64) % NP
    return ti, tj, tk


def reconstructable(g, ev, min_track_hits=7):
    ti, tj, _ = true_cells(g, ev)
    nh = np.asarray(ev.n_track_hits)
    return ((nh >= min_track_hits) & (ti >= 0) & (ti < g["n_rho"]) & (tj >= 0) &
            (tj < g["n_d0"]))


def track_quality(g, ev, assign, peaks=None, min_hits=5, min_track_hits=7):
    """Counts of one event: n_rec, found, track_cands, matched, fakes,
    duplicates, and (with peaks) cand_found / cand_chance for the
    candidate-level measure."""
    assign = np.asarray(assign)
    ok = reconstructable(g, ev, min_track_hits)
    ntr = ok.shape[0]
    m = assign >= 0
    cand = assign[m].astype(np.int64)
    trk = np.asarray(ev.track)[m].astype(np.int64)
    found = np.zeros(ntr, bool)
    track_cands = matched = fakes = dups = 0
    if cand.size:
        ncand = int(cand.max()) + 1
        nass = np.bincount(cand, minlength=ncand)
        is_tc = nass >= min_hits
        track_cands = int(is_tc.sum())
        # majority track of each candidate (true-track hits only)
        t_ok = trk >= 0
        key = cand[t_ok] * (ntr + 1) + trk[t_ok]
        u, c = np.unique(key, return_counts=True)
        uc, ut = u // (ntr + 1), u % (ntr + 1)
        good = (c >= min_hits) & (2 * c > nass[uc])
        owner = np.full(ncand, -1, np.int64)
        owner[uc[good]] = ut[good]            # at most one track can hold > half
        seen = np.zeros(ntr, bool)
        for mm in np.flatnonzero(is_tc):      # increasing candidate index
            t = owner[mm]
            if t < 0:
                fakes += 1
            elif seen[t]:
                dups += 1
                matched += 1
            else:
                seen[t] = True
                matched += 1
        found = seen
    res = dict(n_rec=int(ok.sum()), found=int((found & ok).sum()), track_cands=track_cands,
               matched=matched, fakes=fakes, duplicates=dups)
    if peaks is not None:
        res.update(candidate_level(g, ev, peaks, ok))
    return res


def candidate_level(g, ev, peaks, ok=None):
    """Reconstructable tracks with a candidate in the 3 x 3 x 3 box of their
    true cell (phi0 circular), and the chance that a random box holds one."""
    NR, ND, NP = g["n_rho"], g["n_d0"], g["n_phi0"]
    if ok is None:
        ok = reconstructable(g, ev)
    pk = np.asarray(peaks).reshape(-1, 4)
    ti, tj, tk = true_cells(g, ev)
    f = np.zeros(ok.shape[0], bool)
    if pk.shape[0] and ok.any():
        occ = np.zeros((NR, ND, NP), bool)
        occ[pk[:, 0], pk[:, 1], pk[:, 2]] = True
        t = np.flatnonzero(ok)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                ii, jj = ti[t] + di, tj[t] + dj
                inb = (ii >= 0) & (ii < NR) & (jj >= 0) & (jj < ND)
                for dk in (-1, 0, 1):
                    kk = (tk[t] + dk) % NP
                    f[t[inb]] |= occ[ii[inb], jj[inb], kk[inb]]
    dens = pk.shape[0] / float(NR * ND * NP)
    return dict(cand_found=int((f & ok).sum()), cand_chance=1.0 - (1.0 - dens) ** 27)


def summarize(rows):
    """Sum per-event count dicts and add the rates."""
    tot = {}
    for r in rows:
        for k, v in r.items():
            if k != "cand_chance":
                tot[k] = tot.get(k, 0) + v
    n = max(tot.get("n_rec", 0), 1)
    tc = max(tot.get("track_cands", 0), 1)
    tot["efficiency"] = tot.get("found", 0) / n
    tot["fake_rate"] = tot.get("fakes", 0) / tc
    tot["duplicate_rate"] = tot.get("duplicates", 0) / tc
    if "cand_found" in tot:
        tot["cand_efficiency"] = tot["cand_found"] / n
        ch = [r["cand_chance"] for r in rows if "cand_chance" in r]
        tot["cand_chance"] = float(np.mean(ch)) if ch else 0.0
    return tot
