"""Pins of the oracle's dense-event track finder: the distinct-layer vote, the
circle through three points, the candidate confirmation and the final hit
assignment (Section 5: local maxima are candidates that costlier steps
confirm; Fig. 5 refines them; Section 7 tunes for tracks of seven or more
hits, i.e. layers).

Each check reaches its answer by another route than the oracle's own code:
per-layer plain votes, circles with known centres, noise-free helices at cell
centres, exact rotations of the scene, and hand-built edits of the hits.
Planted mistakes (a copy of the oracle's rule with one step wrong) show that
the properties used here do catch them.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_1309_6275_gb300 import quality


def small_geom(**kw):
    g = dict(n_rho=16, n_d0=32, n_phi0=64, rho_max=0.0114, d0_half=10.0, n_z0=16,
             n_cot=16, z0_max=32.0, cot_max=6.5, threshold=3, count_bits=32)
    g.update(kw)
    return g


def centre_params(g, i, j, k):
    _, _, _, rho = oracle.tables(g)
    delta = 2.0 * g["d0_half"] / g["n_d0"]
    return (rho[i], (j - g["n_d0"] / 2) * delta,
            (2 * k + 1 - g["n_phi0"]) * math.pi / g["n_phi0"])


def helix_scene(g, cells, radii=synth.LAYER_R):
    """Noise-free float32 hits of tracks with parameters at the given cell
    centres; returns x, y, layer, track."""
    xs, ys, ls, ts = [], [], [], []
    for t, (i, j, k) in enumerate(cells):
        rho, d0, phi0 = centre_params(g, i, j, k)
        X, Y, Z, lay, L = synth.helix_hits(rho, d0, phi0, radii=radii)
        xs.append(X); ys.append(Y); ls.append(lay); ts.append(np.full(len(X), t))
    return (np.concatenate(xs).astype(np.float32), np.concatenate(ys).astype(np.float32),
            np.concatenate(ls).astype(np.uint8), np.concatenate(ts).astype(np.int32))


# ----------------------------------------------------------- distinct-layer vote
@pytest.mark.parametrize("seed", [0, 1])
def test_layer_vote_is_the_number_of_layers_with_a_plain_vote(seed):
    """Definition by a second route: a cell's count is the number of layers l
    whose hits alone give the cell at least one plain vote."""
    g = small_geom()
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], seed)
    acc, st = oracle.vote_layers(g, ev.x, ev.y, ev.layer)
    ref = np.zeros_like(acc)
    votes = 0
    for l in range(10):
        s = ev.layer == l
        a, sl = oracle.vote(g, ev.x[s], ev.y[s])
        ref += a > 0
        votes += sl["votes"]
    assert np.array_equal(acc, ref)
    assert st["votes"] == votes
    assert acc.max() <= 10


def test_layer_vote_counts_hits_on_distinct_layers_like_the_plain_vote():
    """Every hit on its own layer: the count is the number of distinct hits
    voting in the cell -- the plain count unless one hit puts both roots in
    one cell."""
    g = small_geom()
    rng = np.random.default_rng(3)
    r = rng.uniform(5.0, 60.0, 12)
    ph = rng.uniform(-math.pi, math.pi, 12)
    x, y = (r * np.cos(ph)).astype(np.float32), (r * np.sin(ph)).astype(np.float32)
    lay = np.arange(12, dtype=np.uint8)
    acc, _ = oracle.vote_layers(g, x, y, lay)
    ref = np.zeros_like(acc)
    for h in range(12):
        a, _ = oracle.vote(g, x[h:h + 1], y[h:h + 1])
        ref += a > 0
    assert np.array_equal(acc, ref)
    plain, _ = oracle.vote(g, x, y)
    assert np.all(acc <= plain)


def test_layer_vote_of_one_layer_is_the_plain_vote_occupancy():
    g = small_geom()
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 4)
    lay = np.zeros(ev.n_hits, np.uint8)
    acc, _ = oracle.vote_layers(g, ev.x, ev.y, lay)
    plain, _ = oracle.vote(g, ev.x, ev.y)
    assert np.array_equal(acc, (plain > 0).astype(np.int64))


def test_layer_vote_of_a_helix_at_centres_peaks_in_its_cell():
    g = synth.geometry_of("event100_256")
    i, j, k = 100, 70, 300
    x, y, lay, _ = helix_scene(g, [(i, j, k)])
    acc, _ = oracle.vote_layers(g, x, y, lay)
    assert acc[i, j, k] == 10 == acc.max()


def test_layer_vote_with_all_masks_open_is_the_unmasked_vote():
    g = small_geom()
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 5)
    a, _ = oracle.vote_layers(g, ev.x, ev.y, ev.layer)
    b, _ = oracle.vote_layers(g, ev.x, ev.y, ev.layer,
                              masks=np.full(ev.n_hits, ~np.uint64(0), np.uint64))
    assert np.array_equal(a, b)


def test_layer_vote_masked_keeps_exactly_the_allowed_hits_layers():
    """With hit h's mask empty, h no longer counts anywhere: the count is the
    layer vote of the other hits."""
    g = small_geom()
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 6)
    masks = np.full(ev.n_hits, ~np.uint64(0), np.uint64)
    drop = np.arange(ev.n_hits) % 3 == 0
    masks[drop] = 0
    a, _ = oracle.vote_layers(g, ev.x, ev.y, ev.layer, masks=masks)
    b, _ = oracle.vote_layers(g, ev.x[~drop], ev.y[~drop], ev.layer[~drop])
    assert np.array_equal(a, b)


# ----------------------------------------------------------- circle through three points
def test_circle3_on_known_circles():
    assert oracle.circle3((5, 0), (0, 5), (-5, 0)) == pytest.approx((0.0, 0.0, 5.0), abs=1e-15)
    assert oracle.circle3((3, 4), (-3, 4), (0, -5)) == pytest.approx((0.0, 0.0, 5.0), abs=1e-15)
    assert oracle.circle3((1, 1), (1, 3), (3, 1)) == pytest.approx((2.0, 2.0, math.sqrt(2)))
    assert oracle.circle3((0, 0), (1, 1), (2, 2)) is None
    assert oracle.circle3((1, 2), (1, 2), (4, 5)) is None


def test_circle3_recovers_random_circles_and_ignores_point_order():
    rng = np.random.default_rng(7)
    for _ in range(200):
        xc, yc = rng.uniform(-2000, 2000, 2)
        R = rng.uniform(50, 3000)
        a = rng.uniform(-math.pi, math.pi, 3)
        pts = [(xc + R * math.cos(t), yc + R * math.sin(t)) for t in a]
        got = oracle.circle3(*pts)
        got2 = oracle.circle3(pts[2], pts[0], pts[1])
        for v in (got, got2):
            assert v is not None
            assert abs(v[0] - xc) < 1e-8 * R and abs(v[1] - yc) < 1e-8 * R
            assert abs(v[2] - R) < 1e-8 * R


def test_circle3_of_a_helix_is_its_perigee_circle():
    """Centre of the track circle: P + n / rho with P = d0 n (the perigee
    parametrisation), radius 1 / |rho|."""
    rho, d0, phi0 = 0.004, 1.5, 0.7
    X, Y, _, _, _ = synth.helix_hits(rho, d0, phi0)
    n = np.array([-math.sin(phi0), math.cos(phi0)])
    centre = (d0 + 1.0 / rho) * n
    xc, yc, R = oracle.circle3((X[0], Y[0]), (X[4], Y[4]), (X[9], Y[9]))
    assert abs(xc - centre[0]) < 1e-7 and abs(yc - centre[1]) < 1e-7
    assert abs(R - 1.0 / rho) < 1e-7


# ----------------------------------------------------------- confirmation
def test_clean_tracks_at_cell_centres_are_confirmed_with_all_their_hits():
    """Noise-free helices at cell centres, far apart: the candidate in each
    track's cell is confirmed with one inlier per layer -- exactly the
    track's hits -- and the final assignment gives every hit to it."""
    g = synth.geometry_of("event100_256")
    cells = [(60, 64, 40), (128, 66, 200), (190, 62, 350), (30, 70, 470)]
    x, y, lay, trk = helix_scene(g, cells)
    acc, _ = oracle.vote_layers(g, x, y, lay)
    pk = np.array([[i, j, k, acc[i, j, k]] for (i, j, k) in cells], np.int32)
    score, seeds, inl = oracle.confirm(g, x, y, lay, pk)
    assert list(score) == [10, 10, 10, 10]
    for m in range(4):
        hits = np.flatnonzero(trk == m)
        assert sorted(inl[m][inl[m] >= 0]) == sorted(hits)
        assert all(inl[m, l] == hits[lay[hits] == l][0] for l in range(10))
        assert np.all(inl[m, 10:] == -1)
        assert set(seeds[m]) <= set(hits) and len(set(seeds[m])) == 3
    asg = oracle.confirm_assign(score, inl, x.shape[0])
    assert np.array_equal(asg, trk)
    q = quality.track_quality(g, _Truth(g, cells, x, trk), asg)
    assert q["found"] == 4 and q["fakes"] == 0


class _Truth:
    """Minimal event truth for quality.track_quality on a helix scene."""

    def __init__(self, g, cells, x, trk):
        p = np.array([centre_params(g, *c) for c in cells])
        self.rho, self.d0, self.phi0 = p[:, 0], p[:, 1], p[:, 2]
        self.track = trk
        self.n_track_hits = np.bincount(trk, minlength=len(cells)).astype(np.int32)


def test_seed_layers_are_the_layers_with_one_own_hit():
    """Seeds: innermost and outermost single-hit layers and the one nearest
    their middle.  A second hit in the candidate's cell on a seed layer
    takes that layer out of the seeds; a hit far from the cell changes
    nothing."""
    g = synth.geometry_of("event100_256")
    cell = (120, 66, 100)
    x, y, lay, trk = helix_scene(g, [cell])
    pk = np.array([[*cell, 10]], np.int32)
    score, seeds, inl = oracle.confirm(g, x, y, lay, pk)
    assert list(lay[seeds[0]]) == [0, 5, 9] or list(lay[seeds[0]]) == [0, 4, 9]
    # (la + lc) / 2 = 4.5: layers 4 and 5 tie; the smaller index wins
    assert list(lay[seeds[0]]) == [0, 4, 9]
    # a second own hit on layer 0, 10 um along the layer from the first
    h0 = int(np.flatnonzero(lay == 0)[0])
    ang = math.atan2(y[h0], x[h0]) + 10e-4 / synth.LAYER_R[0]
    x2 = np.append(x, np.float32(synth.LAYER_R[0] * math.cos(ang)))
    y2 = np.append(y, np.float32(synth.LAYER_R[0] * math.sin(ang)))
    l2 = np.append(lay, np.uint8(0))
    s2, seeds2, inl2 = oracle.confirm(g, x2, y2, l2, pk)
    assert list(l2[seeds2[0]]) == [1, 5, 9]
    assert s2[0] == 10
    # a far hit: outside the pool, no change
    x3 = np.append(x, np.float32(-60.0)); y3 = np.append(y, np.float32(-80.0))
    l3 = np.append(lay, np.uint8(3))
    s3, seeds3, inl3 = oracle.confirm(g, x3, y3, l3, pk)
    assert s3[0] == 10 and np.array_equal(seeds3, seeds) and np.array_equal(inl3, inl)


def test_inliers_follow_the_distance_to_the_seed_circle():
    """Moving a non-seed hit across the layer by more than tol drops it
    (score 9); by less than tol keeps it; a noise hit closer to the circle
    than the track's own hit on a layer replaces it."""
    g = synth.geometry_of("event100_256")
    cell = (120, 66, 100)
    x, y, lay, trk = helix_scene(g, [cell])
    pk = np.array([[*cell, 10]], np.int32)
    base, seeds, inl = oracle.confirm(g, x, y, lay, pk)
    h = int(np.flatnonzero(lay == 7)[0])
    r = synth.LAYER_R[7]
    a = math.atan2(y[h], x[h])
    for shift, expect in ((0.03, 9), (0.004, 10)):
        xs, ys = x.copy(), y.copy()
        xs[h] = np.float32(r * math.cos(a + shift / r))
        ys[h] = np.float32(r * math.sin(a + shift / r))
        s, _, i2 = oracle.confirm(g, xs, ys, lay, pk)
        assert s[0] == expect
    # a hit 1 um from the track's layer-7 hit is nearer the circle than...
    # ...a displaced copy: the nearer one is taken
    xs = np.append(x, np.float32(r * math.cos(a + 0.006 / r)))
    ys = np.append(y, np.float32(r * math.sin(a + 0.006 / r)))
    ls = np.append(lay, np.uint8(7))
    s, _, i2 = oracle.confirm(g, xs, ys, ls, pk)
    assert s[0] == 10 and i2[0, 7] == h
    xs[h], ys[h] = np.float32(r * math.cos(a + 0.008 / r)), np.float32(r * math.sin(a + 0.008 / r))
    s, _, i2 = oracle.confirm(g, xs, ys, ls, pk)
    assert i2[0, 7] == len(x)


def test_confirmation_threshold_and_degenerate_candidates():
    g = synth.geometry_of("event100_256")
    cell = (120, 66, 100)
    x, y, lay, trk = helix_scene(g, [cell])
    pk = np.array([[*cell, 10]], np.int32)
    keep = lay < 7                                   # seven layers only
    s, seeds, inl = oracle.confirm(g, x[keep], y[keep], lay[keep], pk)
    assert s[0] == 0 and np.all(inl == -1)           # below min_layers = 8
    s, seeds, inl = oracle.confirm(g, x[keep], y[keep], lay[keep], pk, cp=dict(min_layers=7))
    assert s[0] == 7
    two = lay <= 1                                   # two layers: no seed triple
    s, seeds, inl = oracle.confirm(g, x[two], y[two], lay[two], pk, cp=dict(min_layers=1))
    assert s[0] == 0 and np.all(seeds == -1)
    # an empty event and an empty candidate list
    s, seeds, inl = oracle.confirm(g, x[:0], y[:0], lay[:0], pk)
    assert s[0] == 0
    s, seeds, inl = oracle.confirm(g, x, y, lay, np.zeros((0, 4), np.int32))
    assert s.shape == (0,)


def test_confirmation_is_covariant_under_rotation_by_whole_columns():
    """Rotating every hit by an exact multiple of the column width moves each
    candidate's result to the rotated column (up to hits whose bins move
    across an edge by rounding, absent here: noise-free centre helices)."""
    g = synth.geometry_of("event100_256")
    NP = g["n_phi0"]
    cells = [(60, 64, 40), (128, 66, 200)]
    shift = 37
    x, y, lay, trk = helix_scene(g, cells)
    rot = [(i, j, (k + shift) % NP) for (i, j, k) in cells]
    xr, yr, lr, tr = helix_scene(g, rot)
    pk = np.array([[*c, 10] for c in cells], np.int32)
    pkr = np.array([[*c, 10] for c in rot], np.int32)
    a = oracle.confirm(g, x, y, lay, pk)
    b = oracle.confirm(g, xr, yr, lr, pkr)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[2], b[2])        # same hit order in both scenes


def test_final_assignment_prefers_the_larger_score_then_the_smaller_index():
    score = np.array([9, 10, 9, 0], np.int32)
    inl = np.full((4, 16), -1, np.int32)
    inl[0, :3] = [0, 1, 2]
    inl[1, :2] = [1, 3]
    inl[2, :2] = [2, 4]
    inl[3, :2] = [4, 5]      # not confirmed: ignored
    asg = oracle.confirm_assign(score, inl, 7)
    assert list(asg) == [0, 1, 0, 1, 2, -1, -1]


def test_final_assignment_by_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(20):
        npk, n = 30, 40
        score = rng.integers(0, 4, npk).astype(np.int32) * rng.integers(0, 2, npk).astype(np.int32)
        inl = np.where(rng.random((npk, 16)) < 0.3, rng.integers(0, n, (npk, 16)), -1).astype(np.int32)
        asg = oracle.confirm_assign(score, inl, n)
        for h in range(n):
            c = [(-score[m], m) for m in range(npk) if score[m] > 0 and h in inl[m]]
            assert asg[h] == (min(c)[1] if c else -1)


# ----------------------------------------------------------- planted mistakes
def _confirm_py(g, x, y, lay, cell, tol=0.01, pool=4, min_layers=8, seed_rule="one",
                strict=True):
    """The confirmation rule restated in numpy, with switches that plant a
    mistake; used only to show the properties above catch each one."""
    _, sn, cs, rho = oracle.tables(g)
    i, j, k = cell
    delta = 2 * g["d0_half"] / g["n_d0"]
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    s = xd * sn[k] - yd * cs[k]
    c = xd * cs[k] + yd * sn[k]
    b = 1 + rho[i] * s
    D = 1 - (rho[i] * c) ** 2
    sq = np.sqrt(np.maximum(D, 0))
    q = -(b + np.where(b >= 0, sq, -sq))
    u = (q / rho[i]) / delta + g["n_d0"] / 2 + 0.5
    u2 = ((rho[i] * (xd * xd + yd * yd) + 2 * s) / q) / delta + g["n_d0"] / 2 + 0.5
    ok = (c > 0) & (D >= 0)
    bins = [np.where(ok & (v >= 0) & (v < g["n_d0"]), np.floor(v), -99) for v in (u, u2)]
    own = (bins[0] == j) | (bins[1] == j)
    inpool = (np.abs(bins[0] - j) <= pool) | (np.abs(bins[1] - j) <= pool)
    n_own = np.bincount(lay[own], minlength=16)
    sl = [l for l in range(10) if (n_own[l] == 1 if seed_rule == "one" else n_own[l] >= 1)]
    if len(sl) < 3:
        return 0
    la, lc = sl[0], sl[-1]
    lb = min(sl[1:-1], key=lambda l: (abs(2 * l - la - lc), l))
    hs = [int(np.flatnonzero(own & (lay == l))[0]) for l in (la, lb, lc)]
    cir = oracle.circle3(*[(xd[h], yd[h]) for h in hs])
    d = np.abs(np.hypot(xd - cir[0], yd - cir[1]) - cir[2])
    sc = 0
    for l in range(10):
        mm = inpool & (lay == l)
        if mm.any():
            dm = d[mm].min()
            sc += (dm < tol) if strict else (dm <= tol)
    return sc if sc >= min_layers else 0


def test_planted_mistakes_fail_the_pins():
    g = synth.geometry_of("event100_256")
    cell = (120, 66, 100)
    x, y, lay, trk = helix_scene(g, [cell])
    assert _confirm_py(g, x, y, lay, cell) == 10          # the rule as stated
    # mistake 1: seed layers with any number of own hits (a second own hit
    # on layer 0, 800 um along the layer -- still in the cell's d0 bin --
    # becomes a seed and bends the circle away from the inner layers)
    h0 = int(np.flatnonzero(lay == 0)[0])
    ang = math.atan2(y[h0], x[h0]) + 800e-4 / synth.LAYER_R[0]
    x2 = np.insert(x, 0, np.float32(synth.LAYER_R[0] * math.cos(ang)))
    y2 = np.insert(y, 0, np.float32(synth.LAYER_R[0] * math.sin(ang)))
    l2 = np.insert(lay, 0, np.uint8(0))
    pk = np.array([[*cell, 10]], np.int32)
    good = oracle.confirm(g, x2, y2, l2, pk)[0][0]
    assert good == 10
    assert _confirm_py(g, x2, y2, l2, cell, seed_rule="any") != good
    # mistake 2: a pool of zero bins (own hits only) loses the outer hits of
    # a track 2 mrad off the column centre: its roots drift by ~0.002 r, so
    # layers 0-6 stay in the cell's bin and layers 7-9 fall in the next one
    rho, d0, phi0 = centre_params(g, *cell)
    X, Y, _, L, _ = synth.helix_hits(rho, d0, phi0 + 0.002)
    xo, yo, lo = X.astype(np.float32), Y.astype(np.float32), L.astype(np.uint8)
    full = oracle.confirm(g, xo, yo, lo, pk, cp=dict(min_layers=3))[0][0]
    assert full == 10
    assert _confirm_py(g, xo, yo, lo, cell, min_layers=3) == full
    assert _confirm_py(g, xo, yo, lo, cell, pool=0, min_layers=3) == 7


