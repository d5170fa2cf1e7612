"""Pins of the oracle's hit association and (z0, cot theta) vote."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_atan2_against_libm():
    rng = np.random.default_rng(0)
    y = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-6, 2000),
                        [0.0, 1.0, 0.0, -1.0, 1.0, -3.0, 1e-300, 1.0]])
    x = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e3, 2000),
                        [1.0, 0.0, -1.0, 0.0, 1.0, -3.0, 1.0, 1e-300]])
    ours = oracle.atan2(y, x)
    ref = np.arctan2(y, x)
    err = np.abs(ours - ref)
    assert np.all(err <= 8 * np.spacing(np.abs(ref)) + 1e-320)
    assert ours[-8] == 0.0 and ours[-6] == math.pi
    assert ours[-7] == math.pi / 2 and ours[-5] == -math.pi / 2


def _vote_cells(g, xf, yf):
    acc, _ = oracle.vote(g, [xf], [yf], threads=1)
    return np.argwhere(acc > 0)


def brute_assign(g, x, y, pk):
    """Compatibility from each hit's full vote set (the vote, not the
    association's own 9-column evaluation), then the best-count rule."""
    NP = g["n_phi0"]
    out = np.full(x.shape[0], -1, np.int32)
    for h in range(x.shape[0]):
        cells = _vote_cells(g, x[h], y[h])
        best, bc = -1, -1
        for m, (im, jm, km, cm) in enumerate(pk):
            if cells.shape[0] == 0:
                break
            dk = np.abs(cells[:, 2] - km)
            dk = np.minimum(dk, NP - dk)
            hit = ((np.abs(cells[:, 0] - im) <= 1) & (np.abs(cells[:, 1] - jm) <= 1)
                   & (dk <= 1))
            if hit.any() and cm > bc:
                best, bc = m, cm
        out[h] = best
    return out


def test_association_matches_vote_set_brute_force():
    g = synth.geometry_of("single_64", threshold=4)
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 1)
    acc, _ = oracle.vote(g, ev.x, ev.y)
    pk, cnt = oracle.peaks(g, acc)
    assert cnt > 10
    sel = np.arange(0, ev.n_hits, 3)
    asg = oracle.associate(g, ev.x, ev.y, pk, hit_idx=sel)
    ref = brute_assign(g, ev.x[sel], ev.y[sel], pk)
    assert np.array_equal(asg, ref)
    assert (asg >= 0).sum() > 0


def test_hits_of_tracks_at_centres_go_to_their_track():
    g = synth.geometry_of("single_64")
    _, sn, cs, rho = oracle.tables(g)
    ND, NP = g["n_d0"], g["n_phi0"]
    delta = 2 * g["d0_half"] / ND
    cells = [(20, 34, 5), (44, 30, 21), (10, 32, 40), (52, 33, 58)]
    xs, ys, owner = [], [], []
    for t, (i, j, k) in enumerate(cells):
        X, Y, *_ = synth.helix_hits(rho[i], (j - ND / 2) * delta,
                                    (2 * k + 1 - NP) * math.pi / NP)
        xs.append(X); ys.append(Y); owner += [t] * len(X)
    x = np.concatenate(xs).astype(np.float32)
    y = np.concatenate(ys).astype(np.float32)
    acc, _ = oracle.vote(g, x, y)
    pk, _ = oracle.peaks(g, acc)
    asg = oracle.associate(g, x, y, pk)
    true_m = [int(np.nonzero((pk[:, 0] == i) & (pk[:, 1] == j) & (pk[:, 2] == k))[0][0])
              for (i, j, k) in cells]
    assert [pk[m, 3] for m in true_m] == [10, 10, 10, 10]
    assert all(asg[h] == true_m[owner[h]] for h in range(x.shape[0]))


def _z_geom():
    return synth.geometry_of("event100_256")


@pytest.mark.parametrize("cell,zq", [((100, 70, 300), (60, 70)),
                                     ((200, 60, 17), (75, 30)),
                                     ((127, 64, 256), (64, 64))])
def test_z_vote_of_a_helix_at_centres(cell, zq):
    """A track with (rho, d0, phi0, z0, cot theta) all at bin centres puts all
    its hits in its own (z0, cot theta) cell."""
    g = _z_geom()
    _, sn, cs, rho = oracle.tables(g)
    ND, NP, NZ, NC = g["n_d0"], g["n_phi0"], g["n_z0"], g["n_cot"]
    i, j, k = cell
    nz, q = zq
    dz = 2 * g["z0_max"] / NZ
    z0 = (nz + 0.5) * dz - g["z0_max"]
    cot = (2 * q + 1 - NC) * g["cot_max"] / NC
    X, Y, Z, lay, L = synth.helix_hits(rho[i], (j - ND / 2) * 2 * g["d0_half"] / ND,
                                       (2 * k + 1 - NP) * math.pi / NP, z0, cot)
    x, y, z = (a.astype(np.float32) for a in (X, Y, Z))
    pk = np.array([[i, j, k, len(x)]], np.int32)
    asg = np.zeros(len(x), np.int32)
    zr = oracle.vote_z(g, x, y, z, asg, pk)
    assert zr.tolist() == [[nz, q, len(x)]]


def test_z_vote_matches_independent_histogram():
    """Independent route: libm atan2 and numpy histogramming, away from edges."""
    g = _z_geom()
    _, sn, cs, rho = oracle.tables(g)
    rng = np.random.default_rng(3)
    ND, NZ, NC = g["n_d0"], g["n_z0"], g["n_cot"]
    delta = 2 * g["d0_half"] / ND
    dz = 2 * g["z0_max"] / NZ
    pk = np.array([[30, 60, 100, 9], [240, 70, 400, 9], [128, 64, 3, 9]], np.int32)
    n = 300
    r = rng.uniform(4, 110, n); ph = rng.uniform(-math.pi, math.pi, n)
    x = (r * np.cos(ph)).astype(np.float32); y = (r * np.sin(ph)).astype(np.float32)
    z = rng.uniform(-40, 40, n).astype(np.float32)
    asg = rng.integers(-1, 3, n).astype(np.int32)
    zr = oracle.vote_z(g, x, y, z, asg, pk)
    tq = (2 * np.arange(NC) + 1 - NC) * g["cot_max"] / NC
    for m, (i, j, k, _) in enumerate(pk):
        hs = np.nonzero(asg == m)[0]
        phi0 = (2 * k + 1 - g["n_phi0"]) * math.pi / g["n_phi0"]
        xd, yd, zd = (a[hs].astype(np.float64) for a in (x, y, z))
        s = xd * math.sin(phi0) - yd * math.cos(phi0)
        c = xd * math.cos(phi0) + yd * math.sin(phi0)
        d0c = (j - ND / 2) * delta
        L = np.arctan2(rho[i] * c, 1 + rho[i] * (s + d0c)) / rho[i]
        u = (zd[:, None] - L[:, None] * tq[None, :] + g["z0_max"]) / dz
        frac = u - np.floor(u)
        assert np.all(np.minimum(frac, 1 - frac) > 1e-9)
        hist = np.zeros((NZ, NC), np.int64)
        ok = (u >= 0) & (u < NZ)
        qq = np.broadcast_to(np.arange(NC), u.shape)
        np.add.at(hist, (np.floor(u[ok]).astype(int), qq[ok]), 1)
        b = int(np.argmax(hist))
        assert zr[m].tolist() == [b // NC, b % NC, int(hist.max())]


def test_z_vote_without_hits_is_empty():
    g = _z_geom()
    pk = np.array([[3, 3, 3, 7]], np.int32)
    zr = oracle.vote_z(g, np.zeros(2, np.float32), np.ones(2, np.float32),
                       np.zeros(2, np.float32), np.array([-1, -1], np.int32), pk)
    assert zr.tolist() == [[-1, -1, 0]]


def test_z_vote_of_a_straight_track():
    """rho = 0 row (odd n_rho): the arc length is the distance along the line."""
    g = synth.geometry_of("event100_256", n_rho=1)
    NP, NZ, NC, ND = g["n_phi0"], g["n_z0"], g["n_cot"], g["n_d0"]
    i, j, k, nz, q = 0, ND // 2 + 5, 77, 50, 90
    dz = 2 * g["z0_max"] / NZ
    z0 = (nz + 0.5) * dz - g["z0_max"]
    cot = (2 * q + 1 - NC) * g["cot_max"] / NC
    X, Y, Z, lay, L = synth.helix_hits(0.0, (j - ND / 2) * 2 * g["d0_half"] / ND,
                                       (2 * k + 1 - NP) * math.pi / NP, z0, cot)
    x, y, z = (a.astype(np.float32) for a in (X, Y, Z))
    zr = oracle.vote_z(g, x, y, z, np.zeros(len(x), np.int32),
                       np.array([[i, j, k, len(x)]], np.int32))
    assert zr.tolist() == [[nz, q, len(x)]]


@pytest.mark.parametrize("name,stride", [("single_64", 1), ("event100_256", 400)])
def test_dense_association_route_agrees(name, stride):
    """The full-size route (each hit's votes against a cell -> candidate map)
    and the per-candidate 9-column route give the same assignment."""
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 2)
    acc, _ = oracle.vote(g, ev.x, ev.y)
    pk, _ = oracle.peaks(g, acc)
    sel = np.arange(0, ev.n_hits, stride)
    a = oracle.associate(g, ev.x, ev.y, pk, hit_idx=sel)
    b = oracle.associate_dense(g, ev.x, ev.y, pk, hit_idx=sel)
    assert np.array_equal(a, b)
    assert (a >= 0).mean() > 0.2
