"""Pins of the swept-interval vote's oracle (oracle vote_swept): it contains
the point vote, it equals a dense-sampling brute force of the continuous
curve wherever the curve stays in its domain across a column, the
straight-line case matches the closed form, and it tends to the point vote
as the phi0 bins shrink."""
import math

import numpy as np

import oracle
import synth


def geom(**kw):
    g = dict(n_rho=16, n_d0=64, n_phi0=32, rho_max=0.008, d0_half=10.0, n_z0=8, n_cot=8,
             z0_max=32.0, cot_max=6.5, threshold=7, count_bits=32)
    g.update(kw)
    return g


def hits(n, seed, rmax=100.0):
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], seed)
    r = np.hypot(ev.x, ev.y)
    keep = r < rmax
    return ev.x[keep][:n], ev.y[keep][:n]


def test_swept_contains_the_point_vote_hit_by_hit():
    g = geom()
    x, y = hits(40, 1)
    for h in range(len(x)):
        a, _ = oracle.vote(g, x[h:h + 1], y[h:h + 1], threads=1)
        b, st = oracle.vote_swept(g, x[h:h + 1], y[h:h + 1], threads=1)
        assert np.all(b <= 1)
        assert np.all(b[a > 0] == 1)
        assert st["votes"] == int(b.sum())


def dense_bins(g, x, y, rho, e0, e1, n=4001):
    """d0 bins the continuous roots reach for phi in [e0, e1] (dense grid,
    the textbook quadratic formula, float64), or None if c <= 0 or D < 0
    somewhere on the grid."""
    phi = np.linspace(e0, e1, n)
    s = x * np.sin(phi) - y * np.cos(phi)
    c = x * np.cos(phi) + y * np.sin(phi)
    D = 1.0 - (rho * c) ** 2
    if np.any(c <= 0) or np.any(D < 0):
        return None
    delta = 2 * g["d0_half"] / g["n_d0"]
    out = set()
    roots = [(-(1 + rho * s) + np.sqrt(D)) / rho, (-(1 + rho * s) - np.sqrt(D)) / rho] \
        if rho != 0 else [-s]
    for d0 in roots:
        u = d0 / delta + g["n_d0"] / 2 + 0.5
        ok = (u >= 0) & (u < g["n_d0"])
        out |= set(np.floor(u[ok]).astype(int).tolist())
    return out


def test_swept_equals_dense_sampling_where_the_curve_stays_in_its_domain():
    g = geom()
    assert g["rho_max"] * 100.0 < 1.0          # D > 0 for every hit below 100 cm
    x, y = hits(12, 2)
    phi0, _, _, rho = oracle.tables(g)
    N = g["n_phi0"]
    n_cmp = 0
    for h in range(len(x)):
        b, _ = oracle.vote_swept(g, x[h:h + 1], y[h:h + 1], threads=1)
        for i in (1, 5, 10, 14):
            for k in range(N):
                e0 = (2 * k - N) * math.pi / N
                want = dense_bins(g, float(np.float64(x[h])), float(np.float64(y[h])), rho[i],
                                  e0, e0 + 2 * math.pi / N)
                if want is None:
                    continue
                got = set(np.flatnonzero(b[i, :, k]).tolist())
                assert got == want, (h, i, k, sorted(got), sorted(want))
                n_cmp += 1
    assert n_cmp > 500


def test_straight_line_columns_by_closed_form():
    """rho = 0 (n_rho = 1): d0 = -s = r sin(psi - phi); for a hit at (50, 0)
    column k sweeps the bins between -50 sin(e_k) and -50 sin(e_k+1)."""
    g = geom(n_rho=1, n_phi0=16, n_d0=40, d0_half=60.0)
    b, _ = oracle.vote_swept(g, np.array([50.0], np.float32), np.array([0.0], np.float32))
    N, ND = g["n_phi0"], g["n_d0"]
    delta = 2 * g["d0_half"] / ND
    for k in range(N):
        e0, e1 = (2 * k - N) * math.pi / N, (2 * k + 2 - N) * math.pi / N
        if not (math.cos(e0) > 0 and math.cos(e1) > 0):
            continue
        u0 = -50 * math.sin(e0) / delta + ND / 2 + 0.5
        u1 = -50 * math.sin(e1) / delta + ND / 2 + 0.5
        lo, hi = sorted((math.floor(u0), math.floor(u1)))
        want = set(range(max(lo, 0), min(hi, ND - 1) + 1))
        assert set(np.flatnonzero(b[0, :, k]).tolist()) == want, k


def test_swept_tends_to_the_point_vote_for_fine_phi0_bins():
    x, y = hits(30, 3)
    ratios = []
    for n_phi0 in (32, 256, 2048):
        g = geom(n_phi0=n_phi0)
        _, a = oracle.vote(g, x, y)
        _, b = oracle.vote_swept(g, x, y)
        ratios.append(b["votes"] / a["votes"])
    assert ratios[0] > ratios[1] > ratios[2] >= 1.0
    assert ratios[2] < 1.5


def test_edge_tables_are_the_column_edges():
    g = geom(n_phi0=12)
    sn, cs = oracle.edge_tables(g)
    phi0, s0, c0, _ = oracle.tables(g)
    e = np.arctan2(sn, cs)
    N = g["n_phi0"]
    assert np.allclose(np.angle(np.exp(1j * (e + math.pi / N - phi0))), 0.0, atol=1e-14)
    assert np.allclose(sn ** 2 + cs ** 2, 1.0, atol=1e-15)
