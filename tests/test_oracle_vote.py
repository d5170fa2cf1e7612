"""Pins of the oracle's Hough vote (Section 5) against what the method fixes.

Every check here reaches the answer by a route other than the oracle's own
floating-point root formula: exact rational arithmetic, track geometry,
the textbook straight-line transform, symmetry.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def small_geom(**kw):
    g = dict(n_rho=8, n_d0=8, n_phi0=16, rho_max=0.04, d0_half=10.0, n_z0=16,
             n_cot=16, z0_max=32.0, cot_max=6.5, threshold=3, count_bits=32)
    g.update(kw)
    return g


def _roots_below(rho, bq, Cq, e):
    """Number of roots of rho d^2 + 2 bq d + Cq strictly below e (exact)."""
    if rho == 0:
        root = -Cq / (2 * bq)
        return 1 if root < e else 0
    disc = bq * bq - rho * Cq
    if disc < 0:
        return 0
    v = -bq / rho
    if disc == 0:
        return 1 if v < e else 0
    F = rho * e * e + 2 * bq * e + Cq
    sF = F if rho > 0 else -F
    if e <= v:
        return 1 if sF < 0 else 0
    return 2 if sF > 0 else 1


def exact_hit_acc(g, xf, yf):
    """Per-hit accumulator by exact rational root counting in each d0 bin."""
    _, sn, cs, rho = oracle.tables(g)
    ND = g["n_d0"]
    delta = Fraction(2.0 * g["d0_half"] / ND)
    off = Fraction(ND * 0.5 + 0.5)
    acc = np.zeros((g["n_rho"], ND, g["n_phi0"]), np.int64)
    X, Y = Fraction(float(xf)), Fraction(float(yf))
    edges = [(j - off) * delta for j in range(ND + 1)]
    for k in range(g["n_phi0"]):
        S, Cc = Fraction(sn[k]), Fraction(cs[k])
        s = X * S - Y * Cc
        c = X * Cc + Y * S
        if not c > 0:
            continue
        r2 = X * X + Y * Y
        for i in range(g["n_rho"]):
            R = Fraction(rho[i])
            bq = 1 + R * s
            Cq = R * r2 + 2 * s
            below = [_roots_below(R, bq, Cq, e) for e in edges]
            for j in range(ND):
                acc[i, j, k] += below[j + 1] - below[j]
    return acc


@pytest.mark.parametrize("seed", [1, 2])
def test_vote_matches_exact_root_counting(seed):
    """Brute force: every cell of every hit, roots counted in exact arithmetic."""
    rng = np.random.default_rng(seed)
    g = small_geom()
    n = 12
    r = rng.uniform(3.0, 70.0, n)
    ph = rng.uniform(-math.pi, math.pi, n)
    x = (r * np.cos(ph)).astype(np.float32)
    y = (r * np.sin(ph)).astype(np.float32)
    total = 0
    for h in range(n):
        acc, st = oracle.vote(g, x[h:h + 1], y[h:h + 1], threads=1)
        ex = exact_hit_acc(g, x[h], y[h])
        assert np.array_equal(acc, ex), f"hit {h}"
        assert st["votes"] == int(ex.sum())
        total += int(ex.sum())
    assert total > 0


def test_vote_includes_branch_b_roots():
    """A hit past a quarter turn votes through the second root (exact check)."""
    g = small_geom(rho_max=0.05, n_rho=8, d0_half=10.0)
    _, sn, cs, rho = oracle.tables(g)
    i, k, j = 7, 5, 3                        # rho_7 > 0, a d0 bin centre
    delta = 2 * g["d0_half"] / g["n_d0"]
    d0c = (j - g["n_d0"] / 2) * delta
    phi0 = (2 * k + 1 - g["n_phi0"]) * math.pi / g["n_phi0"]
    X, Y, Z, lay, L = synth.helix_hits(rho[i], d0c, phi0, radii=[20.0, 35.0, 40.0])
    theta = rho[i] * L
    assert np.any(np.abs(theta) > math.pi / 2), "scene must include a branch-B hit"
    for xh, yh, th in zip(X, Y, theta):
        xf, yf = np.float32(xh), np.float32(yh)
        acc, _ = oracle.vote(g, [xf], [yf], threads=1)
        assert acc[i, j, k] >= 1, f"hit at theta={th} misses its own cell"
        assert np.array_equal(acc, exact_hit_acc(g, xf, yf))


@pytest.mark.parametrize("name", ["single_64", "event100_256", "pileup_512"])
@pytest.mark.parametrize("branch", ["A", "B"])
def test_helix_at_centres_peaks_in_true_cell(name, branch):
    """Noise-free hits of a track at cell centres put the maximum in its cell."""
    g = synth.geometry_of(name)
    _, sn, cs, rho = oracle.tables(g)
    ND = g["n_d0"]
    delta = 2 * g["d0_half"] / ND
    if branch == "A":
        i, j, k = g["n_rho"] // 3, ND // 2 + 3, g["n_phi0"] // 5
        radii = synth.LAYER_R
    else:
        # the highest-curvature row, so that outer hits lie past a quarter turn
        i, j, k = g["n_rho"] - 1, ND // 2 - 2, g["n_phi0"] // 3
        radii = synth.LAYER_R
    d0c = (j - ND / 2) * delta
    phi0 = (2 * k + 1 - g["n_phi0"]) * math.pi / g["n_phi0"]
    X, Y, Z, lay, L = synth.helix_hits(rho[i], d0c, phi0, radii=radii)
    theta = np.abs(rho[i] * L)
    if branch == "B" and not np.any(theta > math.pi / 2):
        # only the widest curvature range turns past a quarter turn in 110 cm
        assert name != "pileup_512"
        pytest.skip("no hit past a quarter turn at this curvature range")
    x, y = X.astype(np.float32), Y.astype(np.float32)
    # restrict the accumulator to a window of rows around the true one
    acc, st = oracle.vote(g, x, y)
    assert acc[i, j, k] == len(x)
    assert acc.max() == len(x)


def test_one_vote_per_phi0_column_per_valid_branch():
    """Each hit gives each column (rho_i, phi0_k) 0, 1 or 2 votes; only c > 0."""
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 3)
    phi0, _, _, _ = oracle.tables(g)
    for h in range(0, ev.n_hits, 37):
        acc, st = oracle.vote(g, ev.x[h:h + 1], ev.y[h:h + 1], threads=1)
        per_col = acc.sum(axis=1)              # [rho, phi0]
        assert per_col.max() <= 2
        assert int(acc.sum()) == st["votes"]
        phh = math.atan2(float(ev.y[h]), float(ev.x[h]))
        backward = np.cos(phi0 - phh) < -1e-9
        assert per_col[:, backward].sum() == 0


def test_rho_zero_is_the_straight_line_transform():
    """n_rho = 1 samples rho = 0: the vote is the normal-form line transform
    d0 = -x sin phi0 + y cos phi0 (Fig. 3's sinusoids).  Scene: 50 straight
    tracks x 10 hits; an independent 10-line routine bins the sinusoids."""
    g = small_geom(n_rho=1, n_d0=64, n_phi0=128, rho_max=0.01, d0_half=20.0)
    rng = np.random.default_rng(7)
    ND, NP = g["n_d0"], g["n_phi0"]
    delta = 2 * g["d0_half"] / ND
    ks = rng.integers(0, NP, 50)
    js = rng.integers(8, ND - 8, 50)
    xs, ys = [], []
    for k, j in zip(ks, js):
        X, Y, *_ = synth.helix_hits(0.0, (j - ND / 2) * delta,
                                    (2 * k + 1 - NP) * math.pi / NP,
                                    radii=np.linspace(20.0, 110.0, 10))
        xs.append(X); ys.append(Y)
    x = np.concatenate(xs).astype(np.float32)
    y = np.concatenate(ys).astype(np.float32)
    assert x.shape[0] == 500
    acc, st = oracle.vote(g, x, y)

    # independent routine: theta = phi0 + pi/2, rho_line = x cos theta + y sin theta
    ref = np.zeros((ND, NP), np.int64)
    th = (2 * np.arange(NP) + 1 - NP) * math.pi / NP + math.pi / 2
    for xh, yh in zip(x.astype(np.float64), y.astype(np.float64)):
        fwd = xh * np.sin(th) - yh * np.cos(th) > 0          # c > 0
        dd = xh * np.cos(th) + yh * np.sin(th)                 # = d0
        u = dd / delta + (ND / 2 + 0.5)
        ok = fwd & (u >= 0) & (u < ND)
        np.add.at(ref, (np.floor(u[ok]).astype(int), np.nonzero(ok)[0]), 1)
    diff = np.abs(acc[0] - ref).sum()
    assert diff <= 2 * st["edge"] + 2
    for k, j in zip(ks, js):
        assert acc[0, j, k] >= 10


def test_rotation_by_whole_columns_rolls_the_accumulator():
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 5)
    m = 7
    a = m * 2 * math.pi / g["n_phi0"]
    x, y = ev.x.astype(np.float64), ev.y.astype(np.float64)
    xr = (x * math.cos(a) - y * math.sin(a)).astype(np.float32)
    yr = (x * math.sin(a) + y * math.cos(a)).astype(np.float32)
    acc, st = oracle.vote(g, ev.x, ev.y)
    accr, str_ = oracle.vote(g, xr, yr)
    rolled = np.roll(acc, m, axis=2)
    mism = np.abs(rolled - accr).sum()
    # fp32 rounding of the rotated hits can only move votes whose bin
    # coordinate lies next to an edge
    assert mism <= 2e-3 * st["votes"]
    assert abs(st["votes"] - str_["votes"]) <= 1e-3 * st["votes"]


def test_uint16_counts_saturate():
    g = small_geom(n_rho=2, n_d0=4, n_phi0=4, count_bits=16)
    n = 70000
    x = np.full(n, 5.0, np.float32)
    y = np.full(n, 1.0, np.float32)
    acc1, _ = oracle.vote(g, x[:1], y[:1], threads=1)
    acc, st = oracle.vote(g, x, y)
    assert st["votes"] == n * int(acc1.sum())
    assert np.array_equal(acc, np.minimum(acc1 * n, 65535))


def test_geometry_tables_cover_the_axes():
    g = synth.geometry_of("event100_256")
    phi0, sn, cs, rho = oracle.tables(g)
    step = 2 * math.pi / g["n_phi0"]
    assert abs(phi0[0] + math.pi - step / 2) < 1e-12
    assert abs(phi0[-1] - math.pi + step / 2) < 1e-12
    assert np.allclose(np.diff(phi0), step, atol=1e-12)
    assert np.allclose(sn ** 2 + cs ** 2, 1.0, atol=1e-15)
    assert abs(rho[-1] - g["rho_max"] * (1 - 1 / g["n_rho"])) < 1e-15
    assert np.allclose(rho, -rho[::-1], atol=0)
