"""Pins of the candidate-refinement oracle (oracle/fit.py)."""
import math

import numpy as np

import synth
from oracle import fit as F


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-80, 80, 20), rng.uniform(-80, 80, 20)
    p = np.array([0.004, 1.3, 0.7])
    _, J = F.residuals(p, x, y)
    for a in range(3):
        h = [1e-9, 1e-7, 1e-8][a]
        e = np.zeros(3); e[a] = h
        fd = (F.residuals(p + e, x, y)[0] - F.residuals(p - e, x, y)[0]) / (2 * h)
        assert np.allclose(J[:, a], fd, rtol=1e-5, atol=1e-6)


def test_residual_is_the_distance_to_the_circle():
    # points at distance eps from the circle (along the radius) give F/2 ~ eps
    rho, d0, phi0 = 0.01, 2.0, -0.4
    n = np.array([-math.sin(phi0), math.cos(phi0)])
    C = (d0 + 1 / rho) * n
    ang = np.linspace(0.1, 1.0, 9)
    for eps in (1e-3, -2e-3):
        R = 1 / rho + eps
        pts = C[None, :] + R * np.stack([np.cos(ang), np.sin(ang)], 1)
        r, _ = F.residuals((rho, d0, phi0), pts[:, 0], pts[:, 1])
        # F = rho (|X - C|^2 - R0^2) = eps (2 + rho eps) for rho > 0
        assert np.allclose(r, eps * (1 + 0.5 * rho * eps), rtol=1e-9)


def test_noise_free_helices_are_recovered_from_a_cell_centre_start():
    for rho, d0, phi0 in [(0.0071, 0.0, 1.1), (-0.0102, 3.7, -2.9), (0.0005, -8.2, 0.3),
                          (-0.003, 12.5, 2.0)]:
        hx, hy, _, _, _ = synth.helix_hits(rho, d0, phi0)
        start = (rho + 4.4e-5, d0 - 0.15, phi0 + 0.006)       # half a cell away
        p, chi2, _, st = F.fit_one(start, hx, hy, iters=6)
        assert st == 1
        assert abs(p[0] - rho) < 1e-12 and abs(p[1] - d0) < 1e-9
        assert abs(math.remainder(p[2] - phi0, 2 * math.pi)) < 1e-11
        assert chi2 < 1e-12


def test_chi2_and_pulls_follow_the_hit_resolution():
    rng = np.random.default_rng(3)
    sig = 20e-4
    chi2s, pulls = [], []
    for t in range(300):
        rho = rng.uniform(-0.01, 0.01)
        d0 = rng.uniform(-5, 5)
        phi0 = rng.uniform(-math.pi, math.pi)
        hx, hy, _, lay, _ = synth.helix_hits(rho, d0, phi0)
        if hx.shape[0] < 6:
            continue
        # smear along the layer (radius kept), as the generator does
        r = np.hypot(hx, hy)
        ph = np.arctan2(hy, hx) + rng.normal(0, sig, hx.shape[0]) / r
        x, y = r * np.cos(ph), r * np.sin(ph)
        p, chi2, cov, _ = F.fit_one((rho, d0, phi0), x, y, iters=5, sigma=sig)
        chi2s.append(chi2 / (x.shape[0] - 3))
        pulls.append((p[1] - d0) / math.sqrt(cov[1, 1]))
    # smearing along the layer is not perpendicular to the track, so chi2/dof
    # sits a little below 1; pulls of d0 have unit width
    assert 0.5 < np.mean(chi2s) < 1.2
    assert 0.8 < np.std(pulls) < 1.25 and abs(np.mean(pulls)) < 0.2


def test_cholesky_and_degenerate_tracks():
    A = np.array([[4.0, 2.0, 0.4], [2.0, 5.0, 1.0], [0.4, 1.0, 3.0]])
    L = F.cholesky3(A)
    assert np.allclose(L @ L.T, A, rtol=1e-14) and np.allclose(L, np.linalg.cholesky(A))
    assert F.cholesky3(np.diag([1.0, 0.0, 1.0])) is None
    # two distinct points cannot fix three parameters: singular normal matrix
    p, chi2, cov, st = F.fit_one((0.001, 0.0, 0.5), [10.0, 10.0, 20.0], [5.0, 5.0, 10.0])
    assert st == -1


def test_fit_candidates_selects_by_hit_count():
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 1)
    import oracle
    r = oracle.run_event(g, ev.x, ev.y, ev.z)
    out = F.fit_candidates(g, ev.x, ev.y, r["assign"], r["peaks"], min_hits=4)
    n_ass = np.bincount(r["assign"][r["assign"] >= 0], minlength=len(r["peaks"]))
    for m, f in enumerate(out):
        assert (f is None) == (n_ass[m] < 4)
        if f is not None:
            assert f["n"] == n_ass[m] and f["status"] in (1, -1)


def test_road_and_cut_drop_foreign_hits():
    """A track's hits plus hits of a crossing track: without selection the fit
    is pulled away; the road and the cut keep exactly the track's hits."""
    g = synth.geometry_of("event100_256")
    import oracle
    phi_t, _, _, rho_t = oracle.tables(g)
    delta = 2 * g["d0_half"] / g["n_d0"]
    i, j, k = 180, 66, 300
    rho, d0, phi0 = rho_t[i] + 1e-5, (j - 64) * delta + 0.05, phi_t[k] - 0.002
    hx, hy, _, _, _ = synth.helix_hits(rho, d0, phi0)
    ox, oy, _, _, _ = synth.helix_hits(-0.004, 6.0, phi0 + 0.3)
    x = np.concatenate([hx, ox[:4]]); y = np.concatenate([hy, oy[:4]])
    assign = np.zeros(x.shape[0], np.int32)
    pk = np.array([[i, j, k, 10]], np.int32)
    plain = F.fit_candidates(g, x, y, assign, pk)[0]
    sel = F.fit_candidates(g, x, y, assign, pk, road=1.0, cut=5.0)[0]
    assert sel["n"] == hx.shape[0] and sel["status"] == 1
    assert abs(sel["p"][1] - d0) < 1e-9 and abs(sel["p"][0] - rho) < 1e-12
    assert abs(plain["p"][1] - d0) > 1e-3
