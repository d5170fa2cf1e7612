"""Pins of the second-transform oracle (oracle/vertex.py)."""
import math

import numpy as np

import synth
from oracle import vertex as V

G = synth.geometry_of("jets4_256")
VD = dict(n_r=16, n_theta=64, r_max=32.0, threshold=3, min_count=0, r_keep=3.0)


def _single(j, k, vd=VD, g=G):
    return V.vote(g, vd, np.array([[0, j, k, 9]], np.int32))[0]


def test_votes_are_line_ray_intersections():
    """Each vote equals the intersection of the candidate's line with the
    ray at theta_q, found by a 2 x 2 linear solve (not the sine formula)."""
    rng = np.random.default_rng(0)
    ND, NP = G["n_d0"], G["n_phi0"]
    delta = 2 * G["d0_half"] / ND
    th, _, _ = V.theta_tables(VD["n_theta"])
    dr = VD["r_max"] / VD["n_r"]
    checked = 0
    for _ in range(60):
        j, k = int(rng.integers(0, ND)), int(rng.integers(0, NP))
        acc = _single(j, k)
        d0 = (j - ND / 2) * delta
        phi0 = (2 * k + 1 - NP) * math.pi / NP
        P = d0 * np.array([-math.sin(phi0), math.cos(phi0)])
        t = np.array([math.cos(phi0), math.sin(phi0)])
        for q, tq in enumerate(th):
            w = np.array([math.cos(tq), math.sin(tq)])
            M = np.stack([t, -w], 1)
            if abs(np.linalg.det(M)) < 1e-12:
                continue
            lam, mu = np.linalg.solve(M, -P)
            u = mu / dr
            col = acc[:, q]
            if abs(u - round(u)) < 1e-9 or abs(u) < 1e-9:
                continue                           # on an edge: either answer
            if 0 <= u < VD["n_r"]:
                assert col.sum() == 1 and col[int(math.floor(u))] == 1, (j, k, q, u)
            else:
                assert col.sum() == 0, (j, k, q, u)
            checked += 1
    assert checked > 1000


def test_prompt_candidate_votes_in_bin_zero_everywhere():
    acc = _single(G["n_d0"] // 2, 17)
    assert (acc[0] == 1).all() and acc[1:].sum() == 0


def test_lines_through_a_vertex_meet_in_its_cell():
    """Candidates chosen as the cells nearest to lines through a vertex at a
    cell centre put one vote each in that cell (closed form)."""
    ND, NP = G["n_d0"], G["n_phi0"]
    delta = 2 * G["d0_half"] / ND
    dr = VD["r_max"] / VD["n_r"]
    jv, q = 5, 11                                  # vertex cell: r = 11 cm
    th = (2 * q + 1 - VD["n_theta"]) * math.pi / VD["n_theta"]
    rv = (jv + 0.5) * dr
    cands = []
    for k in range(NP):
        phi0 = (2 * k + 1 - NP) * math.pi / NP
        sn = math.sin(th - phi0)
        if abs(sn) < 0.5:
            continue                               # nearly parallel to the ray
        d0 = rv * sn
        j = int(round(d0 / delta + ND / 2))
        if 0 <= j < ND:
            cands.append((0, j, k, 9))
    acc = V.vote(G, VD, np.array(cands, np.int32))[0]
    # |d0 error| <= delta / 2 moves r by <= delta / (2 * 0.5) < dr / 2
    assert acc[jv, q] == len(cands)
    pk, cnt, first = V.find(dict(VD, threshold=len(cands) - 1), acc)
    assert [tuple(p) for p in pk] == [(0, jv, q, len(cands))] and first == 0


def test_beam_pipe_filter_is_a_prefix():
    vd = dict(VD, threshold=2)
    acc = np.zeros((vd["n_r"], vd["n_theta"]), np.int64)
    for j, q in [(0, 3), (0, 40), (1, 10), (2, 50), (7, 0)]:
        acc[j, q] = 5
    pk, cnt, first = V.find(vd, acc)
    assert cnt == 5
    # bin centres 1, 1, 3, 5, 15 cm: only the two at 1 cm are inside 3.0 cm
    assert first == 2 and list(pk[:, 1]) == [0, 0, 1, 2, 7]
    assert V.first_kept(dict(vd, r_keep=3.5), pk) == 3


def test_min_count_drops_weak_candidates():
    c = np.array([[0, 70, 5, 8], [0, 80, 9, 12]], np.int32)
    a1, v1 = V.vote(G, dict(VD, min_count=10), c)
    a2, v2 = V.vote(G, VD, c[1:])
    assert np.array_equal(a1, a2) and v1 == v2
