"""Geometries at the edges of the float32 filters' error bounds, on the GPU
against the oracle through the C ABI: d0 bins of 4e-4 cm with hits out to
30 m, curvatures that curl tracks within 7 cm (second roots in the axis on
most columns), and nearly straight tracks with hits at 100-200 m.

Every filter of the vote, the bucket lists, the peak finder's inputs and
the confirmation's screen and seed frame has a margin derived from the
float32 rounding of its inputs; these scenes put hits where those margins
are smallest relative to a bin (fine bins, far hits) or where the second
root decides (tight curls).  Comparisons are exact: accumulators, peak
lists, assignments, confirmation scores and inliers, z results.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_common import (assert_same_acc, assert_same_tracks, batch_event, cuda_ok, gpu_event,
                        gpu_tracks_event, oracle_tracks, to_dev)
from synth.events import Event, helix_hits

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

# name: geometry, layer radii (cm), tracks, noise hits.  With d0 bins far
# finer than a hit's d0 step between phi0 columns (r dphi), or hits far out,
# only tracks on grid nodes make peaks; the confirmation is also run on a
# constructed candidate list (the tracks' own cells and random cells).
SCENES = {
    "fine_bins_far_hits": (
        dict(n_rho=64, n_d0=256, n_phi0=256, rho_max=0.002, d0_half=0.05, n_z0=32, n_cot=16,
             z0_max=20.0, cot_max=3.0, threshold=3, count_bits=16),
        [0.6, 0.9, 1.3, 1.8, 2.4, 3.0, 3.6, 50.0, 400.0, 3000.0], 40, 2000),
    "tight_curls": (
        dict(n_rho=48, n_d0=64, n_phi0=96, rho_max=0.15, d0_half=3.0, n_z0=32, n_cot=16,
             z0_max=20.0, cot_max=3.0, threshold=6, count_bits=16),
        [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 10.0, 12.0], 30, 300),
    "straight_far": (
        dict(n_rho=32, n_d0=64, n_phi0=128, rho_max=2e-5, d0_half=1.0, n_z0=32, n_cot=16,
             z0_max=20.0, cot_max=3.0, threshold=2, count_bits=16),
        [1000.0, 2000.0, 4000.0, 6000.0, 8000.0, 10000.0, 12000.0, 14000.0, 17000.0, 20000.0],
        25, 3000),
}
CP = dict(pool=4, min_layers=6, n_layers=10, tol=0.01)
CP_WIDE = dict(pool=40, min_layers=4, n_layers=10, tol=0.01)


def scene(name, seed):
    """Seeded hits of a scene: tracks on its layers (float64 positions,
    rounded once; every other track on a grid node, the rest anywhere) and
    uniform noise hits on random layers; the layer is the radius index."""
    g, radii, n_tracks, n_noise = SCENES[name]
    rng = np.random.Generator(np.random.Philox(1000 + seed))
    phi0s, _, _, rhos = oracle.tables(g)
    nd = g["n_d0"]
    delta = 2.0 * g["d0_half"] / nd
    xs, ys, zs, ls, ts, truth = [], [], [], [], [], []
    for t in range(n_tracks):
        if t % 2 == 0:
            # on a grid node: every hit's root in the node's column lies in
            # the node's bin up to the float32 rounding of the hit
            i = int(rng.integers(g["n_rho"] // 10, g["n_rho"] - g["n_rho"] // 10))
            rho, phi0 = float(rhos[i]), float(phi0s[int(rng.integers(g["n_phi0"]))])
            d0 = (int(rng.integers(nd // 10, nd - nd // 10)) + 0.5 - nd / 2) * delta
        else:
            rho = rng.uniform(-0.9, 0.9) * g["rho_max"]
            d0 = rng.uniform(-0.8, 0.8) * g["d0_half"]
            phi0 = rng.uniform(-math.pi, math.pi)
        truth.append((rho, d0, phi0))
        X, Y, Z, L, _ = helix_hits(rho, d0, phi0, rng.normal(0, 2.0), rng.uniform(-1, 1), radii)
        xs.append(X); ys.append(Y); zs.append(Z); ls.append(L); ts.append(np.full(X.size, t))
    lay = rng.integers(0, len(radii), n_noise)
    r = np.asarray(radii)[lay] * rng.uniform(0.999, 1.001, n_noise)
    ph = rng.uniform(-math.pi, math.pi, n_noise)
    xs.append(r * np.cos(ph)); ys.append(r * np.sin(ph)); zs.append(rng.uniform(-30, 30, n_noise))
    ls.append(lay); ts.append(np.full(n_noise, -1))
    cat = lambda v, dt: np.concatenate(v).astype(dt)
    ev = Event(x=cat(xs, np.float32), y=cat(ys, np.float32), z=cat(zs, np.float32),
               layer=cat(ls, np.int8), track=cat(ts, np.int32))
    ev.rho, ev.d0, ev.phi0 = np.array(truth).reshape(-1, 3).T
    return dict(g), ev


@pytest.mark.parametrize("name", sorted(SCENES))
def test_plain_path_single_event(name):
    g, ev = scene(name, 0)
    cap = 1 << 16
    r = gpu_event(g, ev.x, ev.y, ev.z, cap)
    acc, st = oracle.vote(g, ev.x, ev.y)
    assert_same_acc(r["acc"], np.minimum(acc, 65535))
    assert int(r["stats"][0]) == st["votes"]
    pk, cnt = oracle.peaks(g, acc, cap=cap)
    assert r["count"] == cnt and np.array_equal(r["peaks"], pk)
    asg = oracle.associate_dense(g, ev.x, ev.y, pk)
    assert np.array_equal(r["assign"], asg)
    assert np.array_equal(r["zres"], oracle.vote_z(g, ev.x, ev.y, ev.z, asg, pk))


@pytest.mark.parametrize("name", sorted(SCENES))
def test_plain_path_batched(name):
    """The batched runtime (bucket lists, persistent tiles) on two events of
    the scene equals the oracle event by event."""
    import torch
    from paper_1309_6275_gb300 import ht
    g = SCENES[name][0]
    evs = [scene(name, s)[1] for s in (1, 2)]
    off = np.array([0, evs[0].n_hits, evs[0].n_hits + evs[1].n_hits], np.int32)
    cat = lambda k: to_dev(np.concatenate([getattr(e, k) for e in evs]).astype(np.float32))
    cap = 1 << 16
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=2, max_hits=int(off[-1]), cap=cap)
    B.run(cat("x"), cat("y"), cat("z"), off)
    torch.cuda.synchronize()
    for e, ev in enumerate(evs):
        r = batch_event(B, off, e)
        o = oracle.run_event(g, ev.x, ev.y, ev.z, cap=cap)
        assert r["count"] == o["count"] and np.array_equal(r["peaks"], o["peaks"]), e
        assert np.array_equal(r["assign"], o["assign"]), e
        assert np.array_equal(r["zres"], o["zres"]), e
    B.close()
    G.close()


def constructed_candidates(g, ev, n_random, seed):
    """Each track's nearest cell (row, bin of d0, column) and n_random
    random cells, sorted by logical index; int32 [m, 4] (count 0)."""
    phi0, _, _, rho = oracle.tables(g)
    nd = g["n_d0"]
    delta = 2.0 * g["d0_half"] / nd
    cells = set()
    for r_, d_, p_ in zip(ev.rho, ev.d0, ev.phi0):
        i = int(np.argmin(np.abs(rho - r_)))
        k = int(np.argmin(np.abs(np.angle(np.exp(1j * (phi0 - p_))))))
        j = min(max(int(math.floor(d_ / delta + nd / 2)), 0), nd - 1)
        cells.add((i, j, k))
    rng = np.random.Generator(np.random.Philox(77 + seed))
    for _ in range(n_random):
        cells.add((int(rng.integers(g["n_rho"])), int(rng.integers(nd)),
                   int(rng.integers(g["n_phi0"]))))
    pk = np.array(sorted(cells, key=lambda c: (c[0] * nd + c[1]) * g["n_phi0"] + c[2]), np.int32)
    return np.concatenate([pk, np.zeros((pk.shape[0], 1), np.int32)], axis=1)


@pytest.mark.parametrize("name", ["fine_bins_far_hits", "straight_far", "tight_curls"])
def test_confirmation_of_constructed_candidates(name):
    """ht_confirm on the scene's track cells and random cells, a wide pool:
    scores, inliers and the final assignment equal the oracle's."""
    import torch
    from paper_1309_6275_gb300 import ht
    g, ev = scene(name, 6)
    pk = constructed_candidates(g, ev, 64, 6)
    m = pk.shape[0]
    score_o, _, inl_o = oracle.confirm(g, ev.x, ev.y, ev.layer, pk, CP_WIDE)
    asg_o = oracle.confirm_assign(score_o, inl_o, ev.n_hits)
    assert (score_o > 0).sum() > 0
    G = ht.Geometry(g)
    n = ev.n_hits
    x, y = to_dev(ev.x), to_dev(ev.y)
    lay = to_dev(ev.layer.astype(np.uint8))
    peaks = to_dev(pk)
    count = torch.tensor([m], dtype=torch.int32, device="cuda")
    ws = torch.empty(ht.ht_confirm_workspace_size(G, n, m), dtype=torch.uint8, device="cuda")
    score = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    inl = torch.full((m, 16), -7, dtype=torch.int32, device="cuda")
    assign = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    ht.ht_confirm(G, CP_WIDE, x, y, lay, peaks, count, m, score, inl, assign, ws)
    torch.cuda.synchronize()
    assert np.array_equal(score.cpu().numpy(), score_o)
    assert np.array_equal(inl.cpu().numpy(), inl_o)
    assert np.array_equal(assign.cpu().numpy(), asg_o)
    G.close()


@pytest.mark.parametrize("name", sorted(SCENES))
def test_track_path_single_event(name):
    g, ev = scene(name, 3)
    cap = 1 << 16
    r = gpu_tracks_event(g, ev, cap, CP)
    o = oracle_tracks(g, ev, cap, CP)
    assert o["count"] > 0
    assert_same_tracks(r, o)


@pytest.mark.parametrize("name", sorted(SCENES))
def test_track_path_batched(name):
    import torch
    from paper_1309_6275_gb300 import ht
    g = SCENES[name][0]
    evs = [scene(name, s)[1] for s in (4, 5)]
    off = np.array([0, evs[0].n_hits, evs[0].n_hits + evs[1].n_hits], np.int32)
    cat = lambda k, t: to_dev(np.concatenate([getattr(e, k) for e in evs]).astype(t))
    cap = 1 << 16
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=2, max_hits=int(off[-1]), cap=cap)
    B.set_confirm(CP)
    B.run_tracks(cat("x", np.float32), cat("y", np.float32), cat("z", np.float32),
                 cat("layer", np.uint8), off)
    torch.cuda.synchronize()
    for e, ev in enumerate(evs):
        r = B.event_results(off, e)
        o = oracle_tracks(g, ev, cap, CP)
        assert r["count"] == o["count"] and np.array_equal(r["peaks"], o["peaks"]), e
        assert np.array_equal(r["score"], o["score"]), e
        assert np.array_equal(r["assign"], o["assign"]), e
        assert np.array_equal(r["zres"], o["zres"]), e
    B.close()
    G.close()
