"""The track path on the GPU against the oracle, through the C ABI: the
distinct-layer vote, peaks, the candidate confirmation, the final hit
assignment and the (z0, cot theta) vote -- single events and batches.

Every comparison is exact: accumulator cells, peak lists, confirmation
scores, inlier hits per layer, assignments and z results.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (assert_same_acc, assert_same_tracks, check_assign, cuda_ok,
                        gpu_tracks_event, oracle_tracks, to_dev)

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CP = dict(pool=4, min_layers=8, n_layers=10, tol=0.01)
CP_SPARSE = dict(pool=20, min_layers=6, n_layers=10, tol=0.01)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_single_event_workload_at_its_threshold(seed):
    g = synth.geometry_of("single_64")
    g["threshold"] = 3
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], seed)
    cap = 1 << 16
    r = gpu_tracks_event(g, ev, cap, CP_SPARSE)
    o = oracle_tracks(g, ev, cap, CP_SPARSE)
    assert_same_tracks(r, o)
    assert (o["score"] > 0).sum() > 0


def test_dense_event_full_size():
    """A whole 10k-hit event of the 100-event workload at T = 9 (about 10^5
    candidates): every cell, candidate, inlier and assignment."""
    g = synth.geometry_of("event100_256")
    g["threshold"] = 9
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 0)
    cap = 1 << 20
    r = gpu_tracks_event(g, ev, cap, CP)
    o = oracle_tracks(g, ev, cap, CP)
    assert_same_tracks(r, o)
    assert (o["score"] > 0).sum() > 300


def test_wide_pool_takes_several_passes():
    """pool = 40 bins: most candidates' pools exceed one pass (384 hits), so
    the later passes, their block skipping and their float64 contenders run."""
    g = synth.geometry_of("event100_256")
    g["threshold"] = 10
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 1)
    cp = dict(CP, pool=40)
    cap = 1 << 20
    r = gpu_tracks_event(g, ev, cap, cp)
    o = oracle_tracks(g, ev, cap, cp)
    assert_same_tracks(r, o)


def test_capacity_truncation_and_empty_event():
    g = synth.geometry_of("event100_256")
    g["threshold"] = 9
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 2, target_hits=3000)
    cap = 500
    r = gpu_tracks_event(g, ev, cap, CP)
    o = oracle_tracks(g, ev, cap, CP)
    assert o["count"] > cap
    assert_same_tracks(r, o)
    empty = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 3, target_hits=3000)
    for k in ("x", "y", "z", "layer", "track"):
        setattr(empty, k, getattr(empty, k)[:0])
    r = gpu_tracks_event(g, empty, cap, CP)
    assert r["count"] == 0 and r["assign"].size == 0 and int(r["acc"].max()) == 0


# ------------------------------------------------------------------ batches
BANDS = [(4000, 7), (7000, 8), (15000, 9)]


def band_threshold(n, default=10):
    for mh, t in BANDS:
        if n <= mh:
            return t
    return default


def make_batch(seed0, sizes, name="stream2000_256"):
    gen = synth.CONFIGS[name]["gen"]
    evs = [synth.make_event(gen, seed0 + i, target_hits=h) for i, h in enumerate(sizes)]
    off = np.zeros(len(evs) + 1, np.int32)
    off[1:] = np.cumsum([ev.n_hits for ev in evs])
    cat = lambda k, t: np.concatenate([getattr(ev, k) for ev in evs]).astype(t)
    return evs, off, cat("x", np.float32), cat("y", np.float32), cat("z", np.float32), \
        cat("layer", np.uint8)


def run_batch(g, evs, off, x, y, z, lay, cap, hit_masks=None, repeat=1):
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=len(evs), max_hits=int(off[-1]) + 64, cap=cap)
    B.set_confirm(dict(CP, bands=BANDS))
    X, Y, Z, L = to_dev(x), to_dev(y), to_dev(z), to_dev(lay)
    HM = to_dev(hit_masks.view(np.int64)) if hit_masks is not None else None
    outs = []
    for _ in range(repeat):
        B.run_tracks(X, Y, Z, L, off, hit_masks=HM)
        torch.cuda.synchronize()
        outs.append([B.event_results(off, e) for e in range(len(evs))])
    B.close()
    G.close()
    return outs


def test_batch_tracks_equal_the_oracle_per_event():
    """A stream batch with 2k- to 40k-hit events; each event at its band
    threshold, against the oracle; a second replay of the graph repeats it."""
    g0 = dict(synth.geometry_of("stream2000_256"), threshold=10)   # above the last band
    sizes = [2000, 40000, 5000, 12000, 2500, 6500]
    evs, off, x, y, z, lay = make_batch(700, sizes)
    cap = 1 << 19
    runs = run_batch(g0, evs, off, x, y, z, lay, cap, repeat=2)
    for e, ev in enumerate(evs):
        g = dict(g0, threshold=band_threshold(ev.n_hits))
        o = oracle_tracks(g, ev, cap, CP)
        r = runs[0][e]
        check_assign(r["assign"], r["count"])
        assert r["count"] == o["count"], e
        assert np.array_equal(r["peaks"], o["peaks"]), e
        assert np.array_equal(r["score"], o["score"]), e
        assert np.array_equal(r["assign"], o["assign"]), e
        assert np.array_equal(r["zres"], o["zres"]), e
        assert r["votes"] == o["votes"], e
        for k in ("peaks", "score", "assign", "zres"):
            assert np.array_equal(runs[1][e][k], r[k]), (e, k)


def test_batch_tracks_with_per_hit_region_sets():
    """Given per-hit region sets restrict each hit's votes (the learned
    proposal's per-hit mode) on the track path."""
    g0 = dict(synth.geometry_of("stream2000_256"), threshold=10)
    sizes = [3000, 9000, 14000]
    evs, off, x, y, z, lay = make_batch(710, sizes)
    rng = np.random.default_rng(5)
    masks = np.zeros(x.shape[0], np.uint64)
    for b in range(12):   # about 12 of 64 regions per hit
        masks |= np.uint64(1) << rng.integers(0, 64, x.shape[0]).astype(np.uint64)
    cap = 1 << 19
    runs = run_batch(g0, evs, off, x, y, z, lay, cap, hit_masks=masks)
    for e, ev in enumerate(evs):
        g = dict(g0, threshold=band_threshold(ev.n_hits))
        o = oracle_tracks(g, ev, cap, CP, masks=masks[off[e]:off[e + 1]])
        r = runs[0][e]
        assert r["count"] == o["count"], e
        assert np.array_equal(r["peaks"], o["peaks"]), e
        assert np.array_equal(r["score"], o["score"]), e
        assert np.array_equal(r["assign"], o["assign"]), e
        assert np.array_equal(r["zres"], o["zres"]), e


def test_host_buffer_call_returns_the_confirmed_candidates():
    """ht_batch_run_tracks_host: the tracks of each event are its confirmed
    candidates in candidate order with their z results, and each hit's
    assignment points at its candidate's track; a too-small track_cap gives
    the first tracks and the capacity status."""
    import torch
    from paper_1309_6275_gb300 import ht
    g0 = dict(synth.geometry_of("stream2000_256"), threshold=10)
    sizes = [3000, 11000, 6000]
    evs, off, x, y, z, lay = make_batch(720, sizes)
    cap = 1 << 19
    dev = run_batch(g0, evs, off, x, y, z, lay, cap)[0]
    G = ht.Geometry(g0)
    B = ht.Batch(G, max_events=len(evs), max_hits=int(off[-1]) + 64, cap=cap)
    B.set_confirm(dict(CP, bands=BANDS))
    tracks = np.zeros((1 << 16, 8), np.int32)
    ntr = np.zeros(len(evs), np.int32)
    asg = np.zeros(int(off[-1]), np.int32)
    assert B.run_tracks_host(x, y, z, lay, off, tracks, ntr, asg)
    base = 0
    for e, r in enumerate(dev):
        conf = np.flatnonzero(r["score"] > 0)
        assert ntr[e] == conf.size, e
        t = tracks[base:base + ntr[e]]
        assert np.array_equal(t[:, :4], r["peaks"][conf]), e
        assert np.array_equal(t[:, 4], r["score"][conf]), e
        assert np.array_equal(t[:, 5:8], r["zres"][conf]), e
        remap = np.full(r["count"], -1, np.int64)
        remap[conf] = np.arange(conf.size)
        a = r["assign"]
        want = np.where(a >= 0, remap[np.maximum(a, 0)], -1)
        assert np.array_equal(asg[off[e]:off[e + 1]], want), e
        base += ntr[e]
    small = np.zeros((5, 8), np.int32)
    ntr2 = np.zeros(len(evs), np.int32)
    assert not B.run_tracks_host(x, y, z, lay, off, small, ntr2, asg)
    assert np.array_equal(ntr2, ntr) and np.array_equal(small, tracks[:5])
    B.close()
    G.close()


def test_pileup_event_full_size():
    """A whole 50k-hit pile-up event (512 x 256 x 1024) on the track path at
    its configured threshold and tolerance: every cell, candidate, score,
    inlier, assignment and z result."""
    name = "pileup_512"
    g = synth.track_geometry(name)
    tk = synth.track_of(name)
    cp = dict(pool=tk["pool"], min_layers=tk["min_layers"], n_layers=tk["n_layers"], tol=tk["tol"])
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 0)
    cap = 1 << 21
    r = gpu_tracks_event(g, ev, cap, cp)
    o = oracle_tracks(g, ev, cap, cp)
    assert_same_tracks(r, o)
