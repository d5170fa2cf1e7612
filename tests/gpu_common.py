"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
binding and the oracle on the same seeded inputs."""
import functools

import numpy as np

import oracle
import synth


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_event(g, x, y, z, cap):
    """The four calls of the path on one event; results as numpy arrays."""
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    p = ht.EventPipeline(G, max(len(x), 1), cap)
    p.run(to_dev(x), to_dev(y), to_dev(z))
    torch.cuda.synchronize()
    r = p.results(len(x))
    G.close()
    check_assign(r["assign"], r["count"])
    return r


def check_assign(assign, count):
    """Every assignment is -1 or the index of a found candidate."""
    a = np.asarray(assign)
    bad = np.nonzero((a < -1) | (a >= count))[0]
    assert bad.size == 0, f"{bad.size} assignments out of [-1, {count}): hits {bad[:5].tolist()} -> {a[bad[:5]].tolist()}"


def batch_event(B, offsets, e):
    """Event e's results from a Batch, with the assignment range checked."""
    r = B.event_results(offsets, e)
    check_assign(r["assign"], r["count"])
    return r


@functools.lru_cache(maxsize=8)
def oracle_event(name, seed, threshold=None):
    """Cached oracle run of a generated event: (event, geometry, results)."""
    g = synth.geometry_of(name)
    if threshold is not None:
        g["threshold"] = threshold
    ev = synth.make_event(synth.CONFIGS[name]["gen"], seed)
    acc, st = oracle.vote(g, ev.x, ev.y)
    pk, cnt = oracle.peaks(g, acc)
    return ev, g, dict(acc=acc, stats=st, peaks=pk, count=cnt)


def assert_same_acc(gpu_acc, ora_acc):
    a = np.asarray(gpu_acc).astype(np.int64)
    b = np.asarray(ora_acc).astype(np.int64)
    assert a.shape == b.shape
    bad = np.argwhere(a != b)
    assert bad.shape[0] == 0, (f"{bad.shape[0]} cells differ; first {bad[:5].tolist()} "
                               f"gpu {a[tuple(bad[:5].T)].tolist()} oracle {b[tuple(bad[:5].T)].tolist()}")


def oracle_sampled_check(g, ev, r, cap, n_hits=256, n_cands=8, seed=0, acc=None):
    """The oracle against a GPU result r of the plain path (peaks, count,
    assign, zres) on one event: the whole peak list; the association of
    n_hits sampled hits; the (z0, cot theta) result of n_cands sampled
    candidates that received hits.  The oracle finds each sampled
    candidate's hits itself: the hits compatible with it alone, then their
    assignment among all candidates.  Returns the oracle's peaks."""
    if acc is None:
        acc, _ = oracle.vote(g, ev.x, ev.y)
    pk, cnt = oracle.peaks(g, acc, cap=cap)
    del acc
    assert r["count"] == cnt
    assert np.array_equal(r["peaks"], pk)
    rng = np.random.default_rng(seed)
    sel = rng.choice(ev.n_hits, min(n_hits, ev.n_hits), replace=False)
    asg = oracle.associate_dense(g, ev.x, ev.y, pk, hit_idx=sel)
    assert np.array_equal(np.asarray(r["assign"])[sel], asg)
    got = np.asarray(r["assign"])
    owners = np.unique(got[got >= 0])
    if owners.size:
        for m in rng.choice(owners, min(n_cands, owners.size), replace=False):
            comp = np.flatnonzero(oracle.associate(g, ev.x, ev.y, pk[[m]]) == 0)
            a = oracle.associate_dense(g, ev.x, ev.y, pk, hit_idx=comp)
            full = np.full(ev.n_hits, -1, np.int32)
            full[comp] = a
            zo = oracle.vote_z(g, ev.x, ev.y, ev.z, full, pk, cand=np.array([m]))
            assert np.array_equal(np.asarray(r["zres"])[m], zo[0]), m
    return pk


# ------------------------------------------------------------------ track path
def gpu_tracks_event(g, ev, cap, cp):
    """The five calls of the track path on one event; numpy results."""
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    n = ev.n_hits
    x, y, z = to_dev(ev.x), to_dev(ev.y), to_dev(ev.z)
    lay = to_dev(ev.layer.astype(np.uint8))
    acc = G.new_accumulator()
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    ht.ht_vote_layers(G, x, y, lay, acc, stats)
    c1 = max(cap, 1)
    peaks = torch.empty((c1, 4), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(max(G.find_peaks_workspace_size(), G.vote_z_workspace_size(max(n, 1), cap),
                         ht.ht_confirm_workspace_size(G, n, cap)), dtype=torch.uint8, device="cuda")
    ht.ht_find_peaks(G, acc, peaks, cap, count, ws)
    score = torch.full((c1,), -7, dtype=torch.int32, device="cuda")
    inl = torch.full((c1, 16), -7, dtype=torch.int32, device="cuda")
    assign = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    ht.ht_confirm(G, cp, x, y, lay, peaks, count, cap, score, inl, assign[:n], ws)
    zres = torch.empty((c1, 3), dtype=torch.int32, device="cuda")
    ht.ht_vote_z(G, x, y, z, assign[:n], peaks, count, cap, zres, ws)
    torch.cuda.synchronize()
    cnt = int(count.item())
    k = min(cnt, cap)
    a = acc.cpu().numpy()
    r = dict(acc=a.view(np.uint16) if a.dtype == np.int16 else a, count=cnt,
             peaks=peaks[:k].cpu().numpy(), score=score[:k].cpu().numpy(),
             inl=inl[:k].cpu().numpy(), assign=assign[:n].cpu().numpy(),
             zres=zres[:k].cpu().numpy(), votes=int(stats[0].item()))
    G.close()
    check_assign(r["assign"], r["count"])
    return r


def oracle_tracks(g, ev, cap, cp, masks=None):
    acc, st = oracle.vote_layers(g, ev.x, ev.y, ev.layer, masks)
    pk, cnt = oracle.peaks(g, acc, cap)
    score, seeds, inl = oracle.confirm(g, ev.x, ev.y, ev.layer, pk, cp)
    asg = oracle.confirm_assign(score, inl, ev.n_hits)
    zr = oracle.vote_z(g, ev.x, ev.y, ev.z, asg, pk)
    return dict(acc=acc, votes=st["votes"], peaks=pk, count=cnt, score=score, inl=inl,
                assign=asg, zres=zr)


def assert_same_tracks(r, o, acc=True):
    if acc:
        assert_same_acc(r["acc"], o["acc"])
        assert r["votes"] == o["votes"]
    assert r["count"] == o["count"]
    assert np.array_equal(r["peaks"], o["peaks"])
    bad = np.flatnonzero(r["score"] != o["score"])
    assert bad.size == 0, f"{bad.size} scores differ, first {bad[:5]}: {r['score'][bad[:5]]} vs {o['score'][bad[:5]]}"
    assert np.array_equal(r["inl"], o["inl"])
    bad = np.flatnonzero(r["assign"] != o["assign"])
    assert bad.size == 0, f"{bad.size} assignments differ, first {bad[:5]}"
    assert np.array_equal(r["zres"], o["zres"])
