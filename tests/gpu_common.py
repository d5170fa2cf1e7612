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
