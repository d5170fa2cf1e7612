"""The second transform (ht_vertex_*) on the GPU against its oracle: vertex
accumulators, peak lists, totals and beam-pipe filter indices identical,
on displaced-jet events (candidates from the batched first transform) and
on a dense candidate list (every peak of a 3000-hit event, prompt
candidates with d0 = 0 included)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import cuda_ok, to_dev
from oracle import vertex as V

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def _check(Vx, vd, g, e, cands):
    r = Vx.event_results(e)
    o = V.run(g, vd, cands)
    assert np.array_equal(r["acc"].astype(np.int64), o["acc"])
    assert r["votes"] == o["votes"]
    assert r["count"] == o["count"]
    assert np.array_equal(r["peaks"], o["peaks"][:Vx.cap])
    assert r["first"] == V.first_kept(vd, o["peaks"][:Vx.cap])
    return r, o


def test_vertex_transform_on_jet_events():
    import torch
    from paper_1309_6275_gb300 import ht
    name = "jets4_256"
    cfg = synth.CONFIGS[name]
    g = synth.geometry_of(name)
    vd = cfg["vertex"]
    evs = [synth.generate(cfg["gen"], 40 + i) for i in range(6)]
    off = np.zeros(len(evs) + 1, np.int32)
    off[1:] = np.cumsum([e.n_hits for e in evs])
    cat = lambda k: to_dev(np.concatenate([getattr(e, k) for e in evs]).astype(np.float32))
    cap = 1 << 16
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=len(evs), max_hits=int(off[-1]), cap=cap)
    B.run(cat("x"), cat("y"), cat("z"), off)
    Vx = ht.Vertex(G, vd, max_events=len(evs), cap=4096)
    Vx.run(B.peaks, B.counts, cap, len(evs))
    torch.cuda.synchronize()
    for e, ev in enumerate(evs):
        cands = B.event_results(off, e)["peaks"]
        r, o = _check(Vx, vd, g, e, cands)
        assert r["votes"] > 0
    # the same candidates through the oracle's first transform
    o1 = oracle.run_event(g, evs[0].x, evs[0].y, evs[0].z)
    assert np.array_equal(o1["peaks"], B.event_results(off, 0)["peaks"])
    Vx.close()
    B.close()
    G.close()


def test_vertex_transform_on_dense_candidates():
    import torch
    from paper_1309_6275_gb300 import ht
    name = "event100_256"
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 77, target_hits=3000)
    acc, _ = oracle.vote(g, ev.x, ev.y)
    pk, cnt = oracle.peaks(g, acc)
    assert (pk[:, 1] == g["n_d0"] // 2).sum() > 100          # prompt candidates
    for vd in (dict(n_r=64, n_theta=256, r_max=32.0, threshold=6, min_count=0, r_keep=3.0),
               dict(n_r=16, n_theta=64, r_max=32.0, threshold=5, min_count=9, r_keep=3.0)):
        G = ht.Geometry(g)
        Vx = ht.Vertex(G, vd, max_events=1, cap=1 << 14)
        d_pk = to_dev(np.ascontiguousarray(pk, np.int32))
        d_cnt = torch.tensor([cnt], dtype=torch.int32, device="cuda")
        Vx.run(d_pk, d_cnt, pk.shape[0], 1)
        torch.cuda.synchronize()
        r, o = _check(Vx, vd, g, 0, pk)
        assert r["redo"] < 0.01 * max(r["votes"], 1) + 64
        Vx.close()
        G.close()


def test_vertex_create_rejects_bad_descriptors():
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of("jets4_256")
    G = ht.Geometry(g)
    for bad in (dict(n_theta=48), dict(n_r=0), dict(threshold=0), dict(r_max=0.0)):
        vd = dict(n_r=16, n_theta=64, r_max=32.0, threshold=5, min_count=0, r_keep=3.0)
        vd.update(bad)
        with pytest.raises(ht.HTError):
            ht.Vertex(G, vd, max_events=1, cap=16)
    G.close()
