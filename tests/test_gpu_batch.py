"""The batched runtime (persistent queue kernels, CUDA graph replay) against
the oracle and against the single-event calls, on a stream of events with
uneven hit counts (the batched-stream workload's generator mix)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import oracle_sampled_check, batch_event, cuda_ok, gpu_event, to_dev

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

NAME = "stream2000_256"


def make_batch(seed0, sizes):
    gen = synth.CONFIGS[NAME]["gen"]
    evs = [synth.make_event(gen, seed0 + i, target_hits=h) for i, h in enumerate(sizes)]
    off = np.zeros(len(evs) + 1, np.int32)
    off[1:] = np.cumsum([ev.n_hits for ev in evs])
    cat = lambda k: np.concatenate([getattr(ev, k) for ev in evs]).astype(np.float32)
    return evs, off, cat("x"), cat("y"), cat("z")


def test_batch_equals_oracle_and_single_event_path():
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(NAME)
    cap = 1 << 20
    # includes events above 32767 hits (unpacked vote tiles) and tiny ones
    sizes = [2000, 40000, 5000, 17000, 2500, 34000, 9000]
    evs, off, x, y, z = make_batch(500, sizes)
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=8, max_hits=int(off[-1]) + 1000, cap=cap)
    B.run(to_dev(x), to_dev(y), to_dev(z), off)
    torch.cuda.synchronize()
    for e, ev in enumerate(evs):
        r = batch_event(B, off, e)
        s = gpu_event(g, ev.x, ev.y, ev.z, cap)
        assert r["count"] == s["count"], e
        assert np.array_equal(r["peaks"], s["peaks"]), e
        assert np.array_equal(r["assign"], s["assign"]), e
        assert np.array_equal(r["zres"], s["zres"]), e
        assert r["votes"] == int(s["stats"][0]), e
    # every event against the oracle: the smallest whole, the others with
    # the whole peak list and sampled association and z results
    ev = evs[0]
    o = oracle.run_event(g, ev.x, ev.y, ev.z, cap=cap)
    r = batch_event(B, off, 0)
    assert r["count"] == o["count"]
    assert np.array_equal(r["peaks"], o["peaks"])
    assert np.array_equal(r["assign"], o["assign"])
    assert np.array_equal(r["zres"], o["zres"])
    for e in range(1, len(evs)):
        oracle_sampled_check(g, evs[e], batch_event(B, off, e), cap, n_hits=128, n_cands=4,
                             seed=e)
    B.close()
    G.close()


def test_graph_replay_with_new_events_and_autotune():
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(NAME)
    cap = 1 << 19
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=4, max_hits=80000, cap=cap)
    xs = []
    for seed0, sizes in [(600, [3000, 8000, 2000, 12000]), (700, [9000, 2100, 2000, 30000])]:
        evs, off, x, y, z = make_batch(seed0, sizes)
        buf = [torch.zeros(80000, dtype=torch.float32, device="cuda") for _ in range(3)]
        for b_, a in zip(buf, (x, y, z)):
            b_[:a.shape[0]] = to_dev(a)
        xs.append((evs, off, buf))
    # same buffers, same event count: the second batch replays the graph
    ref_buf = [torch.zeros(80000, dtype=torch.float32, device="cuda") for _ in range(3)]
    for evs, off, buf in xs:
        for d, s in zip(ref_buf, buf):
            d.copy_(s)
        B.run(ref_buf[0], ref_buf[1], ref_buf[2], off)
        torch.cuda.synchronize()
        for e, ev in enumerate(evs):
            r = batch_event(B, off, e)
            s = gpu_event(g, ev.x, ev.y, ev.z, cap)
            assert r["count"] == s["count"]
            assert np.array_equal(r["peaks"], s["peaks"])
            assert np.array_equal(r["assign"], s["assign"])
            assert np.array_equal(r["zres"], s["zres"])
    choice = B.autotune(ref_buf[0], ref_buf[1], ref_buf[2], xs[-1][1])
    assert choice["kt_pack"] in (1, 2, 4) and choice["kt_assoc"] in (1, 2, 4)
    B.run(ref_buf[0], ref_buf[1], ref_buf[2], xs[-1][1])
    torch.cuda.synchronize()
    evs, off, _ = xs[-1]
    for e, ev in enumerate(evs):
        r = batch_event(B, off, e)
        s = gpu_event(g, ev.x, ev.y, ev.z, cap)
        assert np.array_equal(r["peaks"], s["peaks"])
        assert np.array_equal(r["assign"], s["assign"])
    B.close()
    G.close()


@pytest.mark.parametrize("n_phi0", [8, 24, 136])
def test_hit_lists_on_few_column_groups_and_odd_hits(n_phi0):
    """Batched tiles scan per-event hit lists by groups of 8 phi0 columns:
    one group, three, and a count that is not a power of two; events with
    hits near the origin (windows covering the circle), an empty event, and
    the rest of a generated event -- results equal the single-event path,
    which scans every hit."""
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of("event100_256", n_rho=64, n_d0=64, n_phi0=n_phi0)
    rng = np.random.default_rng(n_phi0)
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 40 + n_phi0, target_hits=3000)
    near = rng.normal(0.0, 0.05, (200, 2)).astype(np.float32)          # r ~ 0.05 cm
    parts = [(ev.x, ev.y, ev.z), (near[:, 0], near[:, 1], np.zeros(200, np.float32)),
             (np.zeros(0, np.float32),) * 3, (ev.x[::3], ev.y[::3], ev.z[::3])]
    off = np.zeros(len(parts) + 1, np.int32)
    off[1:] = np.cumsum([p[0].shape[0] for p in parts])
    cat = lambda i: to_dev(np.concatenate([p[i] for p in parts]).astype(np.float32))
    cap = 1 << 16
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=len(parts), max_hits=int(off[-1]), cap=cap)
    B.run(cat(0), cat(1), cat(2), off)
    torch.cuda.synchronize()
    for e, (px, py, pz) in enumerate(parts):
        r = batch_event(B, off, e)
        if px.shape[0] == 0:
            assert r["count"] == 0
            continue
        s = gpu_event(g, px, py, pz, cap)
        assert r["count"] == s["count"], e
        assert np.array_equal(r["peaks"], s["peaks"]), e
        assert np.array_equal(r["assign"], s["assign"]), e
        assert r["votes"] == int(s["stats"][0]), e
    B.close()
    G.close()


@pytest.mark.parametrize("seed0", [300, 302])
def test_pileup_geometry_batch_equals_single_event_path(seed0):
    """The pile-up-like configuration (512 x 256 x 1024, ~50k hits per event,
    above the packed-counter limit) through the batched runtime equals the
    single-event calls, and a sample of the assignments equals the oracle's
    (the batch and the single-event path tile the association differently,
    so a read outside a tile's key map shows up as a difference)."""
    import torch
    from paper_1309_6275_gb300 import ht
    name = "pileup_512"
    g = synth.geometry_of(name)
    gen = synth.CONFIGS[name]["gen"]
    evs = [synth.make_event(gen, seed0 + i) for i in range(2)]
    off = np.zeros(3, np.int32)
    off[1:] = np.cumsum([e.n_hits for e in evs])
    cat = lambda k: to_dev(np.concatenate([getattr(e, k) for e in evs]).astype(np.float32))
    cap = 1 << 22
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=2, max_hits=int(off[-1]), cap=cap)
    B.run(cat("x"), cat("y"), cat("z"), off)
    torch.cuda.synchronize()
    for e, ev in enumerate(evs):
        r = batch_event(B, off, e)
        s = gpu_event(g, ev.x, ev.y, ev.z, cap)
        assert r["count"] == s["count"], e
        assert np.array_equal(r["peaks"], s["peaks"]), e
        assert np.array_equal(r["assign"], s["assign"]), e
        assert np.array_equal(r["zres"], s["zres"]), e
        assert r["votes"] == int(s["stats"][0]), e
        sel = np.random.default_rng(seed0 + e).choice(ev.n_hits, 24, replace=False)
        asg = oracle.associate_dense(g, ev.x, ev.y, s["peaks"], hit_idx=sel)
        assert np.array_equal(r["assign"][sel], asg), e
    B.close()
    G.close()


def test_packed_and_unpacked_tiles_within_one_event():
    """Tiles whose hit list holds more than 32767 hits take 32-bit counters,
    the others packed 16-bit ones, within one event: 30000 hits near the beam
    line (in every column group's list, and all voting near d0 = 0, so cells
    come close to the 16-bit limit) plus ordinary hits confined to one
    azimuthal sector, which push only the groups around it past the limit.
    Results equal the single-event path (32-bit tiles throughout)."""
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of("event100_256", n_rho=64, n_d0=64, n_phi0=64)
    rng = np.random.default_rng(77)
    near = rng.normal(0.0, 0.05, (30000, 2)).astype(np.float32)
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 78, target_hits=40000)
    psi = np.arctan2(ev.y, ev.x)
    sec = (psi > 0.0) & (psi < 0.6)
    parts = [(np.concatenate([near[:, 0], ev.x[sec]]), np.concatenate([near[:, 1], ev.y[sec]]),
              np.concatenate([np.zeros(30000, np.float32), ev.z[sec]])),
             (ev.x[:5000], ev.y[:5000], ev.z[:5000])]
    assert parts[0][0].shape[0] > 32767
    off = np.zeros(len(parts) + 1, np.int32)
    off[1:] = np.cumsum([p[0].shape[0] for p in parts])
    cat = lambda i: to_dev(np.concatenate([p[i] for p in parts]).astype(np.float32))
    cap = 1 << 18
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=len(parts), max_hits=int(off[-1]), cap=cap)
    B.run(cat(0), cat(1), cat(2), off)
    torch.cuda.synchronize()
    for e, (px, py, pz) in enumerate(parts):
        r = batch_event(B, off, e)
        s = gpu_event(g, px.astype(np.float32), py.astype(np.float32), pz.astype(np.float32), cap)
        assert r["votes"] == int(s["stats"][0]), e
        assert r["count"] == s["count"], e
        assert np.array_equal(r["peaks"], s["peaks"]), e
        assert np.array_equal(r["assign"], s["assign"]), e
        assert np.array_equal(r["zres"], s["zres"]), e
    B.close()
    G.close()
