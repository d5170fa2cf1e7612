"""The learned proposal on the GPU against its oracle (oracle/mlp.py):
MLP forward, gradients and Adam (BF16 numerics: per-tensor relative L2
<= 1e-2 and cosine >= 0.999 against the oracle run on the same BF16
parameters and features), region masks, and the masked vote / peaks / batch
runs (exact: halo cells, peak lists, assignments and z results identical to
the oracle's full path restricted to the mask)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_same_acc, batch_event, cuda_ok, to_dev
from oracle import mlp

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C2 = "event100_256"


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


def bf16_bits(p):
    """BF16 copy of float parameters as int16 bits (round to nearest even)."""
    import torch
    return torch.from_numpy(mlp.bf16(p).astype(np.float32)).to(torch.bfloat16).view(torch.int16)


def to_np_bf16(t):
    import torch
    return t.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)


def params(seed, scale=0.15):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, mlp.n_params())
    return p


def hits(n, seed=0):
    ev = synth.make_event(synth.CONFIGS[C2]["gen"], seed)
    return ev, ev.x[:n], ev.y[:n], ev.z[:n], ev.layer[:n].astype(np.uint8)


def gpu_forward(p, x, y, z, layer):
    import torch
    from paper_1309_6275_gb300 import ht
    n = len(x)
    pb = bf16_bits(p).cuda()
    prob = torch.empty((n, 64), dtype=torch.float32, device="cuda")
    h1 = torch.empty((n, 128), dtype=torch.int16, device="cuda")
    h2 = torch.empty((n, 128), dtype=torch.int16, device="cuda")
    feat = torch.empty((n, 8), dtype=torch.int16, device="cuda")
    ht.ht_mlp_forward(pb, to_dev(x), to_dev(y), to_dev(z), to_dev(layer), prob, h1, h2, feat)
    torch.cuda.synchronize()
    return pb, prob, h1, h2, feat


def test_forward_matches_oracle():
    p = params(1)
    _, x, y, z, layer = hits(3000)
    _, prob, h1, h2, feat = gpu_forward(p, x, y, z, layer)
    f_gpu = to_np_bf16(feat)[:, :6]
    f_ora = mlp.features(x, y, z, layer)
    # float32 features (atan2f vs numpy's arctan2) may differ by one BF16 step
    d = np.abs(f_gpu - f_ora)
    assert np.all(d <= np.abs(f_ora) * 2 ** -7 + 1e-30)
    assert (d > 0).mean() < 0.01
    assert np.all(to_np_bf16(feat)[:, 6:] == 0)
    _, P, (_, H1, H2, _, _, _) = mlp.forward(p, f_gpu)
    for a, b in ((prob.cpu().numpy(), P), (to_np_bf16(h1), H1), (to_np_bf16(h2), H2)):
        assert rel_l2(a, b) <= 1e-2 and cosine(a, b) >= 0.999
    assert np.allclose(prob.cpu().numpy().sum(1), 1.0, atol=1e-5)
    from paper_1309_6275_gb300 import ht
    assert ht.ht_mlp_timeouts() == 0


def test_gradients_match_oracle():
    import torch
    from paper_1309_6275_gb300 import ht
    p = params(2)
    _, x, y, z, layer = hits(2500, seed=1)
    rng = np.random.default_rng(3)
    lab = rng.integers(-1, 64, len(x)).astype(np.int32)
    pb, prob, h1, h2, feat = gpu_forward(p, x, y, z, layer)
    grad = torch.zeros(mlp.n_params(), dtype=torch.float32, device="cuda")
    ws = torch.empty(ht.ht_mlp_backward_workspace_size(len(x)), dtype=torch.uint8, device="cuda")
    ht.ht_mlp_backward(pb, to_dev(lab), prob, h1, h2, feat, grad, ws)
    torch.cuda.synchronize()
    f_gpu = to_np_bf16(feat)[:, :6]
    _, g_ora = mlp.loss_and_grad(p, f_gpu, lab)
    g_gpu = grad.cpu().numpy()
    k = 0
    for (i, o) in mlp.SIZES:
        for part in (i * o, o):
            a, b = g_gpu[k:k + part], g_ora[k:k + part]
            assert rel_l2(a, b) <= 1e-2 and cosine(a, b) >= 0.999, (k, rel_l2(a, b), cosine(a, b))
            k += part
    # gradients add into grad: a second call doubles them
    ht.ht_mlp_backward(pb, to_dev(lab), prob, h1, h2, feat, grad, ws)
    torch.cuda.synchronize()
    assert np.allclose(grad.cpu().numpy(), 2 * g_gpu, rtol=1e-5, atol=1e-9)


def test_adam_matches_oracle():
    import torch
    from paper_1309_6275_gb300 import ht
    rng = np.random.default_rng(4)
    n = mlp.n_params()
    # the same float32 starting values on both sides
    p, m, v, g = (rng.normal(0, s, n).astype(np.float32).astype(np.float64)
                  for s in (0.2, 0.01, 1e-4, 0.05))
    v = np.abs(v)
    P, M, V, Gd = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, m, v, g))
    pb = torch.empty(n, dtype=torch.int16, device="cuda")
    for step in (1, 7):
        ht.ht_mlp_adam(P, M, V, Gd, step, 1e-3, 0.9, 0.999, 1e-8, pb)
        p, m, v = mlp.adam(p, m, v, g, step, 1e-3)
    torch.cuda.synchronize()
    # float32 arithmetic: a few units of 2^-24 of each operand's scale
    for got, want in ((P, p), (M, m), (V, v)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
    pbn = to_np_bf16(pb)
    assert np.mean(pbn == mlp.bf16(P.cpu().numpy())) == 1.0


def test_training_steps_reduce_the_loss():
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(C2)
    ev = synth.make_event(synth.CONFIGS[C2]["gen"], 7)
    lab = mlp.hit_labels(g, ev)
    x, y, z, layer = ev.x, ev.y, ev.z, ev.layer.astype(np.uint8)
    p0 = params(5, 0.1)
    n, npar = len(x), mlp.n_params()
    P = torch.from_numpy(p0.astype(np.float32)).cuda()
    M = torch.zeros(npar, device="cuda"); V = torch.zeros(npar, device="cuda")
    pb = bf16_bits(p0).cuda()
    prob = torch.empty((n, 64), device="cuda")
    h1, h2 = (torch.empty((n, 128), dtype=torch.int16, device="cuda") for _ in range(2))
    feat = torch.empty((n, 8), dtype=torch.int16, device="cuda")
    grad = torch.zeros(npar, device="cuda")
    ws = torch.empty(ht.ht_mlp_backward_workspace_size(n), dtype=torch.uint8, device="cuda")
    dx, dy, dz, dl, dlab = to_dev(x), to_dev(y), to_dev(z), to_dev(layer), to_dev(lab)
    for step in range(1, 31):
        ht.ht_mlp_forward(pb, dx, dy, dz, dl, prob, h1, h2, feat)
        grad.zero_()
        ht.ht_mlp_backward(pb, dlab, prob, h1, h2, feat, grad, ws)
        ht.ht_mlp_adam(P, M, V, grad, step, 3e-3, 0.9, 0.999, 1e-8, pb)
    torch.cuda.synchronize()
    f = mlp.features(x, y, z, layer)
    l0, _ = mlp.loss_and_grad(p0, f, lab)
    l1, _ = mlp.loss_and_grad(P.cpu().numpy().astype(np.float64), f, lab)
    assert l1 < 0.7 * l0, (l0, l1)


def test_region_masks_match_oracle():
    import torch
    from paper_1309_6275_gb300 import ht
    p = params(6, 0.1)
    W = mlp.unpack(p)
    W[5][[4, 12, 20, 44, 52]] += 3.0          # favour a few regions
    gen = synth.CONFIGS[C2]["gen"]
    e0, e2 = synth.make_event(gen, 11, target_hits=3000), synth.make_event(gen, 13, target_hits=1200)
    parts = [(e0.x, e0.y, e0.z, e0.layer), tuple(a[:0] for a in (e0.x, e0.y, e0.z, e0.layer)),
             (e2.x, e2.y, e2.z, e2.layer)]                 # the middle event is empty
    evs = parts
    off = np.zeros(len(parts) + 1, np.int32)
    off[1:] = np.cumsum([len(p_[0]) for p_ in parts])
    cat = lambda k, t: np.concatenate([p_[k] for p_ in parts]).astype(t)
    x, y, z, layer = cat(0, np.float32), cat(1, np.float32), cat(2, np.float32), cat(3, np.uint8)
    pb = bf16_bits(p).cuda()
    mass = torch.empty((len(evs), 64), device="cuda")
    masks = torch.empty(len(evs), dtype=torch.int64, device="cuda")
    tau, fmax = 0.03, 0.5
    for grow in (0, 1):
        ht.ht_mlp_region_mask(pb, to_dev(x), to_dev(y), to_dev(z), to_dev(layer), to_dev(off),
                              tau, fmax, grow, mass, masks)
        torch.cuda.synchronize()
        f = mlp.features(x, y, z, layer)
        _, P, _ = mlp.forward(p, f)
        ms = mass.cpu().numpy()
        got = [int(v) & ((1 << 64) - 1) for v in masks.cpu().numpy()]
        for e in range(len(evs)):
            a, b = off[e], off[e + 1]
            mean_o = mlp.region_mass(P[a:b])
            n = b - a
            if n:
                assert np.allclose(ms[e] / n, mean_o, atol=2e-4)
            want = mlp.region_mask(mean_o, tau, fmax, grow=bool(grow), n_hits=n)
            near = np.abs(mean_o - tau) < 2e-4
            if not near.any():
                assert got[e] == want, (e, hex(got[e]), hex(want))
        assert got[1] == (1 << 64) - 1                # empty event: every region


MASKS = [1 << (3 * 8 + 4),                                # one region, interior
         (1 << 0) | (1 << 63) | (1 << (7 * 8 + 0)),        # corners
         sum(1 << (8 * a + 4) for a in range(8)) | sum(1 << (8 * a + 3) for a in range(2, 6)),
         (1 << 64) - 1]


@pytest.mark.parametrize("name,hits_n", [(C2, 3000), ("single_64", None)])
def test_masked_vote_and_peaks_match_oracle(name, hits_n):
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 21, target_hits=hits_n)
    x, y, z = ev.x, ev.y, ev.z
    acc_o, _ = oracle.vote(g, x, y)
    G = ht.Geometry(g)
    cap = 1 << 20
    dx, dy = to_dev(x), to_dev(y)
    acc = G.new_accumulator()
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    pk = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(G.find_peaks_workspace_size(), dtype=torch.uint8, device="cuda")
    top = 65535 if g["count_bits"] == 16 else 2 ** 31 - 1
    for mask in MASKS:
        dm = torch.tensor([np.int64(np.uint64(mask))], dtype=torch.int64, device="cuda")
        acc.fill_(-1)                                  # unwritten tiles stay visible
        ht.ht_vote_masked(G, dx, dy, dm, acc, stats)
        ht.ht_find_peaks_masked(G, acc, dm, pk, cap, cnt, ws)
        torch.cuda.synchronize()
        m = mlp.masked_event(g, x, y, z, mask, cap=cap, acc=acc_o)
        a = acc.cpu().numpy()
        a = a.view(np.uint16) if a.dtype == np.int16 else a
        halo = m["halo"]
        assert_same_acc(a[halo], np.minimum(acc_o[halo], top))
        assert int(stats[0].item()) == m["votes"]
        k = int(cnt.item())
        assert k == m["count"]
        assert np.array_equal(pk[:k].cpu().numpy(), m["peaks"])
    G.close()


def test_batch_masked_and_learned_runs():
    import torch
    from paper_1309_6275_gb300 import ht
    from gpu_common import gpu_event
    name = "stream2000_256"
    g = synth.geometry_of(name)
    gen = synth.CONFIGS[name]["gen"]
    sizes = [2500, 36000, 4000, 9000]                # one event above 32767 hits
    evs = [synth.make_event(gen, 900 + i, target_hits=h) for i, h in enumerate(sizes)]
    off = np.zeros(len(evs) + 1, np.int32)
    off[1:] = np.cumsum([e.n_hits for e in evs])
    cat = lambda k, t: to_dev(np.concatenate([getattr(e, k) for e in evs]).astype(t))
    x, y, z, layer = cat("x", np.float32), cat("y", np.float32), cat("z", np.float32), cat("layer", np.uint8)
    cap = 1 << 19
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=4, max_hits=int(off[-1]), cap=cap)
    masks = [MASKS[0], MASKS[2], MASKS[3], MASKS[1]]
    dm = torch.tensor([np.int64(np.uint64(m)) for m in masks], dtype=torch.int64, device="cuda")
    B.run_masked(x, y, z, off, dm)
    torch.cuda.synchronize()
    # the smallest event against the oracle
    r = batch_event(B, off, 0)
    o = mlp.masked_event(g, evs[0].x, evs[0].y, evs[0].z, masks[0], cap=cap)
    assert r["count"] == o["count"] and r["votes"] == o["votes"]
    assert np.array_equal(r["peaks"], o["peaks"])
    assert np.array_equal(r["assign"], o["assign"])
    assert np.array_equal(r["zres"], o["zres"])
    # every event against the single-event path restricted to the mask
    full = [gpu_event(g, e.x, e.y, e.z, cap) for e in evs]
    for e, ev in enumerate(evs):
        r = batch_event(B, off, e)
        ins = mlp.cell_allowed(g, masks[e])[0]
        pk = full[e]["peaks"]
        keep = ins[pk[:, 0], pk[:, 1]] if pk.shape[0] else np.zeros(0, bool)
        assert np.array_equal(r["peaks"], pk[keep]), e
        if masks[e] == (1 << 64) - 1:
            assert np.array_equal(r["assign"], full[e]["assign"])
            assert np.array_equal(r["zres"], full[e]["zres"])
    # learned: the masks come from the MLP inside the graph and equal
    # ht_mlp_region_mask's; results equal run_masked with those masks
    p = params(8, 0.1)
    mlp.unpack(p)[5][[4, 12, 20, 28, 36, 44, 52, 60]] += 4.0
    pb = bf16_bits(p).cuda()
    lm = torch.empty(4, dtype=torch.int64, device="cuda")
    for _ in range(2):                              # capture, then replay
        B.run_learned(x, y, z, layer, off, pb, lm, 0.02, 0.6, grow=1)
        torch.cuda.synchronize()
    mass = torch.empty((4, 64), device="cuda")
    ref = torch.empty(4, dtype=torch.int64, device="cuda")
    ht.ht_mlp_region_mask(pb, x, y, z, layer, to_dev(off), 0.02, 0.6, 1, mass, ref)
    torch.cuda.synchronize()
    assert torch.equal(lm, ref)
    res_l = [batch_event(B, off, e) for e in range(4)]
    B.run_masked(x, y, z, off, lm.clone())
    torch.cuda.synchronize()
    for e in range(4):
        r = batch_event(B, off, e)
        for k in ("count", "votes"):
            assert r[k] == res_l[e][k]
        for k in ("peaks", "assign", "zres"):
            assert np.array_equal(r[k], res_l[e][k])
    B.close()
    G.close()


def test_trained_proposal_gain_over_the_plain_path():
    """What the committed, trained network buys on the batched-stream
    workload, judged by assignment-level efficiency on the track path: each
    hit voting only in its top-8 regions casts under a third of the votes,
    and at the learned configuration's thresholds (one layer lower) finds
    tracks within half a point of the plain path's efficiency, with no more
    fakes.  200 events, so that half a point is well above the sampling
    noise."""
    import torch
    from paper_1309_6275_gb300 import ht, learned, quality
    name = "stream2000_256"
    evs = list(synth.make_stream(name, 200, 5000))
    params, meta = learned.load_weights(learned.default_weights_path("event100_256"))
    assert meta["n_events"] >= 100000
    pb = learned.bf16_params(params)
    lcfg = synth.learned_of(name)
    G = ht.Geometry(synth.track_geometry(name))
    Bn = 50
    batches = [evs[i:i + Bn] for i in range(0, len(evs), Bn)]
    mh = max(sum(e.n_hits for e in b) for b in batches)
    B = ht.Batch(G, max_events=Bn, max_hits=mh, cap=1 << 19)
    hm = torch.empty(mh, dtype=torch.int64, device="cuda")

    def run(track, params=None):
        B.set_confirm(track)
        votes, rows = 0, []
        for b in batches:
            off = np.zeros(len(b) + 1, np.int32)
            off[1:] = np.cumsum([e.n_hits for e in b])
            cat = lambda k, t: to_dev(np.concatenate([getattr(e, k) for e in b]).astype(t))
            x, y, z, l = cat("x", np.float32), cat("y", np.float32), cat("z", np.float32), \
                cat("layer", np.uint8)
            if params is None:
                B.run_tracks(x, y, z, l, off)
            else:
                B.run_tracks(x, y, z, l, off, params_bf16=params, hit_masks=hm,
                             topk=lcfg["topk"])
            torch.cuda.synchronize()
            votes += int(B.stats[:2 * len(b)].view(-1, 2)[:, 0].sum())
            asg = B.assign[:int(off[-1])].cpu().numpy()
            for e, ev in enumerate(b):
                rows.append(quality.track_quality(synth.track_geometry(name), ev,
                                                  asg[off[e]:off[e + 1]]))
        return votes, quality.summarize(rows)

    vp, P = run(synth.track_of(name))
    vl, L = run(lcfg["track"], pb)
    assert P["efficiency"] > 0.08 and P["found"] > 1000   # the plain path finds tracks
    assert vl < 0.35 * vp                                  # votes cast
    assert L["efficiency"] >= P["efficiency"] - 0.005      # assignment-level efficiency
    assert L["fake_rate"] <= P["fake_rate"]
    B.close()
    G.close()


def test_training_resumed_from_a_checkpoint_repeats_an_uninterrupted_run(tmp_path):
    """Checkpoint / resume: 2 steps, a checkpoint, then 2 more steps after a
    resume give the same parameter bits as 4 steps in one run (the backward
    pass adds its partial sums in a fixed order, so steps are
    bit-reproducible).  All four steps stay at the constant learning rate of
    the schedule, so the two runs see the same rates."""
    from paper_1309_6275_gb300 import learned
    quiet = lambda *a, **k: None
    a, b = str(tmp_path / "a.npz"), str(tmp_path / "b.npz")
    kw = dict(name=C2, per_chunk=8, ckpt_every=0, workers=2, log=quiet)
    learned.train(n_events=32, out=a, **kw)
    learned.train(n_events=16, out=b, **kw)
    learned.train(n_events=32, out=b, resume=b, **kw)
    pa, ma = learned.load_weights(a)
    pb, mb = learned.load_weights(b)
    assert ma["next_event"] == mb["next_event"] == 32
    assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
