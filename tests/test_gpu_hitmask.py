"""The per-hit region proposal on the GPU against its oracle (oracle/mlp.py
hit_topk_masks, hit_masked_event; oracle vote_hitmask): the restricted vote
bit-exact (whole accumulators, or sampled rho rows at full size), top-k
region sets equal to the oracle's up to near ties, and the batch runs with
given and learned region sets giving the oracle's peaks, assignments and z
results exactly."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_same_acc, batch_event, cuda_ok, to_dev
from oracle import mlp

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C2 = "event100_256"
FULL = (1 << 64) - 1


def random_masks(n, seed, p_full=0.05, p_zero=0.05):
    """Seeded per-hit region sets: mostly one to three random regions, some
    hits with every region and some with none."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, np.uint64)
    u = rng.random(n)
    for h in range(n):
        if u[h] < p_full:
            out[h] = np.uint64(FULL)
        elif u[h] < p_full + p_zero:
            out[h] = np.uint64(0)
        else:
            regs = rng.choice(64, size=rng.integers(1, 4), replace=False)
            out[h] = np.uint64(sum(1 << int(r) for r in regs))
    return out


def dev_masks(m):
    return to_dev(np.asarray(m, np.uint64).view(np.int64))


def gpu_vote(g, x, y, masks):
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    dt = torch.int16 if g.get("count_bits", 32) == 16 else torch.int32
    acc = torch.full((g["n_rho"], g["n_d0"], g["n_phi0"]), -1, dtype=dt, device="cuda")
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    ht.ht_vote_hit_masked(G, to_dev(x), to_dev(y), dev_masks(masks), acc, stats)
    torch.cuda.synchronize()
    a = acc.cpu().numpy()
    if dt == torch.int16:
        a = a.view(np.uint16)
    G.close()
    return a.astype(np.int64), stats.cpu().numpy()


ROWS = [(0, 32), (96, 130), (224, 256)]


@pytest.mark.parametrize("name,n,seed", [("single_64", None, 0), (C2, 3001, 1), (C2, None, 2)])
def test_hit_masked_vote_matches_oracle(name, n, seed):
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], seed)
    x, y = (ev.x, ev.y) if n is None else (ev.x[:n], ev.y[:n])
    masks = random_masks(len(x), seed + 10)
    got, st = gpu_vote(g, x, y, masks)
    if name == "single_64" or n is not None:
        want, ost = oracle.vote_hitmask(g, x, y, masks)
        assert_same_acc(got, want)
        assert int(st[0]) == ost["votes"]
    else:
        for a, b in ROWS:
            want, _ = oracle.vote_hitmask(g, x, y, masks, rows=(a, b))
            assert_same_acc(got[a:b], want)


def test_hit_masked_vote_over_the_packed_limit():
    """40k hits: the unpacked 16-bit tile path, sampled rows."""
    g = synth.geometry_of(C2)
    evs = [synth.make_event(synth.CONFIGS[C2]["gen"], 20 + i) for i in range(4)]
    x = np.concatenate([e.x for e in evs])[:40000]
    y = np.concatenate([e.y for e in evs])[:40000]
    masks = random_masks(len(x), 33)
    got, _ = gpu_vote(g, x, y, masks)
    for a, b in [(0, 16), (120, 136), (240, 256)]:
        want, _ = oracle.vote_hitmask(g, x, y, masks, rows=(a, b))
        assert_same_acc(got[a:b], want)


def test_all_region_masks_give_the_plain_vote_and_empty_masks_nothing():
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(C2)
    ev = synth.make_event(synth.CONFIGS[C2]["gen"], 3)
    x, y = ev.x[:5000], ev.y[:5000]
    full, st = gpu_vote(g, x, y, np.full(len(x), FULL, np.uint64))
    G = ht.Geometry(g)
    acc = torch.zeros((g["n_rho"], g["n_d0"], g["n_phi0"]), dtype=torch.int16, device="cuda")
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    ht.ht_vote(G, to_dev(x), to_dev(y), acc, stats)
    torch.cuda.synchronize()
    assert np.array_equal(full, acc.cpu().numpy().view(np.uint16).astype(np.int64))
    assert int(st[0]) == int(stats[0].item())
    G.close()
    none, st0 = gpu_vote(g, x, y, np.zeros(len(x), np.uint64))
    assert not none.any() and int(st0[0]) == 0
    empty, _ = gpu_vote(g, x[:0], y[:0], np.zeros(0, np.uint64))
    assert not empty.any()


def params_no_azimuth(seed, scale=0.15):
    """Seeded parameters whose first layer ignores the azimuth feature (its
    float32 atan2 may differ by one BF16 step between the two sides), so
    both sides see identical network inputs."""
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, mlp.n_params())
    W1 = mlp.unpack(p)[0]
    W1[4, :] = 0.0
    return p


def bf16_bits(p):
    import torch
    return torch.from_numpy(mlp.bf16(p).astype(np.float32)).to(torch.bfloat16).view(torch.int16)


def oracle_prob(p, x, y, z, layer):
    f = mlp.features(x, y, z, layer)
    _, P, _ = mlp.forward(mlp.bf16(p), f)
    return P


def compare_topk(got, P, k, pmin, tol=1e-5):
    """got: GPU masks; P: oracle probabilities.  Identical sets, except that
    a hit whose k-th and (k+1)-th probabilities, or whose top-k sum and pmin,
    lie within tol may differ.  Returns the indices of hits that differ."""
    want = mlp.hit_topk_masks(P, k, pmin)
    bad = np.flatnonzero(got != want)
    for h in bad:
        s = np.sort(P[h])[::-1]
        near_tie = k < 64 and s[k - 1] - s[k] <= tol * s[0]
        near_pmin = abs(s[:k].sum() - pmin) <= tol
        assert near_tie or near_pmin, (h, hex(int(got[h])), hex(int(want[h])), s[:k + 1])
    return bad


@pytest.mark.parametrize("k,pmin", [(1, 0.0), (2, 0.0), (3, 0.3), (64, 0.0)])
def test_hit_topk_masks_match_oracle(k, pmin):
    import torch
    from paper_1309_6275_gb300 import ht
    ev = synth.make_event(synth.CONFIGS[C2]["gen"], 4)
    n = 4000
    x, y, z = ev.x[:n], ev.y[:n], ev.z[:n]
    layer = ev.layer[:n].astype(np.uint8)
    p = params_no_azimuth(5)
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    ht.ht_mlp_hit_masks(bf16_bits(p).cuda(), to_dev(x), to_dev(y), to_dev(z), to_dev(layer), k,
                        pmin, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    bad = compare_topk(got, oracle_prob(p, x, y, z, layer), k, pmin)
    assert len(bad) <= n // 500
    if k >= 64:
        assert np.all(got == np.uint64(FULL))
    elif pmin == 0.0:
        assert all(bin(int(m)).count("1") == k for m in got)


def batch_events(name, seeds):
    evs = [synth.generate(synth.CONFIGS[name]["gen"], s) for s in seeds]
    off = np.zeros(len(evs) + 1, np.int32)
    off[1:] = np.cumsum([e.n_hits for e in evs])
    cat = lambda k, t: np.concatenate([getattr(e, k) for e in evs]).astype(t)
    return evs, off, cat("x", np.float32), cat("y", np.float32), cat("z", np.float32), \
        cat("layer", np.uint8)


def check_event(B, off, e, res):
    r = batch_event(B, off, e)
    assert r["count"] == res["count"]
    assert np.array_equal(r["peaks"], res["peaks"])
    assert np.array_equal(r["assign"], res["assign"])
    assert np.array_equal(r["zres"], res["zres"])
    assert r["votes"] == res["votes"]


def test_batch_with_given_hit_masks_matches_oracle():
    import torch
    from paper_1309_6275_gb300 import ht
    name = "jets4_256"
    g = synth.geometry_of(name)
    evs, off, x, y, z, _ = batch_events(name, [80, 81, 82])
    masks = random_masks(int(off[-1]), 9, p_full=0.3, p_zero=0.02)
    cap = 1 << 14
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=3, max_hits=int(off[-1]), cap=cap)
    B.run_hit_masked(to_dev(x), to_dev(y), to_dev(z), off, dev_masks(masks))
    torch.cuda.synchronize()
    for e in range(3):
        a, b = off[e], off[e + 1]
        res = mlp.hit_masked_event(g, x[a:b], y[a:b], z[a:b], masks[a:b], cap=cap)
        check_event(B, off, e, res)
    B.close()
    G.close()


def test_learned_hit_batch_matches_oracle_where_the_sets_agree():
    import torch
    from paper_1309_6275_gb300 import ht
    name = "jets4_256"
    g = synth.geometry_of(name)
    evs, off, x, y, z, layer = batch_events(name, [90, 91, 92, 93])
    p = params_no_azimuth(6)
    k, pmin = 3, 0.2
    cap = 1 << 14
    G = ht.Geometry(g)
    B = ht.Batch(G, max_events=4, max_hits=int(off[-1]), cap=cap)
    hm = torch.zeros(int(off[-1]), dtype=torch.int64, device="cuda")
    B.run_learned_hits(to_dev(x), to_dev(y), to_dev(z), to_dev(layer), off, bf16_bits(p).cuda(),
                       hm, k, pmin)
    torch.cuda.synchronize()
    got = hm.cpu().numpy().view(np.uint64)
    P = oracle_prob(p, x, y, z, layer)
    bad = compare_topk(got, P, k, pmin)
    want = mlp.hit_topk_masks(P, k, pmin)
    n_cmp = 0
    for e in range(4):
        a, b = off[e], off[e + 1]
        if np.any((bad >= a) & (bad < b)):
            continue
        res = mlp.hit_masked_event(g, x[a:b], y[a:b], z[a:b], want[a:b], cap=cap)
        check_event(B, off, e, res)
        n_cmp += 1
    assert n_cmp >= 3
    B.close()
    G.close()
