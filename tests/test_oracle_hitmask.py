"""Pins of the per-hit region proposal's oracle: the top-k region sets
(oracle/mlp.py hit_topk_masks) and the vote restricted per hit
(oracle vote_hitmask, hit_masked_event)."""
import numpy as np

import oracle
import synth
from oracle import mlp

FULL = np.uint64((1 << 64) - 1)


def small_event(seed=0):
    g = synth.geometry_of("single_64")
    return g, synth.make_event(synth.CONFIGS["single_64"]["gen"], seed)


def test_topk_by_hand():
    p = np.zeros((4, 64))
    p[0, [5, 17, 40]] = [0.5, 0.3, 0.2]
    p[1, [3, 9]] = [0.4, 0.4]            # tie: the smaller index first
    p[1, 60] = 0.2
    p[2, :] = 1.0 / 64                    # all tied: regions 0 .. k-1
    p[3, [1, 2]] = [0.25, 0.25]           # top-2 sum 0.5 < pmin = 0.6: every region
    p[3, 3:] = 0.5 / 61
    m1 = mlp.hit_topk_masks(p, 1)
    assert list(m1[:3]) == [1 << 5, 1 << 3, 1 << 0]
    m2 = mlp.hit_topk_masks(p, 2, pmin=0.6)
    assert m2[0] == (1 << 5) | (1 << 17)
    assert m2[1] == (1 << 3) | (1 << 9)
    assert m2[2] == FULL                  # 2/64 < 0.6
    assert m2[3] == FULL
    m2b = mlp.hit_topk_masks(p, 2, pmin=0.5)
    assert m2b[3] == (1 << 1) | (1 << 2)  # exactly pmin keeps the set
    assert np.all(mlp.hit_topk_masks(p, 64) == FULL)


def test_topk_properties_on_random_probabilities():
    rng = np.random.default_rng(3)
    p = rng.dirichlet(np.full(64, 0.3), size=200)
    for k in (1, 3, 8):
        m = mlp.hit_topk_masks(p, k)
        for h in range(p.shape[0]):
            bits = np.array([(int(m[h]) >> r) & 1 for r in range(64)], bool)
            assert bits.sum() == k
            assert p[h][bits].min() >= p[h][~bits].max()


def test_region_of_cell_centres_matches_the_track_labels():
    # the cell -> region map of the restricted vote (8 (i 8 / n_rho) + j 8 / n_d0)
    # is the labelling map region_of at the cell centres
    for name in ("single_64", "event100_256"):
        g = synth.geometry_of(name)
        _, _, _, rho = oracle.tables(g)
        delta = 2 * g["d0_half"] / g["n_d0"]
        d0 = (np.arange(g["n_d0"]) - g["n_d0"] / 2) * delta
        R, D = np.meshgrid(rho, d0, indexing="ij")
        reg = mlp.region_of(g, R.ravel(), D.ravel()).reshape(R.shape)
        i = np.arange(g["n_rho"])[:, None]
        j = np.arange(g["n_d0"])[None, :]
        assert np.array_equal(reg, (i * 8 // g["n_rho"]) * 8 + j * 8 // g["n_d0"])


def test_full_masks_give_the_plain_vote():
    g, ev = small_event(1)
    acc, st = oracle.vote(g, ev.x, ev.y)
    acc2, st2 = oracle.vote_hitmask(g, ev.x, ev.y, np.full(ev.n_hits, FULL))
    assert np.array_equal(acc, acc2) and st["votes"] == st2["votes"]
    acc0, st0 = oracle.vote_hitmask(g, ev.x, ev.y, np.zeros(ev.n_hits, np.uint64))
    assert not acc0.any() and st0["votes"] == 0


def test_brute_force_sum_of_single_hit_votes_times_their_halo():
    """Sum over hits of (the hit's own plain vote) x (its allowed cells, built
    with array shifts by cell_allowed), against the C loop."""
    g, ev = small_event(2)
    x, y = ev.x[:60], ev.y[:60]
    rng = np.random.default_rng(5)
    masks = np.zeros(x.shape[0], np.uint64)
    for h in range(x.shape[0]):
        regs = rng.choice(64, size=rng.integers(1, 4), replace=False)
        masks[h] = np.uint64(sum(1 << int(r) for r in regs))
    want = np.zeros((g["n_rho"], g["n_d0"], g["n_phi0"]), np.int64)
    inside_only = np.zeros_like(want)
    for h in range(x.shape[0]):
        a, _ = oracle.vote(g, x[h:h + 1], y[h:h + 1], threads=1)
        inside, halo = mlp.cell_allowed(g, int(masks[h]))
        want += a * halo[:, :, None]
        inside_only += a * inside[:, :, None]
    got, st = oracle.vote_hitmask(g, x, y, masks)
    assert np.array_equal(got, want)
    assert st["votes"] == int(want.sum())
    assert np.all(got <= oracle.vote(g, x, y)[0])
    # the halo matters here: the region cells alone give fewer votes
    assert inside_only.sum() < want.sum()


def test_one_shared_mask_equals_the_plain_vote_on_its_halo():
    g, ev = small_event(3)
    m = (1 << 27) | (1 << 28) | (1 << 36)
    acc, _ = oracle.vote(g, ev.x, ev.y)
    got, _ = oracle.vote_hitmask(g, ev.x, ev.y, np.full(ev.n_hits, m, np.uint64))
    _, halo = mlp.cell_allowed(g, m)
    assert np.array_equal(got, acc * halo[:, :, None])


def test_one_shared_mask_keeps_exactly_the_plain_peaks_inside_it():
    """With every hit under the same mask m the restricted accumulator is
    the plain one on m's halo, so its peaks inside m are the plain peaks
    inside m (the per-event proposal's result, masked_event)."""
    g, ev = small_event(4)
    full = oracle.run_event(g, ev.x, ev.y, ev.z)
    regs = (full["peaks"][:, 0] * 8 // g["n_rho"]) * 8 + full["peaks"][:, 1] * 8 // g["n_d0"]
    m = 0
    for r in np.unique(regs)[::2]:                 # every other region holding a peak
        m |= 1 << int(r)
    res = mlp.hit_masked_event(g, ev.x, ev.y, ev.z, np.full(ev.n_hits, m, np.uint64))
    ref = mlp.masked_event(g, ev.x, ev.y, ev.z, m)
    inside, _ = mlp.cell_allowed(g, m)
    pk = res["peaks"]
    keep = inside[pk[:, 0], pk[:, 1]] if pk.shape[0] else np.zeros(0, bool)
    assert ref["peaks"].shape[0] > 3
    assert np.array_equal(pk[keep], ref["peaks"])


def test_row_slices_are_the_full_vote_rows():
    g, ev = small_event(6)
    rng = np.random.default_rng(7)
    masks = rng.integers(0, 2 ** 63, ev.n_hits, dtype=np.int64).astype(np.uint64)
    full, _ = oracle.vote_hitmask(g, ev.x, ev.y, masks)
    part, _ = oracle.vote_hitmask(g, ev.x, ev.y, masks, rows=(20, 37))
    assert np.array_equal(part, full[20:37])
