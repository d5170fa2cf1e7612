"""Pins of the oracle's peak finder (local maxima, Sections 5-7)."""
import itertools

import numpy as np
import pytest

import oracle


def geom(shape, T):
    return dict(n_rho=shape[0], n_d0=shape[1], n_phi0=shape[2], rho_max=0.01,
                d0_half=10.0, n_z0=8, n_cot=8, z0_max=32.0, cot_max=6.5,
                threshold=T, count_bits=32)


def brute_peaks(acc, T):
    """Independent vectorised statement of the rule: shift the whole array by
    each of the 26 offsets (rho, d0 padded as 'absent', phi0 rolled) and
    compare values with the tie rule on the logical index."""
    NR, ND, NP = acc.shape
    lidx = np.arange(acc.size).reshape(acc.shape)
    ok = acc >= T
    for di, dj, dk in itertools.product((-1, 0, 1), repeat=3):
        if (di, dj, dk) == (0, 0, 0):
            continue
        big = np.full((NR + 2, ND + 2, NP), -1, np.int64)
        bigl = np.full((NR + 2, ND + 2, NP), -1, np.int64)
        big[1:-1, 1:-1] = acc
        bigl[1:-1, 1:-1] = lidx
        nb = np.roll(big, -dk, axis=2)[1 + di:1 + di + NR, 1 + dj:1 + dj + ND]
        nl = np.roll(bigl, -dk, axis=2)[1 + di:1 + di + NR, 1 + dj:1 + dj + ND]
        exists = nl >= 0
        cond = np.where(nl < lidx, acc > nb, acc >= nb)
        ok &= cond | ~exists
    i, j, k = np.nonzero(ok)
    return np.stack([i, j, k, acc[i, j, k]], 1).astype(np.int32)


@pytest.mark.parametrize("seed", range(4))
def test_random_grids_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    shape = (5, 6, 7) if seed % 2 else (4, 9, 3)
    acc = rng.integers(0, 6, shape).astype(np.int64)
    g = geom(shape, 3)
    pk, cnt = oracle.peaks(g, acc)
    ref = brute_peaks(acc, 3)
    assert cnt == ref.shape[0]
    assert np.array_equal(pk, ref)


def test_plateau_keeps_smallest_index_only():
    acc = np.zeros((3, 4, 8), np.int64)
    acc[1, 2, 3:6] = 9          # a line of equal values along phi0
    acc[2, 0, 1] = 8
    acc[2, 1, 1] = 8            # an L-shaped plateau
    acc[2, 1, 2] = 8
    pk, cnt = oracle.peaks(geom(acc.shape, 1), acc)
    assert pk.tolist() == [[1, 2, 3, 9], [2, 0, 1, 8]]


def test_plateau_across_the_phi0_wrap():
    acc = np.zeros((2, 3, 6), np.int64)
    acc[0, 1, 0] = 5
    acc[0, 1, 5] = 5            # neighbours through the wrap; l(k=0) < l(k=5)
    pk, cnt = oracle.peaks(geom(acc.shape, 1), acc)
    assert pk.tolist() == [[0, 1, 0, 5]]
    acc[0, 1, 5] = 6            # now the wrapped neighbour wins
    pk, cnt = oracle.peaks(geom(acc.shape, 1), acc)
    assert pk.tolist() == [[0, 1, 5, 6]]


def test_rho_and_d0_do_not_wrap():
    acc = np.zeros((3, 3, 5), np.int64)
    acc[0, 0, 2] = 4
    acc[2, 2, 2] = 4            # would be a neighbour of [0,0,2] only with wrap
    pk, _ = oracle.peaks(geom(acc.shape, 1), acc)
    assert pk.tolist() == [[0, 0, 2, 4], [2, 2, 2, 4]]


def test_threshold_and_capacity():
    rng = np.random.default_rng(11)
    acc = rng.integers(0, 12, (6, 6, 6)).astype(np.int64)
    for T in (1, 7, 11, 12):
        pk, cnt = oracle.peaks(geom(acc.shape, T), acc)
        assert np.all(pk[:, 3] >= T)
        assert np.array_equal(pk, brute_peaks(acc, T))
    pk_all, cnt = oracle.peaks(geom(acc.shape, 1), acc)
    pk3, cnt3 = oracle.peaks(geom(acc.shape, 1), acc, cap=3)
    assert cnt3 == cnt and cnt > 3
    assert np.array_equal(pk3, pk_all[:3])
    logical = (pk_all[:, 0] * 6 + pk_all[:, 1]) * 6 + pk_all[:, 2]
    assert np.all(np.diff(logical) > 0)
