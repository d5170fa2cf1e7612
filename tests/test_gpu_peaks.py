"""The peak finder on crafted accumulators, against the oracle: tiles whose
peaks fit the spill slots (the stencil runs once, pass 2 copies), tiles
with more (pass 2 runs the stencil again), the boundary between them,
capacity truncation, masks, and the no-allocation variant (two stencil
passes, no spill) on the same inputs."""
import numpy as np
import pytest

import oracle
from gpu_common import cuda_ok, to_dev

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

# 2 phi0 blocks of 256 columns, 3 blocks of 16 d0 bins: 2 x 3 x 16 = 96 tiles
G0 = dict(n_rho=16, n_d0=48, n_phi0=512, rho_max=0.01, d0_half=2.0, n_z0=16, n_cot=16,
          z0_max=20.0, cot_max=3.0, threshold=5, count_bits=16)
SPILL_Q = 64   # spill slots per tile (one row, 16 bins, 256 columns)


def crafted(seed, dense):
    """Random noise below the threshold plus random isolated peaks, and the
    given dense tiles: (row, first bin, first column, peaks)."""
    rng = np.random.Generator(np.random.Philox(seed))
    acc = rng.integers(0, 5, (G0["n_rho"], G0["n_d0"], G0["n_phi0"])).astype(np.int64)
    for _ in range(300):
        i, j, k = (int(rng.integers(n)) for n in (G0["n_rho"], G0["n_d0"], G0["n_phi0"]))
        acc[i, j, k] = int(rng.integers(5, 40))
    for i, j0, k0, n in dense:
        acc[i, j0:j0 + 16, k0:k0 + 256] = 0
        cells = [(j, k) for j in range(j0, j0 + 16, 2) for k in range(k0, k0 + 256, 2)][:n]
        for j, k in cells:
            acc[i, j, k] = 7 + (j + k) % 5
        # the neighbouring rows must not outvote them
        for ii in (i - 1, i + 1):
            if 0 <= ii < G0["n_rho"]:
                acc[ii, j0:j0 + 16, k0:k0 + 256] = np.minimum(acc[ii, j0:j0 + 16, k0:k0 + 256], 4)
    return acc


def gpu_peaks(g, acc, cap, mask=None, noalloc=False):
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    a = to_dev(acc.astype(np.uint16).view(np.int16))
    pk = torch.full((max(cap, 1), 4), -7, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    if noalloc:
        ht.ht_find_peaks_noalloc(G, a, pk, cap, n)
    else:
        ws = torch.empty(G.find_peaks_workspace_size(), dtype=torch.uint8, device="cuda")
        if mask is None:
            ht.ht_find_peaks(G, a, pk, cap, n, ws)
        else:
            m = torch.tensor([mask - (1 << 64) if mask >= (1 << 63) else mask], dtype=torch.int64,
                             device="cuda")
            ht.ht_find_peaks_masked(G, a, m, pk, cap, n, ws)
    torch.cuda.synchronize()
    cnt = int(n.item())
    out = pk[:min(cnt, cap)].cpu().numpy()
    G.close()
    return out, cnt


@pytest.mark.parametrize("dense", [
    [],                                                    # every tile spilled
    [(5, 16, 256, SPILL_Q)],                               # a tile exactly full
    [(5, 16, 256, SPILL_Q + 1)],                           # one peak over: stencil again
    [(0, 0, 0, 1024), (15, 32, 256, 700), (8, 16, 0, 65)],  # dense tiles at the edges
])
def test_spilled_and_recomputed_tiles_equal_the_oracle(dense):
    acc = crafted(11, dense)
    cap = 1 << 16
    pk_o, cnt_o = oracle.peaks(G0, acc, cap=cap)
    for noalloc in (False, True):
        pk, cnt = gpu_peaks(G0, acc, cap, noalloc=noalloc)
        assert cnt == cnt_o, noalloc
        assert np.array_equal(pk, pk_o), noalloc


def test_truncation_keeps_the_first_peaks_in_index_order():
    acc = crafted(12, [(3, 0, 256, 300), (9, 32, 0, 40)])
    pk_o, cnt_o = oracle.peaks(G0, acc, cap=1 << 16)
    for cap in (1, 37, cnt_o // 2, cnt_o - 1):
        pk, cnt = gpu_peaks(G0, acc, cap)
        assert cnt == cnt_o
        assert np.array_equal(pk, pk_o[:cap])


def test_masked_peaks_with_dense_tiles():
    acc = crafted(13, [(5, 16, 256, 200), (12, 0, 0, 30)])
    rng = np.random.Generator(np.random.Philox(5))
    mask = int(rng.integers(0, 2 ** 63)) | (1 << 63)
    pk, cnt = gpu_peaks(G0, acc, 1 << 16, mask=mask)
    pk_all, _ = oracle.peaks(G0, acc, cap=1 << 16)
    # inside the mask: the cell's region bit (8 x 8 blocks of rows and bins)
    rb = pk_all[:, 0] * 8 // G0["n_rho"]
    db = pk_all[:, 1] * 8 // G0["n_d0"]
    keep = np.array([(mask >> int(8 * r + d)) & 1 for r, d in zip(rb, db)], bool)
    assert cnt == int(keep.sum())
    assert np.array_equal(pk, pk_all[keep])
