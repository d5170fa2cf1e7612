"""ht_find_peaks_noalloc: peak finding for callers that cannot allocate.

Some callers may not call cudaMalloc -- trigger code that must not allocate
once data taking has started, or plug-ins inside a host framework that owns
all device memory -- so the library offers this variant of ht_find_peaks
whose scratch is a fixed array inside the library instead of a caller-owned
workspace.  It must give exactly what ht_find_peaks gives, also on a second
call right after the first (the array still holds the first call's contents),
and refuse geometries whose scratch would not fit.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import synth
from gpu_common import cuda_ok, to_dev

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def test_noalloc_peaks_equal_workspace_peaks_on_two_calls():
    import torch
    from paper_1309_6275_gb300 import ht
    name = "event100_256"
    g = synth.geometry_of(name)
    G = ht.Geometry(g)
    cap = 1 << 20
    acc = G.new_accumulator()
    ws = torch.empty(G.find_peaks_workspace_size(), dtype=torch.uint8, device="cuda")
    pk_ref = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    pk_new = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    n_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
    n_new = torch.zeros(1, dtype=torch.int32, device="cuda")
    for seed in (21, 22):                      # two calls in a row, different events
        ev = synth.make_event(synth.CONFIGS[name]["gen"], seed)
        ht.ht_vote(G, to_dev(ev.x), to_dev(ev.y), acc)
        ht.ht_find_peaks(G, acc, pk_ref, cap, n_ref, ws)
        pk_new.fill_(-7)
        n_new.fill_(-7)
        ht.ht_find_peaks_noalloc(G, acc, pk_new, cap, n_new)
        torch.cuda.synchronize()
        cnt = int(n_ref.item())
        assert cnt > 1000
        assert int(n_new.item()) == cnt
        k = min(cnt, cap)
        assert np.array_equal(pk_new[:k].cpu().numpy(), pk_ref[:k].cpu().numpy())
    G.close()


def test_noalloc_peaks_refuse_geometries_beyond_the_scratch():
    from paper_1309_6275_gb300 import ht
    g = dict(n_rho=4096, n_d0=512, n_phi0=256, rho_max=0.01, d0_half=10.0, n_z0=64,
             n_cot=64, z0_max=32.0, cot_max=6.5, threshold=7, count_bits=16)
    G = ht.Geometry(g)                          # 2^21 segments, above the 2^19 limit
    import torch
    acc = torch.empty(8, dtype=torch.int16, device="cuda")     # never touched
    pk = torch.empty((1, 4), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ht.HTError, match="524288 segments"):
        ht.ht_find_peaks_noalloc(G, acc, pk, 1, n)
    G.close()
