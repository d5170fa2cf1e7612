"""The swept-interval vote (ht_vote_swept) on the GPU against its oracle
(oracle vote_swept): accumulators bit-exact, whole or on sampled rho rows,
on the single-event geometry, the 100-event geometry (packed and 32-bit
output), a coarse phi0 binning, the straight-line geometry and degenerate
sizes."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_same_acc, cuda_ok, to_dev

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C2 = "event100_256"


def gpu_swept(g, x, y):
    import torch
    from paper_1309_6275_gb300 import ht
    G = ht.Geometry(g)
    dt = torch.int16 if g.get("count_bits", 32) == 16 else torch.int32
    acc = torch.full((g["n_rho"], g["n_d0"], g["n_phi0"]), -1, dtype=dt, device="cuda")
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    ht.ht_vote_swept(G, to_dev(np.ascontiguousarray(x, np.float32)),
                     to_dev(np.ascontiguousarray(y, np.float32)), acc, stats)
    torch.cuda.synchronize()
    a = acc.cpu().numpy()
    if dt == torch.int16:
        a = a.view(np.uint16)
    G.close()
    return a.astype(np.int64), stats.cpu().numpy()


def event(name, seed, n=None):
    ev = synth.make_event(synth.CONFIGS[name]["gen"], seed)
    return (ev.x, ev.y) if n is None else (ev.x[:n], ev.y[:n])


def test_single_event_geometry_whole_accumulator():
    g = synth.geometry_of("single_64")
    x, y = event("single_64", 0)
    got, st = gpu_swept(g, x, y)
    want, ost = oracle.vote_swept(g, x, y)
    assert_same_acc(got, want)
    assert int(st[0]) == ost["votes"]


@pytest.mark.parametrize("n,bits", [(3001, 16), (2000, 32)])
def test_event100_geometry_sampled_rows(n, bits):
    g = synth.geometry_of(C2)
    g["count_bits"] = bits
    x, y = event(C2, 1, n)
    got, _ = gpu_swept(g, x, y)
    for a, b in [(0, 16), (100, 140), (240, 256)]:
        want, _ = oracle.vote_swept(g, x, y, rows=(a, b))
        assert_same_acc(got[a:b], want)


def test_coarse_phi0_binning_whole_accumulator():
    """64 phi0 columns over the 100-event geometry's rho and d0 axes (each
    column sweeps several d0 bins for the outer layers)."""
    g = synth.geometry_of(C2)
    g["n_phi0"] = 64
    x, y = event(C2, 2, 6000)
    got, st = gpu_swept(g, x, y)
    want, ost = oracle.vote_swept(g, x, y)
    assert_same_acc(got, want)
    assert int(st[0]) == ost["votes"]


def test_straight_line_geometry_and_degenerate_sizes():
    g = synth.geometry_of(C2, n_rho=1)
    x, y = event(C2, 3, 4000)
    got, _ = gpu_swept(g, x, y)
    want, _ = oracle.vote_swept(g, x, y)
    assert_same_acc(got, want)
    g1 = synth.geometry_of("single_64")
    for n in (0, 1, 255, 257):
        x, y = event("single_64", 4, n)
        got, st = gpu_swept(g1, x, y)
        want, ost = oracle.vote_swept(g1, x, y)
        assert_same_acc(got, want)
        assert int(st[0]) == ost["votes"]


def test_swept_contains_the_point_vote_on_the_gpu():
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(C2)
    x, y = event(C2, 5, 5000)
    sw, _ = gpu_swept(g, x, y)
    G = ht.Geometry(g)
    acc = G.new_accumulator()
    ht.ht_vote(G, to_dev(x), to_dev(y), acc, None)
    torch.cuda.synchronize()
    pt = acc.cpu().numpy().view(np.uint16).astype(np.int64)
    G.close()
    assert np.all(sw[pt > 0] > 0)
