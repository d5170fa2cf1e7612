"""CUDA path vs the oracle, element by element, through the C ABI.

Bars: accumulators bit-exact (votes within 1e-5 of a bin edge included: the
float64 redo reproduces the definition's bits), peak lists, counts,
assignments and (z0, cot theta) results identical.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_common import oracle_sampled_check, assert_same_acc, cuda_ok, gpu_event, oracle_event, to_dev

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def full_check(g, x, y, z, cap=1 << 20, assoc_hits=None, z_all=True):
    r = gpu_event(g, x, y, z, cap)
    acc, st = oracle.vote(g, x, y)
    assert_same_acc(r["acc"], np.minimum(acc, 65535 if g["count_bits"] == 16 else 2**31 - 1))
    assert int(r["stats"][0]) == st["votes"]
    pk, cnt = oracle.peaks(g, acc, cap=cap)
    assert r["count"] == cnt
    assert np.array_equal(r["peaks"], pk)
    sel = np.arange(len(x)) if assoc_hits is None else assoc_hits
    asg = oracle.associate_dense(g, x, y, pk, hit_idx=sel)
    assert np.array_equal(r["assign"][sel], asg)
    if z_all:
        zr = oracle.vote_z(g, x, y, z, asg, pk)
        assert np.array_equal(r["zres"], zr)
    return r, pk, asg


@pytest.mark.parametrize("seed", range(4))
def test_single_event_whole_path(seed):
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], seed)
    g = synth.geometry_of("single_64")
    r, pk, asg = full_check(g, ev.x, ev.y, ev.z)
    assert pk.shape[0] > 0 and (asg >= 0).any()


def test_event100_whole_path():
    ev, g, o = oracle_event("event100_256", 0)
    r = gpu_event(g, ev.x, ev.y, ev.z, 1 << 20)
    assert_same_acc(r["acc"], o["acc"])
    assert int(r["stats"][0]) == o["stats"]["votes"]
    assert r["count"] == o["count"]
    assert np.array_equal(r["peaks"], o["peaks"])
    asg = oracle.associate_dense(g, ev.x, ev.y, o["peaks"])
    assert np.array_equal(r["assign"], asg)
    zr = oracle.vote_z(g, ev.x, ev.y, ev.z, asg, o["peaks"])
    assert np.array_equal(r["zres"], zr)


def test_event100_hit_subset_all_rows():
    """400 hits of a 10k-hit event at the full 256x128x512 geometry."""
    ev = synth.make_event(synth.CONFIGS["event100_256"]["gen"], 7)
    g = synth.geometry_of("event100_256")
    sl = slice(0, 400)
    full_check(g, ev.x[sl], ev.y[sl], ev.z[sl])


def test_pileup_vote_and_peaks():
    """50k hits, 512x256x1024: the whole accumulator and peak list exactly;
    association on a sample of hits; the z vote of sampled candidates."""
    name = "pileup_512"
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 0)
    cap = 1 << 22
    r = gpu_event(g, ev.x, ev.y, ev.z, cap)
    acc, st = oracle.vote(g, ev.x, ev.y)
    assert_same_acc(r["acc"], np.minimum(acc, 65535))
    assert int(r["stats"][0]) == st["votes"]
    oracle_sampled_check(g, ev, r, cap, n_hits=128, n_cands=6, acc=acc)


@pytest.mark.parametrize("hits", [2000, 60000])
def test_stream_event_sizes_whole(hits):
    """Smallest and largest event of the batched stream: the whole
    accumulator and peak list, sampled association and z results."""
    g = synth.geometry_of("stream2000_256")
    gen = synth.CONFIGS["stream2000_256"]["gen"]
    ev = synth.make_event(gen, 11, target_hits=hits)
    cap = 1 << 21
    r = gpu_event(g, ev.x, ev.y, ev.z, cap)
    acc, st = oracle.vote(g, ev.x, ev.y)
    assert_same_acc(r["acc"], np.minimum(acc, 65535))
    assert int(r["stats"][0]) == st["votes"]
    oracle_sampled_check(g, ev, r, cap, acc=acc)


@pytest.mark.parametrize("n", [0, 1, 3, 257])
def test_tiny_and_ragged_hit_counts(n):
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 9)
    g = synth.geometry_of("single_64", threshold=2)
    x = np.resize(ev.x, n).astype(np.float32)
    y = np.resize(ev.y, n).astype(np.float32)
    z = np.resize(ev.z, n).astype(np.float32)
    r, pk, asg = full_check(g, x, y, z)
    if n == 0:
        assert r["count"] == 0 and r["acc"].sum() == 0


def test_odd_rho_axis_with_a_zero_curvature_row():
    """n_rho odd samples rho = 0 exactly: one root per column, straight-line
    arc length in z."""
    g = synth.geometry_of("single_64", n_rho=63, threshold=5)
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 4)
    full_check(g, ev.x, ev.y, ev.z)


def test_small_axes_and_wide_curvature():
    """n_phi0 = 8 (minimum), n_d0 = 16, curvature range that makes outer hits
    turn past a quarter turn (second root in range)."""
    g = dict(n_rho=40, n_d0=16, n_phi0=8, rho_max=0.05, d0_half=10.0, n_z0=32,
             n_cot=16, z0_max=32.0, cot_max=6.5, threshold=3, count_bits=32)
    rng = np.random.default_rng(5)
    n = 300
    r_ = rng.uniform(3, 60, n); ph = rng.uniform(-math.pi, math.pi, n)
    x = (r_ * np.cos(ph)).astype(np.float32); y = (r_ * np.sin(ph)).astype(np.float32)
    z = rng.uniform(-30, 30, n).astype(np.float32)
    full_check(g, x, y, z)


def test_uint16_saturation_and_big_candidates():
    """40k identical hits: cells saturate at 65535; one candidate gets every
    hit, so the z vote takes the shared-histogram path (> 32 hits)."""
    g = synth.geometry_of("event100_256", n_rho=32, n_phi0=64)
    n = 40000
    x = np.full(n, 30.0, np.float32)
    y = np.full(n, 12.5, np.float32)
    z = np.full(n, 3.0, np.float32)
    r = gpu_event(g, x, y, z, 1 << 16)
    acc1, _ = oracle.vote(g, x[:1], y[:1])
    assert_same_acc(r["acc"], np.minimum(acc1 * n, 65535))
    pk, cnt = oracle.peaks(g, np.minimum(acc1 * n, 65535))
    assert r["count"] == cnt and np.array_equal(r["peaks"], pk)
    asg1 = oracle.associate(g, x[:1], y[:1], pk)
    assert np.all(r["assign"] == asg1[0])
    zr = oracle.vote_z(g, x, y, z, np.full(n, asg1[0], np.int32), pk)
    assert np.array_equal(r["zres"], zr)


def test_association_keys_with_counts_above_4095():
    """A normal event plus 5000 copies of one of its hits: cells on that
    hit's curve pass 4095 votes, so association tiles there take the
    sorted-rank keys while the others use index-offset keys."""
    g = synth.geometry_of("single_64", count_bits=16)
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 7)
    rep = 5000
    x = np.concatenate([ev.x, np.full(rep, ev.x[3], np.float32)])
    y = np.concatenate([ev.y, np.full(rep, ev.y[3], np.float32)])
    z = np.concatenate([ev.z, np.full(rep, ev.z[3], np.float32)])
    r, pk, _ = full_check(g, x, y, z)
    assert pk[:, 3].max() > 4095 and (pk[:, 3] < 4096).any()


def test_capacity_truncates_the_candidate_list():
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 2)
    g = synth.geometry_of("single_64", threshold=3)
    cap = 5
    r = gpu_event(g, ev.x, ev.y, ev.z, cap)
    acc, _ = oracle.vote(g, ev.x, ev.y)
    pk, cnt = oracle.peaks(g, acc, cap=cap)
    assert cnt > cap and r["count"] == cnt
    assert np.array_equal(r["peaks"], pk)
    asg = oracle.associate(g, ev.x, ev.y, pk)
    assert np.array_equal(r["assign"], asg)
    assert np.array_equal(r["zres"], oracle.vote_z(g, ev.x, ev.y, ev.z, asg, pk))


def test_vote_z_alone_on_a_seeded_assignment():
    """The z-vote kernels on the oracle's candidates of a 10k-hit event and a
    seeded assignment in which some candidates get far more than 32 hits."""
    import torch
    from paper_1309_6275_gb300 import ht
    ev, g, o = oracle_event("event100_256", 0)
    pk = o["peaks"]
    rng = np.random.default_rng(1)
    m = pk.shape[0]
    asg = rng.integers(-1, m, ev.n_hits).astype(np.int32)
    asg[:3000] = rng.integers(0, 20, 3000)   # 20 candidates with ~150 hits each
    G = ht.Geometry(g)
    cap = m
    out = torch.zeros((cap, 3), dtype=torch.int32, device="cuda")
    cnt = torch.tensor([m], dtype=torch.int32, device="cuda")
    ws = torch.empty(G.vote_z_workspace_size(ev.n_hits, cap), dtype=torch.uint8, device="cuda")
    ht.ht_vote_z(G, to_dev(ev.x), to_dev(ev.y), to_dev(ev.z), to_dev(asg), to_dev(pk), cnt,
                 cap, out, ws)
    got = out.cpu().numpy()
    cand = np.unique(asg[asg >= 0])
    ref = oracle.vote_z(g, ev.x, ev.y, ev.z, asg, pk, cand=cand)
    assert np.array_equal(got[cand], ref)
    empty = np.setdiff1d(np.arange(m), cand)[:1000]
    assert np.all(got[empty] == np.array([-1, -1, 0]))


@pytest.mark.parametrize("name", ["single_64", "event100_256"])
def test_host_buffer_entry_point(name):
    """ht_run_event (host buffers, copies inside) equals the device calls."""
    import torch
    from paper_1309_6275_gb300 import ht
    g = synth.geometry_of(name)
    ev = synth.make_event(synth.CONFIGS[name]["gen"], 3)
    cap = 1 << 20
    r = gpu_event(g, ev.x, ev.y, ev.z, cap)
    G = ht.Geometry(g)
    n = ev.n_hits
    ws = torch.empty(G.event_workspace_size(n, cap), dtype=torch.uint8, device="cuda")
    hp = torch.zeros((cap, 4), dtype=torch.int32).pin_memory()
    hz = torch.zeros((cap, 3), dtype=torch.int32).pin_memory()
    ha = torch.zeros(n, dtype=torch.int32).pin_memory()
    hc = torch.zeros(1, dtype=torch.int32)
    hs = torch.zeros(2, dtype=torch.int64)
    hx, hy, hzz = (torch.from_numpy(a).pin_memory() for a in (ev.x, ev.y, ev.z))
    ht.ht_run_event(G, hx, hy, hzz, ws, hp, cap, hc, ha, hz, hs)
    k = min(int(hc[0]), cap)
    assert int(hc[0]) == r["count"]
    assert np.array_equal(hp[:k].numpy(), r["peaks"])
    assert np.array_equal(ha.numpy(), r["assign"])
    assert np.array_equal(hz[:k].numpy(), r["zres"])
    assert int(hs[0]) == int(r["stats"][0])


@pytest.mark.parametrize("scene", ["single_64_seed0", "straight_50x10", "helices_4"])
def test_fixture_scenes_through_the_c_abi(scene):
    """The GPU path on the oracle's regression scenes (tests/golden/) gives
    the stored results: accumulator hash, votes, peaks, assignments, z."""
    import hashlib
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(here, "oracle_small_scenes.json")) as f:
        want = {d["scene"]: d for d in json.load(f)}[scene]
    for name, g, x, y, z in mg.scenes():
        if name != scene:
            continue
        r = gpu_event(g, x, y, z, 1 << 16)
        acc = np.ascontiguousarray(r["acc"], np.int64)
        assert hashlib.sha256(acc.tobytes()).hexdigest() == want["acc_sha256"]
        assert int(r["stats"][0]) == want["votes"]
        assert r["count"] == want["count"]
        assert r["peaks"].tolist() == want["peaks"]
        assert r["assign"].tolist() == want["assign"]
        assert r["zres"].tolist() == want["zres"]
