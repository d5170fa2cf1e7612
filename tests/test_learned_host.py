"""Host side of the learned proposal (no GPU): training labels equal the
oracle's, the event generator workers, the efficiency measure and the
checkpoint format."""
import json

import numpy as np

import synth
from oracle import mlp
from paper_1309_6275_gb300 import learned


def test_training_labels_equal_the_oracle_labels():
    for name in ("event100_256", "single_64", "pileup_512"):
        g = synth.geometry_of(name)
        for seed in range(3):
            ev = synth.make_event(synth.CONFIGS[name]["gen"], seed,
                                  target_hits=3000 if name == "pileup_512" else None)
            assert np.array_equal(learned.labels_of(g, ev), mlp.hit_labels(g, ev))


def test_spawned_generator_workers_match_a_serial_run():
    a = list(learned.chunk_stream("single_64", 40, 5, 2, workers=2))
    b = list(learned.chunk_stream("single_64", 40, 5, 2, workers=1))
    assert len(a) == 3
    for u, v in zip(a, b):
        for p, q in zip(u, v):
            assert np.array_equal(p, q)


def test_efficiency_of_truth_like_results():
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 3)
    # candidates at the true cells, every track hit assigned to its track
    NR, ND, NP = g["n_rho"], g["n_d0"], g["n_phi0"]
    delta = 2 * g["d0_half"] / ND
    ti = np.floor((ev.rho + g["rho_max"]) / (2 * g["rho_max"] / NR)).astype(int)
    tj = np.floor(ev.d0 / delta + ND / 2 + 0.5).astype(int)
    tk = np.floor((ev.phi0 + np.pi) / (2 * np.pi / NP)).astype(int) % NP
    peaks = np.stack([ti, tj, tk, ev.n_track_hits], 1).astype(np.int32)
    n_rec, fa, fc = learned.efficiency(g, ev, peaks, ev.track.astype(np.int32))
    assert n_rec > 0 and fc == n_rec
    assert fa == np.sum((ev.n_track_hits >= max(g["threshold"], 5)) &
                        (ev.n_track_hits >= g["threshold"]) &
                        (np.abs(ev.rho) < g["rho_max"]) &
                        (np.abs(ev.d0 / delta + ND / 2 + 0.5 - ND / 2) < ND / 2))
    # nothing assigned, no candidates: nothing found
    assert learned.efficiency(g, ev, peaks[:0], np.full(ev.n_hits, -1, np.int32))[1:] == (0, 0)


def test_checkpoint_round_trip(tmp_path):
    class Fake:
        def state(self):
            return dict(params=np.arange(5, dtype=np.float32), m=np.ones(5, np.float32),
                        v=np.zeros(5, np.float32), step=7)
    path = str(tmp_path / "w.npz")
    learned.save_checkpoint(path, Fake(), dict(workload="event100_256", next_event=56))
    p, meta = learned.load_weights(path)
    assert np.array_equal(p, np.arange(5, dtype=np.float32))
    assert meta == dict(workload="event100_256", next_event=56)
    with np.load(path) as f:
        assert int(f["step"]) == 7 and json.loads(str(f["meta"]))["next_event"] == 56


def test_init_params_layout():
    p = learned.init_params(0)
    assert p.shape == (mlp.n_params(),) and p.dtype == np.float32
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p.astype(np.float64))
    assert not b1.any() and not b2.any() and not b3.any()
    assert abs(W2.std() - np.sqrt(2 / 128)) < 0.01
