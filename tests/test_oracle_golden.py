"""The oracle against its own regression fixtures (tests/golden/): three
small seeded scenes whose outputs tests/golden/make_golden.py wrote from the
oracle.  The paper prints no worked example of the transform, so these pin
the oracle against unintended change, not against the paper; a deliberate
change to the oracle's arithmetic regenerates them and says why."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from oracle import mlp

HERE = os.path.dirname(os.path.abspath(__file__))
sys_path_golden = os.path.join(HERE, "golden")


def load():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(sys_path_golden, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(sys_path_golden, "oracle_small_scenes.json")) as f:
        want = {d["scene"]: d for d in json.load(f)}
    return mg, want


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, np.int64).tobytes()).hexdigest()


@pytest.mark.parametrize("scene", ["single_64_seed0", "straight_50x10", "helices_4"])
def test_oracle_reproduces_its_fixtures(scene):
    mg, want = load()
    w = want[scene]
    for name, g, x, y, z in mg.scenes():
        if name != scene:
            continue
        assert hashlib.sha256(np.concatenate([x, y, z]).astype(np.float32).tobytes()).hexdigest() \
            == w["hits_sha256"], "the scene's inputs changed"
        r = oracle.run_event(g, x, y, z, threads=1)
        assert r["stats"]["votes"] == w["votes"]
        assert sha(r["acc"]) == w["acc_sha256"]
        assert r["count"] == w["count"]
        assert r["peaks"].tolist() == w["peaks"]
        assert np.asarray(r["assign"]).tolist() == w["assign"]
        assert np.asarray(r["zres"]).tolist() == w["zres"]
        masks = mlp.hit_topk_masks(np.full((x.shape[0], 64), 1.0 / 64), 2)
        acc_h, st_h = oracle.vote_hitmask(g, x, y, masks, threads=1)
        assert st_h["votes"] == w["hitmask_votes"] and sha(acc_h) == w["hitmask_acc_sha256"]
        acc_s, st_s = oracle.vote_swept(g, x, y, threads=1)
        assert st_s["votes"] == w["swept_votes"] and sha(acc_s) == w["swept_acc_sha256"]
        return
    raise AssertionError(f"scene {scene} not generated")
