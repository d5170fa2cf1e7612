"""Write the oracle regression fixtures in this directory.

The paper prints no worked example of the transform (its results are plots),
so the fixtures here are not the paper's values: they are the oracle's own
outputs on three small seeded scenes, written by this script (which calls
only the oracle and the input generators), so that any later change to the
oracle's arithmetic shows up as a failing test and has to be justified.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth   # noqa: E402
from oracle import mlp  # noqa: E402


def scenes():
    """(name, geometry, x, y, z): the scenes the fixtures cover."""
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 0)
    yield "single_64_seed0", g, ev.x, ev.y, ev.z
    # Fig. 3-like straight-line scene: 50 tracks of 10 hits, rho = 0 geometry
    gs = synth.geometry_of("single_64", n_rho=1, n_d0=64, n_phi0=128, d0_half=20.0)
    rng = np.random.default_rng(3)
    xs, ys, zs = [], [], []
    for _ in range(50):
        d0, phi0 = rng.uniform(-15.0, 15.0), rng.uniform(-math.pi, math.pi)
        hx, hy, hz, _, _ = synth.helix_hits(0.0, d0, phi0)
        xs.append(hx); ys.append(hy); zs.append(hz)
    yield ("straight_50x10", gs, np.concatenate(xs).astype(np.float32),
           np.concatenate(ys).astype(np.float32), np.concatenate(zs).astype(np.float32))
    # helices with both signs of curvature and displaced perigees, 100-event geometry
    g2 = synth.geometry_of("event100_256")
    xs, ys, zs = [], [], []
    for rho, d0, phi0, z0, cot in [(0.004, 0.0, 0.7, 1.0, 0.3), (-0.006, 3.1, -2.2, -4.0, 1.2),
                                    (0.0011, -7.5, 2.9, 0.0, -0.8), (-0.009, 12.0, -0.4, 6.0, 2.5)]:
        hx, hy, hz, _, _ = synth.helix_hits(rho, d0, phi0, z0, cot)
        xs.append(hx); ys.append(hy); zs.append(hz)
    yield ("helices_4", g2, np.concatenate(xs).astype(np.float32),
           np.concatenate(ys).astype(np.float32), np.concatenate(zs).astype(np.float32))


def record(name, g, x, y, z):
    r = oracle.run_event(g, x, y, z, threads=1)
    acc = np.ascontiguousarray(r["acc"], np.int64)
    masks = mlp.hit_topk_masks(np.full((x.shape[0], 64), 1.0 / 64), 2)
    acc_h, st_h = oracle.vote_hitmask(g, x, y, masks, threads=1)
    acc_s, st_s = oracle.vote_swept(g, x, y, threads=1)
    return {
        "scene": name, "geometry": g, "n_hits": int(x.shape[0]),
        "hits_sha256": hashlib.sha256(np.concatenate([x, y, z]).astype(np.float32).tobytes()).hexdigest(),
        "votes": r["stats"]["votes"],
        "acc_sha256": hashlib.sha256(acc.tobytes()).hexdigest(),
        "count": int(r["count"]),
        "peaks": r["peaks"].tolist(),
        "assign": np.asarray(r["assign"]).tolist(),
        "zres": np.asarray(r["zres"]).tolist(),
        "hitmask_votes": st_h["votes"],
        "hitmask_acc_sha256": hashlib.sha256(np.ascontiguousarray(acc_h, np.int64).tobytes()).hexdigest(),
        "swept_votes": st_s["votes"],
        "swept_acc_sha256": hashlib.sha256(np.ascontiguousarray(acc_s, np.int64).tobytes()).hexdigest(),
    }


def main():
    out = [record(*s) for s in scenes()]
    with open(os.path.join(HERE, "oracle_small_scenes.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
