#!/usr/bin/env python3
"""Throughput of the Hough-transform track finder on GB300.

One step = the whole track path over every event of the batched-stream
workload (2000 events, hit counts log-uniform on [2k, 60k], 256 rho x 128 d0
x 512 phi0 uint16 accumulator, 128 x 128 (z0, cot theta) grid): the
distinct-layer vote, 3x3x3 peaks at each event's band threshold, the
candidate confirmation and hit assignment, and the (z0, cot theta) vote, run
by the batched runtime (ht_batch_run_tracks: persistent queue kernels, CUDA
graph replay, 50 events per batch).  Hits are synthetic (seeded generator)
and resident in HBM before timing (442 MB, larger than L2, which is also
flushed by a 256 MiB write before every timed step); steps are timed with
CUDA events on the launching stream.  Stage times come from CUDA events
recorded inside the graphs, in an untimed pass.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed (one process per GPU); every rank takes
its LPT share of N x 2000 events (weak scaling: events are independent, no
data-path collective).  --impl reference times the float64 CPU oracle on the
host cores, one event of the workload per step.  Prints one JSON line on
rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "stream2000_256"
METRIC = "events/s"
# candidate capacity per event slot: the densest events give ~2e5 peaks at
# their band threshold (10k-hit events at T = 9), the pile-up ones ~1.2e5
CAP_OF = {"stream2000_256": 1 << 19, "event100_256": 1 << 19, "pileup_512": 1 << 21}
BATCH_OF = {"stream2000_256": 50, "event100_256": 25, "pileup_512": 4}
SECONDARY = ("event100_256", "pileup_512")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--events", type=int, default=None, help="events per step (default: workload's)")
    p.add_argument("--batch", type=int, default=None, help="events per ht_batch_run_tracks")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--no-vertex", action="store_true")
    p.add_argument("--no-swept", action="store_true")
    p.add_argument("--topk", type=int, default=None,
                   help="regions per hit of the per-hit proposal (default: the workload's)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(name, events, budget_s=10.0, max_events=16):
    """The oracle's whole track path on all host cores, on a bounded sample of
    the workload: its events in stream order until budget_s has passed (at
    most max_events).  Event sizes vary, so the sample's hit rate is scaled
    to the workload's mean hits per event; the sample's own events/s is given
    beside it."""
    import oracle
    cores = os.cpu_count() or 1
    mean_hits = sum(e.n_hits for e in events) / len(events)
    done, hits, total = 0, 0, 0.0
    for ev in events[:max_events]:
        g = synth.track_geometry(name, ev.n_hits)
        t = time.perf_counter()
        oracle.run_event_tracks(g, ev.x, ev.y, ev.z, ev.layer, cp=synth.track_of(name),
                                cap=CAP_OF.get(name), threads=cores)
        total += time.perf_counter() - t
        done += 1
        hits += ev.n_hits
        if total >= budget_s:
            break
    return {"value": hits / total / mean_hits, "unit": "events/s", "cores": cores,
            "kind": "oracle", "sample_events_per_s": done / total,
            "sample": f"the first {done} events of {name} in stream order ({hits} hits, mean "
                      f"{hits / done:.0f} against the workload's {mean_hits:.0f}; the whole "
                      f"track path: distinct-layer vote, peaks, confirmation, z vote; float64 "
                      f"C oracle, {cores} threads), {total:.1f} s; value = the sample's hits/s "
                      f"over the workload's mean hits per event"}


def run_reference(args):
    """The reference arm: the float64 CPU oracle (the only reference there is:
    the reference directory holds the paper alone), one event per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    name = args.workload
    cfg = synth.CONFIGS[name]
    cores = os.cpu_count() or 1
    n = args.warmup + args.steps
    evs = [synth.generate(cfg["gen"], cfg["seed0"] + e) for e in range(n)]

    def one(ev):
        g = synth.track_geometry(name, ev.n_hits)
        oracle.run_event_tracks(g, ev.x, ev.y, ev.z, ev.layer, cp=synth.track_of(name),
                                cap=CAP_OF.get(name), threads=cores)

    for s in range(args.warmup):
        one(evs[s])
    times = []
    for s in range(args.steps):
        t = time.perf_counter()
        one(evs[args.warmup + s])
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "events_per_step": 1,
                   "note": "reference arm = plain float64 CPU oracle of the track path, one "
                           "event of the workload per step"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} events (hits "
                                   f"{[e.n_hits for e in evs[args.warmup:]]}), one per step, "
                                   f"{cores} threads"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Minimal float32 issue slots of one vote: b, rho*c, D (3 FMA/MUL), rsqrt,
# sqrt(D), q, C, 1/q, d0, bin coordinate, floor, range test, shared atomic.
OPS_PER_VOTE = 13


def alu_peak_ops(dev_props, peaks):
    """Issue-limited float32 lane rate: SMs x 128 lanes x max SM clock."""
    mhz = peaks.get("sm_max_mhz") or 2070.0
    return dev_props.multi_processor_count * 128 * mhz * 1e6


def make_events(name, n_ev, world, rank):
    """This rank's events: the job is world * n_ev seeded events, split over
    the ranks by the LPT partition (weak scaling: about n_ev per rank)."""
    cfg = synth.CONFIGS[name]
    every = [synth.generate(cfg["gen"], cfg["seed0"] + e) for e in range(world * n_ev)]
    if world == 1:
        return list(range(n_ev)), every
    from paper_1309_6275_gb300 import shard
    mine = shard.partition([ev.n_hits for ev in every], world)[rank]
    return mine, [every[e] for e in mine]


class TrackRun:
    """A workload's events as device-resident batches on the track path
    (ht_batch_run_tracks), optionally with the per-hit learned proposal."""

    def __init__(self, ht, name, events, B):
        import torch
        self.ht, self.name, self.events, self.B = ht, name, events, B
        self.g = synth.track_geometry(name)     # per-event thresholds come from the bands
        self.G = ht.Geometry(self.g)
        self.batches = [events[i:i + B] for i in range(0, len(events), B)]
        self.max_hits = max(sum(e.n_hits for e in b) for b in self.batches)
        self.cap = CAP_OF[name]
        self.bt = ht.Batch(self.G, max_events=B, max_hits=self.max_hits, cap=self.cap)
        self.bt.set_confirm(synth.track_of(name))
        self.dev = []
        for b in self.batches:
            off = np.zeros(len(b) + 1, np.int32)
            off[1:] = np.cumsum([e.n_hits for e in b])
            cat = lambda k, t: torch.from_numpy(
                np.concatenate([getattr(e, k) for e in b]).astype(t)).cuda()
            self.dev.append((off, cat("x", np.float32), cat("y", np.float32),
                             cat("z", np.float32), cat("layer", np.uint8)))
        self.hmasks = torch.empty(self.max_hits, dtype=torch.int64, device="cuda")
        self.n_hits = sum(e.n_hits for e in events)

    def run(self, d, params=None, topk=8):
        off, x, y, z, l = d
        if params is None:
            self.bt.run_tracks(x, y, z, l, off)
        else:
            self.bt.run_tracks(x, y, z, l, off, params_bf16=params, hit_masks=self.hmasks,
                               topk=topk)

    def step(self, params=None, topk=8):
        for d in self.dev:
            self.run(d, params, topk)

    def time_steps(self, steps, warmup, flush, params=None, topk=8):
        """CUDA-event time (ms) of each of `steps` steps after `warmup`."""
        import torch
        for _ in range(warmup):
            self.step(params, topk)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        out = []
        for s in range(steps):
            flush.fill_(s & 0xff)                      # evict L2 before the step
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            self.step(params, topk)
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    def profile(self, params=None, topk=8):
        """One untimed pass, batch by batch: stage ms, votes, float64 redos,
        candidates, confirmed candidates and track-finding quality."""
        import torch
        from paper_1309_6275_gb300 import quality
        stages = np.zeros(5)
        votes = redo = cands = conf = 0
        rows = []
        for d, b in zip(self.dev, self.batches):
            self.run(d, params, topk)
            torch.cuda.synchronize()
            stages += np.array(self.bt.stage_ms())
            ne = len(b)
            st = self.bt.stats[:2 * ne].view(-1, 2).sum(0).tolist()
            votes += int(st[0])
            redo += int(st[1])
            cnt = self.bt.counts[:ne].cpu().numpy()
            cands += int(cnt.sum())
            score = self.bt.score[:ne * self.cap].view(ne, self.cap)
            conf += int((score > 0).sum().item())
            off = d[0]
            asg = self.bt.assign[:int(off[-1])].cpu().numpy()
            for e, ev in enumerate(b):
                rows.append(quality.track_quality(self.g, ev, asg[off[e]:off[e + 1]]))
        q = quality.summarize(rows)
        n = len(self.events)
        return dict(stage_ms=stages, votes=votes, redo=redo,
                    candidates_per_event=cands / n, confirmed_per_event=conf / n,
                    quality={k: q[k] for k in ("n_rec", "found", "efficiency", "track_cands",
                                               "fakes", "fake_rate", "duplicates",
                                               "duplicate_rate")})

    def close(self):
        self.bt.close()
        self.G.close()


def e2e_run(tr, steps):
    """End to end through the host-buffer C call (ht_batch_run_tracks_host):
    every step copies each batch's hits from pinned host memory, runs the
    track path and copies back the found tracks and the hits' assignments.
    Returns the JSON object and the per-event quality of the last step."""
    import torch
    from paper_1309_6275_gb300 import quality
    hin = []
    for b in tr.batches:
        off = np.zeros(len(b) + 1, np.int32)
        off[1:] = np.cumsum([e.n_hits for e in b])
        cat = lambda k, t: torch.from_numpy(
            np.concatenate([getattr(e, k) for e in b]).astype(t)).pin_memory()
        hin.append((off, cat("x", np.float32), cat("y", np.float32), cat("z", np.float32),
                    cat("layer", np.uint8)))
    tcap = tr.B * 16384
    tracks = torch.zeros((tcap, 8), dtype=torch.int32).pin_memory()
    ntr = torch.zeros(tr.B, dtype=torch.int32).pin_memory()
    asg = torch.zeros(tr.max_hits, dtype=torch.int32).pin_memory()
    h2d = d2h = 0

    def one_step(keep=None):
        nonlocal h2d, d2h
        h2d = d2h = 0
        for i, (off, x, y, z, l) in enumerate(hin):
            ne, nh = len(off) - 1, int(off[-1])
            ok = tr.bt.run_tracks_host(x, y, z, l, off, tracks, ntr, asg)
            assert ok, "track capacity exceeded"
            nt = int(ntr[:ne].sum())
            h2d += 13 * nh
            d2h += 32 * nt + 4 * nh + 4 * (ne + 1)
            if keep is not None:
                a = asg[:nh].numpy().copy()
                for e, ev in enumerate(tr.batches[i]):
                    keep.append(quality.track_quality(tr.g, ev, a[off[e]:off[e + 1]]))

    rows = []
    one_step(rows)                       # warm-up, and the quality of what the caller gets
    tt = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        one_step()
        tt.append(time.perf_counter() - t0)
    q = quality.summarize(rows)
    return {"value": len(tr.events) * len(tt) / sum(tt), "unit": "events/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "ht_batch_run_tracks_host: pinned host hits in, found tracks and hit "
                   "assignments out, synchronous per batch of "
                   f"{tr.B} events",
            "efficiency": q["efficiency"], "fake_rate": q["fake_rate"]}


STAGES = ["proposal", "vote", "peaks", "confirmation+assignment", "z vote"]


def learned_leg(args, tr, plain, flush):
    """The learned proposal on the track path against the plain track path,
    on the same events (the learned configuration's evaluation: the batched
    stream): each hit votes only in its network's top-k regions (computed in
    the same graph by the tcgen05 forward pass); peaks, confirmation and the
    z vote are unchanged.  Two thresholds: the learned configuration's own
    (one layer lower: the restricted vote lacks most background votes) and
    the plain path's.  Events/s (same timing rules as the headline) and
    assignment-level efficiency, fakes, votes and candidates of each."""
    from paper_1309_6275_gb300 import learned
    path = learned.default_weights_path("event100_256")
    lcfg = synth.learned_of(tr.name)
    if not os.path.exists(path) or lcfg is None:
        return None
    params, meta = learned.load_weights(path)
    pb = learned.bf16_params(params)
    topk = args.topk if args.topk is not None else lcfg["topk"]
    n = len(tr.events)
    P = plain["quality"]

    def measure(track):
        tr.bt.set_confirm(track)
        ms = tr.time_steps(max(1, args.steps), max(1, args.warmup), flush, params=pb, topk=topk)
        prof = tr.profile(params=pb, topk=topk)
        L = prof["quality"]
        return {"value": n * len(ms) / (sum(ms) / 1e3), "efficiency": L["efficiency"],
                "difference_points": 100.0 * (L["efficiency"] - P["efficiency"]),
                "fake_rate": L["fake_rate"], "quality": L,
                "vote_frac": prof["votes"] / max(plain["votes"], 1),
                "candidate_frac": prof["candidates_per_event"] /
                                  max(plain["candidates_per_event"], 1),
                "stage_ms_per_event": [round(v / n, 4) for v in prof["stage_ms"]],
                "bands": track["bands"]}

    own = measure(lcfg["track"])
    same = measure(synth.track_of(tr.name))
    tr.bt.set_confirm(synth.track_of(tr.name))
    return {"value": own["value"], "unit": "events/s", "plain_value": plain["value"],
            "speedup": own["value"] / plain["value"],
            "workload": f"{tr.name}: the headline's {n} events",
            "efficiency": {"plain": P["efficiency"], "learned": own["efficiency"],
                           "difference_points": own["difference_points"]},
            "fake_rate": {"plain": P["fake_rate"], "learned": own["fake_rate"]},
            "quality": {"plain": P, "learned": own["quality"]},
            "vote_frac": own["vote_frac"], "candidate_frac": own["candidate_frac"],
            "stage_ms_per_event": {"stages": STAGES,
                                   "plain": [round(v / n, 4) for v in plain["stage_ms"]],
                                   "learned": own["stage_ms_per_event"]},
            "thresholds": {"plain": synth.track_of(tr.name)["bands"], "learned": own["bands"]},
            "at_plain_thresholds": {k: same[k] for k in ("value", "efficiency",
                                                         "difference_points", "fake_rate",
                                                         "vote_frac", "candidate_frac")},
            "topk": topk, "pmin": 0.0,
            "path": "ht_batch_run_tracks with a per-hit proposal (MLP top-k per hit, then the "
                    "per-hit restricted distinct-layer vote, in one graph)",
            "weights": os.path.relpath(path, ROOT),
            "trained_on": f"{meta.get('n_events')} {meta.get('workload')} events"}


def secondary_leg(args, ht, name, flush):
    """Another configuration on the track path: events/s, hit-votes/s, stage
    split, vote roofline fraction and track-finding quality."""
    import torch
    cfg = synth.CONFIGS[name]
    evs = [synth.generate(cfg["gen"], cfg["seed0"] + e) for e in range(cfg["events"])]
    tr = TrackRun(ht, name, evs, BATCH_OF[name])
    ms = tr.time_steps(max(1, args.steps), max(1, args.warmup), flush)
    prof = tr.profile()
    n = len(evs)
    t = sum(ms) / 1e3
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak_ops = alu_peak_ops(props, measured_peaks())
    vote_s = prof["stage_ms"][1] / 1e3
    g = tr.g
    tk = synth.track_of(name)
    out = {"value": n * len(ms) / t, "unit": "events/s", "events": n,
           "hits_per_event": tr.n_hits / n,
           "hit_votes_per_s": prof["votes"] / (prof["stage_ms"].sum() / 1e3),
           "geometry": f"{g['n_rho']}x{g['n_d0']}x{g['n_phi0']} uint16, T={tk['threshold']} "
                       f"layers, pool {tk['pool']}, {tk['min_layers']} inlier layers within "
                       f"{tk['tol'] * 1e4:.0f} um",
           "stage_ms_per_event": {s: round(v / n, 4) for s, v in zip(STAGES, prof["stage_ms"])},
           "vote_alu_frac": OPS_PER_VOTE * prof["votes"] / vote_s / peak_ops,
           "candidates_per_event": prof["candidates_per_event"],
           "confirmed_per_event": prof["confirmed_per_event"],
           "quality": prof["quality"],
           "path": f"ht_batch_run_tracks, {tr.B} events per batch"}
    tr.close()
    return out


def swept_leg(args):
    """Swept-interval phi0 vote against the point vote on the single-event
    workload (200 events of ~275 hits), at its own 64 phi0 columns and at
    256: device ms per event for the vote alone and for the whole
    single-event path (vote, peaks, association, z vote), votes cast,
    candidates, and track-finding efficiency."""
    import torch
    from paper_1309_6275_gb300 import ht, learned
    name = "single_64"
    evs = [synth.make_event(synth.CONFIGS[name]["gen"], 1000 + i) for i in range(200)]
    out = {}
    for n_phi0 in (64, 256):
        g = synth.geometry_of(name, n_phi0=n_phi0)
        G = ht.Geometry(g)
        P = ht.EventPipeline(G, max(e.n_hits for e in evs), 1 << 16)
        dev = [tuple(torch.from_numpy(getattr(e, k)).cuda() for k in ("x", "y", "z"))
               for e in evs]
        res = {}
        for swept in (False, True):
            vote = ht.ht_vote_swept if swept else ht.ht_vote
            for _ in range(max(3, args.warmup)):
                P.run(*dev[0], swept=swept)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for x, y, _z in dev:
                vote(G, x, y, P.acc, P.stats)
            b.record()
            b.synchronize()
            vote_ms = a.elapsed_time(b) / len(dev)
            q = np.zeros(5)
            t = 0.0
            for e, (x, y, z) in zip(evs, dev):
                a.record()
                P.run(x, y, z, swept=swept)
                b.record()
                b.synchronize()
                t += a.elapsed_time(b)
                r = P.results(e.n_hits)
                nr, fa, fc = learned.efficiency(g, e, r["peaks"], r["assign"])
                q += [nr, fa, fc, int(r["stats"][0]), r["count"]]
            res["swept" if swept else "point"] = {
                "vote_ms_per_event": round(vote_ms, 4), "path_ms_per_event": round(t / len(dev), 4),
                "eff_candidate": q[2] / max(q[0], 1), "eff_assign": q[1] / max(q[0], 1),
                "votes_per_event": q[3] / len(dev), "candidates_per_event": q[4] / len(dev)}
        out[f"n_phi0_{n_phi0}"] = res
        G.close()
    return {"workload": f"{name}: 200 events of ~275 hits, 64x64xN int32, one event per call",
            "path": "ht_vote_swept then ht_find_peaks, ht_associate, ht_vote_z", **out}


def vertex_leg(args):
    """Displaced-jet finding on the 4-jet workload (100 events of ~400 hits):
    the batched first transform, then the second transform over its
    candidates.  Events/s of the pair, the second transform's share of the
    device time (the paper quotes about +30% for its version), vertex
    efficiency and fakes per event."""
    import torch
    from paper_1309_6275_gb300 import displaced
    name = "jets4_256"
    cfg = synth.CONFIGS[name]
    g, vd = dict(cfg["geom"]), cfg["vertex"]
    evs = [synth.generate(cfg["gen"], cfg["seed0"] + e) for e in range(cfg["events"])]
    B = 25
    batches = [evs[i:i + B] for i in range(0, len(evs), B)]
    dev_in = []
    for b in batches:
        off = np.zeros(len(b) + 1, np.int32)
        off[1:] = np.cumsum([ev.n_hits for ev in b])
        dev_in.append((off, [torch.from_numpy(np.concatenate([getattr(ev, k) for ev in b])).cuda()
                             for k in "xyz"]))
    pipe = displaced.DisplacedJetPipeline(g, vd, B, max(int(o[-1]) for o, _ in dev_in))
    for off, (x, y, z) in dev_in:
        pipe.run(x, y, z, off)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t1 = t2 = 0.0
    steps = max(1, args.steps)
    for _ in range(steps):
        for off, (x, y, z) in dev_in:
            ev3 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev3[0].record(stream)
            pipe.B.run(x, y, z, off)
            ev3[1].record(stream)
            pipe.V.run(pipe.B.peaks, pipe.B.counts, pipe.cap, len(off) - 1)
            ev3[2].record(stream)
            ev3[2].synchronize()
            t1 += ev3[0].elapsed_time(ev3[1]) / 1e3
            t2 += ev3[1].elapsed_time(ev3[2]) / 1e3
    jets = found = fakes = 0
    # candidate refinement (least-squares circle fit) after the first transform
    from paper_1309_6275_gb300 import ht
    cap = pipe.cap
    fit_out = torch.zeros(B * cap * 64, dtype=torch.uint8, device="cuda")
    fit_ws = torch.empty(ht.ht_fit_workspace_size(B, cap, max(int(o[-1]) for o, _ in dev_in)),
                         dtype=torch.uint8, device="cuda")
    t_fit, n_fit, res_d0, res_rho = 0.0, 0, [], []
    for (off, (x, y, z)), b in zip(dev_in, batches):
        pipe.run(x, y, z, off)
        d_off = torch.from_numpy(off).cuda()
        a, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ht.ht_fit_tracks(pipe.G, x, y, d_off, pipe.B.assign, pipe.B.peaks, pipe.B.counts, cap,
                         fit_out, fit_ws, road=0.5, cut=5.0)
        e_.record(stream)
        e_.synchronize()
        t_fit += a.elapsed_time(e_) / 1e3
        for e, ev in enumerate(b):
            nj, nf, nk = displaced.match(vd, ev, pipe.kept(e))
            jets += nj; found += nf; fakes += nk
            r = pipe.B.event_results(off, e)
            tr = ht.tracks_to_numpy(fit_out[e * cap * 64:], r["count"])
            nfit, rd, rr = displaced.fit_quality(ev, r["assign"], tr)
            n_fit += nfit
            res_d0 += list(rd); res_rho += list(rr)
    pipe.close()
    res_d0, res_rho = np.array(res_d0), np.array(res_rho)
    return {"workload": name, "events": len(evs), "value": len(evs) * steps / (t1 + t2),
            "unit": "events/s", "first_transform_ms_per_event": 1e3 * t1 / (steps * len(evs)),
            "second_transform_ms_per_event": 1e3 * t2 / (steps * len(evs)),
            "second_transform_share": t2 / (t1 + t2),
            "vertex_efficiency": found / max(jets, 1), "fakes_per_event": fakes / len(evs),
            "refit": {"ms_per_event": 1e3 * t_fit / len(evs),
                      "fitted_per_event": n_fit / len(evs),
                      "one_track_fits": int(res_d0.size),
                      "d0_resolution_cm": float(np.median(np.abs(res_d0))) if res_d0.size else None,
                      "rho_resolution_per_cm": float(np.median(np.abs(res_rho)))
                      if res_rho.size else None,
                      "cell_d0_half_width_cm": g["d0_half"] / g["n_d0"],
                      "path": "ht_fit_tracks (min 4 hits, 0.5 cm road, 5 Gauss-Newton "
                              "steps, 5 sigma cut, 3 more steps, float64)"},
            "vertex_space": f"{vd['n_r']} x {vd['n_theta']}, T2={vd['threshold']}, "
                            f"min_count={vd['min_count']}, beam pipe {vd['r_keep']} cm",
            "path": "ht_batch_run then ht_vertex_vote + ht_vertex_find, 25 events per batch"}


# DRAM bytes (read + write) per event of the dominant kernel, from one ncu
# capture of a smaller case (8 stream events in one launch: the traffic is
# the accumulator write-back plus the hits and hit lists, in proportion to
# the events); reported only while the kernel's sources hash to the same value.
PROFILED_TRAFFIC = {"k_vote_batch": {"sha": "c8576bebcabab381",
                                     "bytes_per_event": (78121216 + 293925632) / 8}}
KERNEL_SOURCES = ["paper_1309_6275_gb300/csrc/k_vote_layers.cu",
                  "paper_1309_6275_gb300/csrc/tiles.cuh",
                  "paper_1309_6275_gb300/csrc/ht_internal.cuh",
                  "paper_1309_6275_gb300/csrc/df32.cuh"]


def kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def launches_per_batch(ne, learned=False):
    """Kernels one ht_batch_run_tracks replays: hit lists (count, 3-kernel
    scan, fill), the vote, per event two peak passes and a 3-kernel scan,
    the confirmation (prefix, grouping 2 + scan 3, hit index 3 + scan 3,
    confirmation, offers, decode) and the z vote (4 + scan 3); with the
    proposal one more (the network's top-k per hit)."""
    return 5 + 1 + 5 * ne + 15 + 7 + (1 if learned else 0)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1309_6275_gb300 import ht

    name = args.workload
    n_ev = args.events or synth.CONFIGS[name]["events"]
    B = args.batch or BATCH_OF.get(name, 50)
    ids, events = make_events(name, n_ev, world, rank)
    n_job = world * n_ev
    n_ev = len(events)
    tr = TrackRun(ht, name, events, B)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        tr.step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(1.5)          # let nvidia-smi's start-up pass before the timed region
    step_ms = tr.time_steps(args.steps, 0, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop() if rank == 0 else None
    total_s = sum(step_ms) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_s = float(t.item())
    value = n_job * args.steps / max_s

    plain = tr.profile()
    plain["value"] = n_ev * args.steps / total_s

    # per-event track counts to rank 0 (the only collective; outside the timing)
    from paper_1309_6275_gb300 import shard
    mine = {}
    for d, b, base in zip(tr.dev, tr.batches, range(0, n_ev, B)):
        tr.run(d)
        ne = len(b)
        score = tr.bt.score[:ne * tr.cap].view(ne, tr.cap)
        conf = (score > 0).sum(1).cpu().tolist()
        for i in range(ne):
            mine[int(ids[base + i])] = int(conf[i])
    gathered = shard.gather_results(mine)

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(tr, args.steps)
        et = torch.tensor([n_ev / e2e["value"]], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(et, op=dist.ReduceOp.MAX)
        e2e["value"] = n_job / float(et.item())

    if rank != 0:
        tr.close()
        if dist:
            dist.destroy_process_group()
        return

    learned_res = None if args.no_learned else learned_leg(args, tr, plain, flush)
    secondary = {}
    if not args.no_secondary:
        for nm in SECONDARY:
            if nm != name:
                secondary[nm] = secondary_leg(args, ht, nm, flush)
    swept_res = None if args.no_swept else swept_leg(args)
    vertex_res = None if args.no_vertex else vertex_leg(args)

    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    peak_ops = alu_peak_ops(props, peaks)
    stage_s = plain["stage_ms"] / 1e3
    dom = int(np.argmax(stage_s))
    votes = plain["votes"]
    g = tr.g
    cells = g["n_rho"] * g["n_d0"] * g["n_phi0"]
    roof = {"kernel": {1: "k_vote_batch (distinct-layer mode)", 3: "k_confirm"}.get(dom, STAGES[dom]),
            "stage_ms_per_event": {s: round(1e3 * v / n_ev, 4) for s, v in zip(STAGES, stage_s)}}
    if dom == 1:
        achieved = OPS_PER_VOTE * votes / stage_s[1]
        prof = PROFILED_TRAFFIC.get("k_vote_batch")
        from paper_1309_6275_gb300 import probe
        atom = probe.shared_atomic_rate(1 << 14)
        roof.update({"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9,
                     "unit": "Gop/s", "frac": achieved / peak_ops,
                     "traffic": (prof["bytes_per_event"] * B
                                 if prof and prof["sha"] == kernel_sha() else None),
                     "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 "
                                    f"lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                                    f"(issue-limited), {OPS_PER_VOTE} algorithmic ops per vote",
                     "shared_atomic_frac": (votes / stage_s[1]) / atom,
                     "shared_atomic_peak_gops": atom / 1e9})
    else:
        roof.update({"bound": "alu", "achieved": None, "peak": peak_ops / 1e9, "unit": "Gop/s",
                     "frac": None, "traffic": None,
                     "note": "the dominant stage is not the vote; its work has no "
                             "algorithmic op count here"})
    roof["float64_redo_per_vote"] = plain["redo"] / max(votes, 1)
    roof["hbm_peaks_stage"] = {
        "algorithmic_bytes_per_event": cells * 2,
        "achieved_gbs": cells * 2 / (stage_s[2] / n_ev) / 1e9,
        "peak_gbs": peaks.get("hbm_gbs", 6800.0),
        "frac": cells * 2 / (stage_s[2] / n_ev) / 1e9 / peaks.get("hbm_gbs", 6800.0),
        "note": "the count pass reads each uint16 accumulator once and spills its peaks; the "
                "write pass copies them (tiles with more than 64 peaks are read again)"}
    tk = synth.track_of(name)
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * max_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded detector MC)",
        "config": {"workload": name, "events_per_step": n_job, "hits_per_step": tr.n_hits,
                   "geometry": f"{g['n_rho']}x{g['n_d0']}x{g['n_phi0']} uint16, "
                               f"{g['n_z0']}x{g['n_cot']} z grid",
                   "track": {"threshold_bands": tk["bands"], "threshold_else": tk["threshold"],
                             "pool": tk["pool"], "min_layers": tk["min_layers"],
                             "tol_cm": tk["tol"]},
                   "path": f"ht_batch_run_tracks, {B} events per batch, CUDA graph replay",
                   "l2": "inputs larger than L2, and flushed (256 MiB write) before each timed step",
                   "parallelism": f"events sharded (LPT by hits), {world} rank(s), no data-path "
                                  "collective; per-event track counts gathered to rank 0 "
                                  "after timing"},
        "hit_votes_per_s": world * votes / (plain["stage_ms"].sum() / 1e3),
        "step_ms": [round(v, 3) for v in step_ms],
        "gpu_launches": args.steps * sum(launches_per_batch(len(b)) for b in tr.batches),
        "candidates_per_event": plain["candidates_per_event"],
        "confirmed_per_event": plain["confirmed_per_event"],
        "quality": plain["quality"],
        "roofline": roof,
        "clocks": clk,
    }
    if gathered is not None:
        line["events_gathered"] = len(gathered)
    if e2e:
        line["e2e"] = e2e
    if learned_res:
        line["learned"] = learned_res
    line.update(secondary)
    if swept_res:
        line["swept_vote"] = swept_res
    if vertex_res:
        line["displaced_jets"] = vertex_res
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, events)
    tr.close()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
