#!/usr/bin/env python3
"""Throughput of the Hough-transform track-finding path on GB300.

One step = the whole path (vote, 3x3x3 peaks, hit association, (z0, cot theta)
vote) over every event of the 100-event workload (~10k hits per event,
256 rho x 128 d0 x 512 phi0 uint16 accumulator, 128 x 128 z grid).  Hits are
synthetic (seeded generator) and resident in HBM before timing; L2 is flushed
(256 MiB write) before every timed step; each step is timed with CUDA events
on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed (one process per GPU, launched by
torch.distributed.run); every rank processes its own 100 events (weak
scaling: events are independent, there is no data-path collective).
--impl reference times the CPU oracle (plain float64 C) on the host cores on
one event per step.  Prints one JSON line on rank 0.
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

WORKLOAD = "event100_256"
METRIC = "events/s"
CAP = 1 << 20          # candidate capacity per event (the 10k-hit events give ~5e5)
KERNELS_PER_EVENT = 11  # vote 1, peaks 3, association 2, z vote 5


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--events", type=int, default=None, help="events per step (default: workload's)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
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


def cpu_baseline(g, ev, cap):
    """The oracle on one event of the workload, on all host cores."""
    import oracle
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.run_event(g, ev.x, ev.y, ev.z, cap=cap, threads=cores)
    dt = time.perf_counter() - t
    return {"value": 1.0 / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"1 event of {ev.n_hits} hits (whole path, float64 C oracle, "
                      f"{cores} threads), {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cfg = synth.CONFIGS[args.workload]
    g = dict(cfg["geom"])
    n_ev = args.events or cfg["events"]
    cores = os.cpu_count() or 1
    evs = [synth.make_event(cfg["gen"], cfg["seed0"] + e) for e in range(min(n_ev, args.warmup + args.steps))]
    for s in range(args.warmup):
        ev = evs[s % len(evs)]
        oracle.run_event(g, ev.x, ev.y, ev.z, cap=CAP, threads=cores)
    times = []
    for s in range(args.steps):
        ev = evs[(args.warmup + s) % len(evs)]
        t = time.perf_counter()
        oracle.run_event(g, ev.x, ev.y, ev.z, cap=CAP, threads=cores)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "events_per_step": 1,
                   "note": "reference arm = plain float64 CPU oracle, one event per step"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} events, one per step, {cores} threads"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1309_6275_gb300 import ht

    cfg = synth.CONFIGS[args.workload]
    g = dict(cfg["geom"])
    n_ev = args.events or cfg["events"]
    seed0 = cfg["seed0"] + rank * 1_000_003
    events = [synth.make_event(cfg["gen"], seed0 + e) for e in range(n_ev)]
    G = ht.Geometry(g)
    max_hits = max(ev.n_hits for ev in events)
    pipe = ht.EventPipeline(G, max_hits, CAP)
    dev_hits = [tuple(torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z)) for ev in events]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    n_hits_total = sum(ev.n_hits for ev in events)

    vote_t0 = [torch.cuda.Event(enable_timing=True) for _ in events]
    vote_t1 = [torch.cuda.Event(enable_timing=True) for _ in events]
    votes_dev = torch.zeros((len(events), 2), dtype=torch.int64, device="cuda")

    def step(timed_vote=False):
        for e, (x, y, z) in enumerate(dev_hits):
            if timed_vote:
                vote_t0[e].record(stream)
            ht.ht_vote(G, x, y, pipe.acc, pipe.stats)
            if timed_vote:
                vote_t1[e].record(stream)
                votes_dev[e] = pipe.stats
            ht.ht_find_peaks(G, pipe.acc, pipe.peaks, CAP, pipe.count, pipe.workspace)
            n = x.numel()
            ht.ht_associate(G, x, y, pipe.peaks, pipe.count, CAP, pipe.assign[:n], pipe.workspace)
            ht.ht_vote_z(G, x, y, z, pipe.assign[:n], pipe.peaks, pipe.count, CAP, pipe.zres,
                         pipe.workspace)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    step_ms, vote_ms = [], []
    votes_total = 0
    redo_total = 0
    for s in range(args.steps):
        flush.fill_(s & 0xff)                          # evict L2 before the step
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(timed_vote=True)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        vote_ms.append(sum(vote_t0[e].elapsed_time(vote_t1[e]) for e in range(len(events))))
        vsum = votes_dev.sum(0).tolist()
        votes_total += int(vsum[0])
        redo_total += int(vsum[1])
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
    value = world * n_ev * args.steps / max_s
    hit_votes_per_s = world * votes_total / max_s

    # ---- e2e: host buffers through ht_run_event (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hcap = CAP
        ws = torch.empty(G.event_workspace_size(max_hits, hcap), dtype=torch.uint8, device="cuda")
        hin = [tuple(torch.from_numpy(a).pin_memory() for a in (ev.x, ev.y, ev.z)) for ev in events]
        hp = torch.empty((hcap, 4), dtype=torch.int32).pin_memory()
        hz = torch.empty((hcap, 3), dtype=torch.int32).pin_memory()
        ha = torch.empty(max_hits, dtype=torch.int32).pin_memory()
        hc = torch.empty(1, dtype=torch.int32).pin_memory()
        h2d = sum(12 * ev.n_hits for ev in events)
        d2h = 0

        def e2e_step():
            nonlocal d2h
            d2h = 0
            for (x, y, z) in hin:
                ht.ht_run_event(G, x, y, z, ws, hp, hcap, hc, ha[:x.numel()], hz)
                k = min(int(hc[0]), hcap)
                d2h += 4 + 4 * x.numel() + 16 * k + 12 * k

        e2e_step()
        torch.cuda.synchronize()
        tt = []
        for s in range(max(1, args.steps)):
            t0 = time.perf_counter()
            e2e_step()
            tt.append(time.perf_counter() - t0)
        et = torch.tensor([sum(tt)], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(et, op=dist.ReduceOp.MAX)
        e2e = {"value": world * n_ev * len(tt) / float(et.item()), "unit": "events/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    atom_rate = ht.ht_probe_shared_atomic_rate(1 << 14)
    vote_s = sum(vote_ms) / 1e3
    achieved = votes_total / vote_s                 # one shared atomic per vote
    roof = {"bound": "alu", "kernel": "k_vote", "achieved": achieved / 1e9,
            "peak": atom_rate / 1e9, "unit": "Gatomic/s", "frac": achieved / atom_rate,
            "traffic": None,
            "peak_source": "measured here: conflict-free shared atomicAdd microbenchmark "
                           "(ht_probe_shared_atomic_rate)",
            "vote_kernel_ms_per_event": 1e3 * vote_s / (args.steps * n_ev),
            "float64_redo_per_vote": redo_total / max(votes_total, 1),
            "vote_share_of_step": vote_s / total_s,
            "hbm_gbs_measured": peaks.get("hbm_gbs")}
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * max_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "events_per_step": n_ev,
                   "hits_per_step": n_hits_total, "accumulator": "256x128x512 uint16",
                   "z_grid": "128x128", "l2": "flushed (256 MiB write) before each timed step",
                   "parallelism": f"events sharded, {world} rank(s), no collective"},
        "hit_votes_per_s": hit_votes_per_s,
        "gpu_launches": KERNELS_PER_EVENT * n_ev * args.steps + args.steps * 0,
        "roofline": roof,
        "clocks": clk,
    }
    if e2e:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, events[0], CAP)
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
