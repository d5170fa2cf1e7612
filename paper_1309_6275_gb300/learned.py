"""Learned region proposal: training with the library's own MLP kernels and
evaluation of the proposal-restricted path against the plain one.

The paper has no learned part.  This is the proposal's reading: a per-hit
network (ht_mlp_* in include/ht.h) predicts which of 64 (rho, d0) regions
an 8 x 8 grid of blocks over the accumulator's rho rows and d0 bins holds
the hit's track; an event's mask keeps the regions whose mean softmax mass
over its hits reaches tau, and the vote and peak finding of Sections 5-7 run
only there (ht_batch_run_learned), with the full vote as the fallback.

Training data: events from the seeded generator (synth), generated on host
cores in spawned worker processes.  Label of a hit: the region of its
track's true (rho, d0), binned exactly as the vote bins a cell (row
floor((rho + rho_max) / (2 rho_max / n_rho)), bin floor(d0 / delta + n_d0/2
+ 1/2)); noise hits and tracks outside the axes get -1 and are left out of
the loss.  Every arithmetic step of training (forward, backward, weight
gradients, Adam) runs in the library's kernels; this module only moves
data and keeps the checkpoint.

Command line:
  python -m paper_1309_6275_gb300.learned train --events 200000 --out W.npz
  python -m paper_1309_6275_gb300.learned evaluate --weights W.npz
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
WEIGHTS_DIR = os.path.join(HERE, "weights")
N_REGIONS = 64


def default_weights_path(name="event100_256"):
    return os.path.join(WEIGHTS_DIR, f"proposal_{name}.npz")


# --------------------------------------------------------------- labels
def region_of(g, rho, d0):
    """Region of track parameters (rho, d0); -1 outside the axes."""
    NR, ND = g["n_rho"], g["n_d0"]
    rho = np.asarray(rho, np.float64)
    d0 = np.asarray(d0, np.float64)
    row = np.floor((rho + g["rho_max"]) / (2.0 * g["rho_max"] / NR))
    delta = 2.0 * g["d0_half"] / ND
    col = np.floor(d0 / delta + (ND / 2.0 + 0.5))
    ok = (row >= 0) & (row < NR) & (col >= 0) & (col < ND)
    row = np.where(ok, row, 0).astype(np.int64)
    col = np.where(ok, col, 0).astype(np.int64)
    return np.where(ok, (row * 8 // NR) * 8 + col * 8 // ND, -1)


def labels_of(g, ev):
    """int32 label of every hit of a generated event."""
    reg = region_of(g, ev.rho, ev.d0)
    tr = np.asarray(ev.track)
    return np.where(tr >= 0, reg[np.maximum(tr, 0)], -1).astype(np.int32)


# --------------------------------------------------------- data (host)
def _ensure_path():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _gen_chunk(job):
    """Worker: events seed0 .. seed0 + n - 1 of a workload, concatenated."""
    _ensure_path()
    import synth
    name, seed0, n = job
    gen = synth.CONFIGS[name]["gen"]
    g = synth.geometry_of(name)
    parts = []
    for s in range(seed0, seed0 + n):
        ev = synth.make_event(gen, s)
        parts.append((ev.x, ev.y, ev.z, ev.layer.astype(np.uint8), labels_of(g, ev)))
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(5))


def chunk_stream(name, seed0, n_events, per_chunk, workers):
    """Yield (x, y, z, layer, labels) host arrays of per_chunk events each,
    generated by `workers` spawned processes (spawn: safe after CUDA init)."""
    jobs = [(name, seed0 + a, min(per_chunk, n_events - a)) for a in range(0, n_events, per_chunk)]
    if workers <= 1:
        for j in jobs:
            yield _gen_chunk(j)
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_ensure_path) as pool:
        for out in pool.imap(_gen_chunk, jobs, chunksize=1):
            yield out


# -------------------------------------------------------------- trainer
class Trainer:
    """Adam on float32 master parameters; BF16 copy for the kernels."""

    def __init__(self, max_hits, seed=1, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                 init=None):
        import torch
        from . import ht
        self.ht = ht
        self.npar = ht.ht_mlp_param_count()
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        if init is None:
            init = init_params(seed)
        dev = torch.device("cuda")
        self.P = torch.from_numpy(np.asarray(init, np.float32)).to(dev)
        self.M = torch.zeros(self.npar, device=dev)
        self.V = torch.zeros(self.npar, device=dev)
        self.pb = torch.empty(self.npar, dtype=torch.int16, device=dev)
        self.grad = torch.zeros(self.npar, device=dev)
        self.step_no = 0
        self._alloc(max_hits)
        self._to_bf16()

    def _alloc(self, n):
        import torch
        dev = torch.device("cuda")
        self.cap = n
        self.prob = torch.empty((n, N_REGIONS), device=dev)
        self.h1 = torch.empty((n, 128), dtype=torch.int16, device=dev)
        self.h2 = torch.empty((n, 128), dtype=torch.int16, device=dev)
        self.feat = torch.empty((n, 8), dtype=torch.int16, device=dev)
        self.ws = torch.empty(self.ht.ht_mlp_backward_workspace_size(n), dtype=torch.uint8,
                              device=dev)

    def _to_bf16(self):
        # an Adam step with zero moments and zero gradient leaves the master
        # weights as they are and writes their BF16 copy
        import torch
        z = torch.zeros(self.npar, device=self.P.device)
        self.ht.ht_mlp_adam(self.P, z.clone(), z.clone(), z, 1, 0.0, self.b1, self.b2,
                            self.eps, self.pb)

    def step(self, x, y, z, layer, labels, lr=None):
        """One minibatch (device tensors) through forward, backward, Adam."""
        n = x.numel()
        if n > self.cap:
            self._alloc(n)
        ht = self.ht
        ht.ht_mlp_forward(self.pb, x, y, z, layer, self.prob[:n], self.h1[:n], self.h2[:n],
                          self.feat[:n])
        self.grad.zero_()
        ht.ht_mlp_backward(self.pb, labels, self.prob[:n], self.h1[:n], self.h2[:n],
                           self.feat[:n], self.grad, self.ws)
        self.step_no += 1
        ht.ht_mlp_adam(self.P, self.M, self.V, self.grad, self.step_no,
                       self.lr if lr is None else lr, self.b1, self.b2, self.eps, self.pb)

    def loss_sample(self, labels_host, n):
        """Mean cross entropy of the last minibatch's first n hits (host)."""
        p = self.prob[:n].cpu().numpy().astype(np.float64)
        lab = labels_host[:n]
        m = lab >= 0
        if not m.any():
            return float("nan")
        return float(-np.log(np.maximum(p[m, lab[m]], 1e-30)).mean())

    def state(self):
        return dict(params=self.P.cpu().numpy(), m=self.M.cpu().numpy(),
                    v=self.V.cpu().numpy(), step=self.step_no)

    def load_state(self, st):
        import torch
        self.P.copy_(torch.from_numpy(np.asarray(st["params"], np.float32)))
        self.M.copy_(torch.from_numpy(np.asarray(st["m"], np.float32)))
        self.V.copy_(torch.from_numpy(np.asarray(st["v"], np.float32)))
        self.step_no = int(st["step"])
        self._to_bf16()


def init_params(seed):
    """He-normal weights, zero biases, in the flat layout of ht_mlp_*."""
    rng = np.random.default_rng(seed)
    out = []
    for i, o in [(6, 128), (128, 128), (128, 64)]:
        out.append(rng.normal(0.0, math.sqrt(2.0 / i), i * o))
        out.append(np.zeros(o))
    return np.concatenate(out).astype(np.float32)


def bf16_params(params):
    """Device BF16 copy (int16 bits) of float32 parameters, written by the
    library's Adam kernel with a zero step."""
    import torch
    from . import ht
    P = torch.from_numpy(np.asarray(params, np.float32)).cuda()
    z = torch.zeros_like(P)
    pb = torch.empty(P.numel(), dtype=torch.int16, device="cuda")
    ht.ht_mlp_adam(P, z.clone(), z.clone(), z, 1, 0.0, 0.9, 0.999, 1e-8, pb)
    return pb


def save_checkpoint(path, trainer, meta):
    st = trainer.state()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.npz"
    np.savez(tmp, params=st["params"], m=st["m"], v=st["v"], step=st["step"],
             meta=json.dumps(meta))
    os.replace(tmp, path)


def load_weights(path):
    """(float32 parameters, metadata dict) of a checkpoint."""
    with np.load(path, allow_pickle=False) as f:
        return f["params"].astype(np.float32), json.loads(str(f["meta"]))


def train(name="event100_256", n_events=200000, seed0=1_000_000, per_chunk=8, lr=2e-3,
          seed=1, workers=None, out=None, ckpt_every=2000, resume=None, log=print):
    """Train on n_events generated events, per_chunk events per minibatch;
    checkpoints (parameters, Adam moments, step, next event) go to out."""
    import torch
    out = out or default_weights_path(name)
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    start_event = 0
    tr = Trainer(max_hits=per_chunk * 16000, seed=seed, lr=lr)
    meta = dict(workload=name, n_events=n_events, seed0=seed0, per_chunk=per_chunk, lr=lr,
                seed=seed, next_event=0)
    if resume and os.path.exists(resume):
        with np.load(resume, allow_pickle=False) as f:
            tr.load_state(dict(params=f["params"], m=f["m"], v=f["v"], step=f["step"]))
            meta = json.loads(str(f["meta"]))
        start_event = int(meta.get("next_event", 0))
        log(f"resumed at event {start_event}, step {tr.step_no}")
    total_steps = math.ceil(n_events / per_chunk)
    t0 = time.time()
    hits = 0
    ev_done = start_event
    for x, y, z, layer, lab in chunk_stream(name, seed0 + start_event, n_events - start_event,
                                            per_chunk, workers):
        k = tr.step_no
        # constant rate, then linear decay over the last fifth of the steps
        frac = k / max(total_steps, 1)
        cur = lr * (1.0 if frac < 0.8 else max(0.05, (1.0 - frac) / 0.2))
        dev = [torch.from_numpy(a).cuda(non_blocking=True) for a in (x, y, z, layer, lab)]
        tr.step(*dev, lr=cur)
        hits += x.shape[0]
        ev_done = min(n_events, ev_done + per_chunk)
        if tr.step_no % 500 == 0 or ev_done >= n_events:
            l = tr.loss_sample(lab, min(8192, x.shape[0]))
            el = time.time() - t0
            log(f"step {tr.step_no} events {ev_done} loss {l:.4f} "
                f"hits/s {hits / max(el, 1e-9):.3g} elapsed {el:.0f}s")
        if ckpt_every and tr.step_no % ckpt_every == 0:
            meta["next_event"] = ev_done
            save_checkpoint(out, tr, meta)
    torch.cuda.synchronize()
    meta["next_event"] = ev_done
    meta["train_seconds"] = time.time() - t0
    meta["hits"] = int(hits)
    save_checkpoint(out, tr, meta)
    return out, meta


# ----------------------------------------------------------- evaluation
def efficiency(g, ev, peaks, assign, min_hits=5):
    """Track-finding efficiency of one event's results.

    Reconstructable tracks: at least T hits and true (rho, d0) inside the
    axes.  'assign': a track is found when some candidate has at least
    min_hits assigned hits and more than half of them are the track's.
    'candidate': a track is found when some candidate lies in the 3 x 3 x 3
    box (phi0 circular) around the cell of its true parameters.
    Returns (n_reconstructable, found_assign, found_candidate)."""
    NR, ND, NP = g["n_rho"], g["n_d0"], g["n_phi0"]
    T = g["threshold"]
    ntr = len(ev.rho)
    nh = np.asarray(ev.n_track_hits)
    delta = 2.0 * g["d0_half"] / ND
    ti = np.floor((ev.rho + g["rho_max"]) / (2.0 * g["rho_max"] / NR)).astype(np.int64)
    tj = np.floor(ev.d0 / delta + ND / 2.0 + 0.5).astype(np.int64)
    tk = np.floor((np.asarray(ev.phi0) + math.pi) / (2.0 * math.pi / NP)).astype(np.int64) % NP
    ok = (nh >= T) & (ti >= 0) & (ti < NR) & (tj >= 0) & (tj < ND)
    found_a = np.zeros(ntr, bool)
    m = assign >= 0
    if m.any():
        cand = assign[m]
        trk = np.asarray(ev.track)[m]
        order = np.argsort(cand, kind="stable")
        cand, trk = cand[order], trk[order]
        bounds = np.flatnonzero(np.diff(cand)) + 1
        for seg in np.split(np.arange(cand.shape[0]), bounds):
            t = trk[seg]
            t = t[t >= 0]
            if t.size == 0:
                continue
            vals, cnts = np.unique(t, return_counts=True)
            b = int(np.argmax(cnts))
            if cnts[b] >= min_hits and cnts[b] * 2 > seg.shape[0]:
                found_a[vals[b]] = True
    found_c = np.zeros(ntr, bool)
    pk = np.asarray(peaks)
    if pk.shape[0] and ok.any():
        occ = np.zeros((NR, ND, NP), bool)
        occ[pk[:, 0], pk[:, 1], pk[:, 2]] = True
        t = np.flatnonzero(ok)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                ii, jj = ti[t] + di, tj[t] + dj
                inb = (ii >= 0) & (ii < NR) & (jj >= 0) & (jj < ND)
                for dk in (-1, 0, 1):
                    kk = (tk[t] + dk) % NP
                    found_c[t[inb]] |= occ[ii[inb], jj[inb], kk[inb]]
    return int(ok.sum()), int((found_a & ok).sum()), int((found_c & ok).sum())


def evaluate(weights=None, name="stream2000_256", n_events=100, seed0=0, batch=25, tau=0.02,
             fmax=0.6, grow=1, cap=1 << 20, log=print, topk=8):
    """Plain and learned batched paths on the same events -- the per-event
    region mask ("learned") and the per-hit top-k region sets ("hits"):
    events/s (device time of whole batches, graphs replayed), votes cast,
    candidate counts and both efficiencies."""
    import torch
    _ensure_path()
    import synth
    from . import ht
    weights = weights or default_weights_path("event100_256")
    params, meta = load_weights(weights)
    g = synth.geometry_of(name)
    evs = list(synth.make_stream(name, n_events, seed0))
    G = ht.Geometry(g)
    batches = [evs[i:i + batch] for i in range(0, len(evs), batch)]
    max_hits = max(sum(e.n_hits for e in b) for b in batches)
    B = ht.Batch(G, max_events=batch, max_hits=max_hits, cap=cap)
    pb = bf16_params(params)
    dev = []
    for b in batches:
        off = np.zeros(len(b) + 1, np.int32)
        off[1:] = np.cumsum([e.n_hits for e in b])
        cat = lambda k, t: torch.from_numpy(np.concatenate([getattr(e, k) for e in b]).astype(t)).cuda()
        dev.append((off, cat("x", np.float32), cat("y", np.float32), cat("z", np.float32),
                    cat("layer", np.uint8)))
    masks = torch.empty(batch, dtype=torch.int64, device="cuda")
    hmasks = torch.empty(max_hits, dtype=torch.int64, device="cuda")
    out = {}
    for mode in ("plain", "learned", "hits"):
        def run(d):
            off, x, y, z, l = d
            if mode == "plain":
                B.run(x, y, z, off)
            elif mode == "learned":
                B.run_learned(x, y, z, l, off, pb, masks, tau, fmax, grow)
            else:
                B.run_learned_hits(x, y, z, l, off, pb, hmasks, topk, 0.0)
        for d in dev:                    # capture the graphs, warm up
            run(d)
        torch.cuda.synchronize()
        t = 0.0
        res = dict(votes=0, cands=0, n_rec=0, f_assign=0, f_cand=0, masks=[])
        for (off, *_), b, d in zip(dev, batches, dev):
            a, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run(d)
            e_.record()
            e_.synchronize()
            t += a.elapsed_time(e_) / 1e3
            for i, ev in enumerate(b):
                r = B.event_results(off, i)
                res["votes"] += r["votes"]
                res["cands"] += r["count"]
                nr, fa, fc = efficiency(g, ev, r["peaks"], r["assign"])
                res["n_rec"] += nr; res["f_assign"] += fa; res["f_cand"] += fc
            if mode == "learned":
                res["masks"] += [int(v) & ((1 << 64) - 1) for v in masks[:len(b)].cpu().tolist()]
        res["events_per_s"] = n_events / t
        res["eff_assign"] = res["f_assign"] / max(res["n_rec"], 1)
        res["eff_candidate"] = res["f_cand"] / max(res["n_rec"], 1)
        if mode == "learned":
            mk = res.pop("masks")
            res["mean_regions"] = float(np.mean([bin(m).count("1") for m in mk]))
            res["fallback_frac"] = float(np.mean([m == (1 << 64) - 1 for m in mk]))
        else:
            res.pop("masks")
        out[mode] = res
        log(mode, {k: v for k, v in res.items()})
    out["vote_frac"] = out["learned"]["votes"] / max(out["plain"]["votes"], 1)
    out["speedup"] = out["learned"]["events_per_s"] / out["plain"]["events_per_s"]
    out["hits_vote_frac"] = out["hits"]["votes"] / max(out["plain"]["votes"], 1)
    out["hits_speedup"] = out["hits"]["events_per_s"] / out["plain"]["events_per_s"]
    out["params"] = dict(workload=name, events=n_events, seed0=seed0, batch=batch, tau=tau,
                         fmax=fmax, grow=grow, topk=topk, weights=os.path.basename(weights),
                         trained_on=meta.get("workload"), train_events=meta.get("n_events"))
    B.close()
    G.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--workload", default="event100_256")
    t.add_argument("--events", type=int, default=200000)
    t.add_argument("--per-chunk", type=int, default=8)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=1)
    t.add_argument("--workers", type=int, default=0)
    t.add_argument("--out", default=None)
    t.add_argument("--resume", default=None)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=None)
    e.add_argument("--workload", default="stream2000_256")
    e.add_argument("--events", type=int, default=100)
    e.add_argument("--seed0", type=int, default=0)
    e.add_argument("--batch", type=int, default=25)
    e.add_argument("--tau", type=float, default=0.02)
    e.add_argument("--fmax", type=float, default=0.6)
    e.add_argument("--grow", type=int, default=1)
    e.add_argument("--topk", type=int, default=8)
    e.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        path, meta = train(a.workload, a.events, per_chunk=a.per_chunk, lr=a.lr, seed=a.seed,
                           workers=a.workers or None, out=a.out, resume=a.resume)
        print(json.dumps(dict(weights=path, **meta)))
    else:
        r = evaluate(a.weights, a.workload, a.events, a.seed0, a.batch, a.tau, a.fmax, a.grow,
                     topk=a.topk)
        s = json.dumps(r)
        print(s)
        if a.json:
            with open(a.json, "w") as f:
                f.write(s + "\n")


if __name__ == "__main__":
    main()
