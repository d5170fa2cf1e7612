"""Oracle of the learned region proposal: per-hit MLP, loss, gradients, Adam,
region labels, region masses and masks.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; it shares no code with the
CUDA path.

The network (the proposal's reading; the paper has no learned part): per-hit
features f = (x/110, y/110, z/(110 sinh 2.5), r/110, phi/pi, layer/9),
6 -> 128 -> 128 -> 64 with ReLU, softmax over 64 (rho, d0) regions (an 8 x 8
grid of equal blocks of the accumulator's rho rows and d0 bins).  BF16
weights and biases and BF16 activations between layers, wider accumulation:
the oracle accumulates in float64 and rounds to BF16 at exactly the points
the kernels do (parameters, features, the two hidden layers); logits and
softmax stay unrounded.

Parameter layout (one flat float array): W1[6][128], b1[128], W2[128][128],
b2[128], W3[128][64], b3[64]; W[i][o] multiplies input i into output o.
"""
import math

import numpy as np

SIZES = [(6, 128), (128, 128), (128, 64)]
N_REGIONS = 64
ETA_MAX = 2.5


def n_params():
    return sum(i * o + o for i, o in SIZES)


def unpack(p):
    """Views (W1, b1, W2, b2, W3, b3) of a flat parameter array."""
    out, k = [], 0
    for i, o in SIZES:
        out.append(p[k:k + i * o].reshape(i, o)); k += i * o
        out.append(p[k:k + o]); k += o
    return out


def bf16(a):
    """Round to bfloat16 (round to nearest, ties to even) via float32 bits."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def features(x, y, z, layer):
    """Per-hit features in float32 arithmetic, then rounded to BF16."""
    x = np.asarray(x, np.float32); y = np.asarray(y, np.float32)
    z = np.asarray(z, np.float32); layer = np.asarray(layer)
    r = np.sqrt(x * x + y * y, dtype=np.float32)
    zs = np.float32(110.0) * np.float32(math.sinh(ETA_MAX))   # a float32 product
    f = np.stack([x / np.float32(110), y / np.float32(110), z / zs, r / np.float32(110),
                  np.arctan2(y, x).astype(np.float32) / np.float32(math.pi),
                  layer.astype(np.float32) / np.float32(9)], axis=1).astype(np.float32)
    return bf16(f)


def forward(p, f, round_bf16=True):
    """Logits, probabilities and the cached activations (float64)."""
    rnd = bf16 if round_bf16 else (lambda a: a)
    W1, b1, W2, b2, W3, b3 = unpack(rnd(np.asarray(p, np.float64)))
    a1 = f @ W1 + b1
    h1 = rnd(np.maximum(a1, 0.0))
    a2 = h1 @ W2 + b2
    h2 = rnd(np.maximum(a2, 0.0))
    logits = h2 @ W3 + b3
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    prob = e / e.sum(axis=1, keepdims=True)
    return logits, prob, (f, h1, h2, W1, W2, W3)


def loss_and_grad(p, f, labels, round_bf16=True):
    """Mean softmax cross entropy over hits with label >= 0 and its gradient
    with respect to the (unrounded) parameters.  Rounding points are treated
    as identity in the backward pass (the usual straight-through reading)."""
    labels = np.asarray(labels)
    logits, prob, (f, h1, h2, W1, W2, W3) = forward(p, f, round_bf16)
    m = labels >= 0
    nl = max(int(m.sum()), 1)
    loss = -np.log(prob[m, labels[m]]).sum() / nl
    dL = prob.copy()
    dL[np.arange(len(labels))[m], labels[m]] -= 1.0
    dL[~m] = 0.0
    dL /= nl
    gW3 = h2.T @ dL
    gb3 = dL.sum(0)
    dh2 = (dL @ W3.T) * (h2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    gW1 = f.T @ dh1
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba), bias-corrected; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def region_of(g, rho, d0):
    """Region (8 x 8 grid over rho rows and d0 bins) of track parameters, -1
    outside the axes.  The bins are the vote's: rho row floor((rho + rho_max)
    / (2 rho_max / n_rho)), d0 bin floor(d0 / delta + n_d0/2 + 1/2)."""
    NR, ND = g["n_rho"], g["n_d0"]
    rho = np.asarray(rho, np.float64); d0 = np.asarray(d0, np.float64)
    i = np.floor((rho + g["rho_max"]) / (2 * g["rho_max"] / NR)).astype(np.int64)
    delta = 2.0 * g["d0_half"] / ND
    j = np.floor(d0 / delta + (ND * 0.5 + 0.5)).astype(np.int64)
    ok = (i >= 0) & (i < NR) & (j >= 0) & (j < ND)
    return np.where(ok, (i * 8 // NR) * 8 + (j * 8 // ND), -1)


def hit_labels(g, ev):
    """Label of every hit: its track's region, -1 for noise hits."""
    reg = region_of(g, ev.rho, ev.d0)
    return np.where(ev.track >= 0, reg[np.maximum(ev.track, 0)], -1).astype(np.int32)


def region_mass(prob):
    """Mean softmax mass per region over an event's hits."""
    return prob.mean(axis=0) if prob.shape[0] else np.zeros(N_REGIONS)


def region_mask(mass, tau, fmax, grow=False, n_hits=None):
    """64-bit mask: regions with mean mass >= tau; with grow, also their
    8 neighbours on the 8 x 8 region grid (no wrap); every region if more
    than fmax of the 64 are selected or the event has no hits (the full vote
    is the fallback)."""
    sel = (np.asarray(mass) >= tau).reshape(8, 8)
    if grow:
        g = sel.copy()
        for a in range(8):
            for b in range(8):
                if sel[a, b]:
                    g[max(a - 1, 0):a + 2, max(b - 1, 0):b + 2] = True
        sel = g
    bits = sel.ravel()
    if bits.sum() > fmax * N_REGIONS or n_hits == 0:
        bits = np.ones(N_REGIONS, bool)
    return int(sum(1 << int(r) for r in np.nonzero(bits)[0]))


def cell_allowed(g, mask):
    """Cells (i, j) the masked vote counts: inside a masked region or within
    one rho row / d0 bin of one (the halo that keeps masked peaks exact)."""
    NR, ND = g["n_rho"], g["n_d0"]
    reg = np.zeros((8, 8), bool)
    for r in range(64):
        if (mask >> r) & 1:
            reg[r // 8, r % 8] = True
    inside = reg[np.arange(NR) * 8 // NR][:, np.arange(ND) * 8 // ND]
    halo = inside.copy()
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            sh = np.zeros_like(inside)
            si = slice(max(di, 0), NR + min(di, 0)); ti = slice(max(-di, 0), NR + min(-di, 0))
            sj = slice(max(dj, 0), ND + min(dj, 0)); tj = slice(max(-dj, 0), ND + min(-dj, 0))
            sh[ti, tj] = inside[si, sj]
            halo |= sh
    return inside, halo


def masked_event(g, x, y, z, mask, cap=None, threads=None, acc=None):
    """The path with the vote and the peak finding restricted to a region
    mask: the full event's peaks (Sections 5-7) that are inside the mask, in
    the same order, then association and the z vote on them unchanged.
    Also returns the halo (cells the masked vote must count exactly) and the
    votes that fall in it.  acc: the full accumulator, if already voted."""
    from . import oracle as O
    if acc is None:
        acc, _ = O.vote(g, x, y, threads)
    pk_all, _ = O.peaks(g, acc, None, threads)
    inside, halo = cell_allowed(g, mask)
    keep = inside[pk_all[:, 0], pk_all[:, 1]] if pk_all.shape[0] else np.zeros(0, bool)
    pk = pk_all[keep]
    count = int(pk.shape[0])
    if cap is not None:
        pk = pk[:cap]
    pk = np.ascontiguousarray(pk)
    asg = O.associate_dense(g, x, y, pk, threads=threads)
    zr = O.vote_z(g, x, y, z, asg, pk, threads=threads)
    votes = int(acc[halo].sum())
    return dict(acc=acc, halo=halo, peaks=pk, count=count, assign=asg, zres=zr, votes=votes)


def hit_topk_masks(prob, k, pmin=0.0):
    """Per-hit region sets of the per-hit proposal (reading): the k regions
    of largest probability (ties to the smaller region index) as a 64-bit
    mask; every region when k >= 64 or when those k probabilities sum to
    less than pmin (an unsure hit votes everywhere)."""
    prob = np.asarray(prob, np.float64)
    out = np.zeros(prob.shape[0], np.uint64)
    full = np.uint64((1 << 64) - 1)
    for h in range(prob.shape[0]):
        if k >= N_REGIONS:
            out[h] = full
            continue
        top = np.argsort(-prob[h], kind="stable")[:k]
        if prob[h][top].sum() < pmin:
            out[h] = full
            continue
        out[h] = np.uint64(sum(1 << int(r) for r in top))
    return out


def hit_masked_event(g, x, y, z, masks, cap=None, threads=None):
    """The path with each hit's votes restricted to its region set plus a
    one-cell halo (Section 5's vote, then the peaks of that accumulator,
    association and the z vote unchanged).  masks: uint64 per hit."""
    from . import oracle as O
    acc, st = O.vote_hitmask(g, x, y, masks, threads)
    pk, count = O.peaks(g, acc, cap, threads)
    pk = np.ascontiguousarray(pk)
    asg = O.associate_dense(g, x, y, pk, threads=threads)
    zr = O.vote_z(g, x, y, z, asg, pk, threads=threads)
    return dict(acc=acc, peaks=pk, count=count, assign=asg, zres=zr, votes=st["votes"])
