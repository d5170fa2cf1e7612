"""Python front end of the CPU oracle (ht_oracle.c).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module.  It shares no code with the
CUDA path and never imports it.

Every function here marshals numpy arrays into the C oracle.  Work is split
across threads only along axes whose results are independent (rows of the
accumulator, hits, candidates); ctypes releases the GIL during each call, and
no arithmetic is reordered.
"""
import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libht_oracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: every floating-point operation stays a single IEEE op (no FMA
# contraction, no fast-math); portable across x86_64 and aarch64.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force=False):
    """Compile the oracle library in-tree (oracle/_build/libht_oracle.so)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrGeom(ctypes.Structure):
    _fields_ = [("n_rho", ctypes.c_int32), ("n_d0", ctypes.c_int32),
                ("n_phi0", ctypes.c_int32), ("n_z0", ctypes.c_int32),
                ("n_cot", ctypes.c_int32), ("threshold", ctypes.c_int32),
                ("count_max", ctypes.c_int64), ("rho_max", ctypes.c_double),
                ("d0_half", ctypes.c_double), ("z0_max", ctypes.c_double),
                ("cot_max", ctypes.c_double)]


class OrConfirm(ctypes.Structure):
    _fields_ = [("pool", ctypes.c_int32), ("min_layers", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tol", ctypes.c_double)]


# Confirmation parameters of the dense-event track finder (see or_confirm):
# inlier pool of +-4 bins, 8 inlier layers, ten layers, 100 um (5 sigma of
# the 20 um hit resolution).
CONFIRM_DEFAULT = dict(pool=4, min_layers=8, n_layers=10, tol=0.01)


def _geom(g):
    cm = 65535 if g.get("count_bits", 32) == 16 else 2147483647
    return OrGeom(g["n_rho"], g["n_d0"], g["n_phi0"], g["n_z0"], g["n_cot"],
                  g["threshold"], cm, g["rho_max"], g["d0_half"], g["z0_max"],
                  g["cot_max"])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            G = P(OrGeom)
            vp = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            L.or_tables.argtypes = [G, vp, vp, vp, vp]
            L.or_vote.argtypes = [G, vp, vp, i64, i32, i32, vp, vp]
            L.or_vote_hitmask.argtypes = [G, vp, vp, vp, i64, i32, i32, vp, vp]
            L.or_vote_swept.argtypes = [G, vp, vp, i64, i32, i32, vp, vp]
            L.or_edge_tables.argtypes = [G, vp, vp]
            L.or_peaks.argtypes = [G, vp, i32, i32, vp, i64]
            L.or_peaks.restype = i64
            L.or_associate.argtypes = [G, vp, vp, vp, i64, vp, i64, vp]
            L.or_atan2.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_atan2.restype = ctypes.c_double
            L.or_atan2_array.argtypes = [vp, vp, i64, vp]
            L.or_vote_z.argtypes = [G, vp, vp, vp, vp, vp, i64, vp, vp, vp]
            L.or_associate_dense.argtypes = [G, vp, vp, vp, i64, vp, vp, vp]
            L.or_vote_layers.argtypes = [G, vp, vp, vp, vp, i64, i32, i32, vp, vp]
            L.or_circle3.argtypes = [ctypes.c_double] * 6 + [vp, vp, vp]
            L.or_circle3.restype = ctypes.c_int
            L.or_confirm.argtypes = [G, ctypes.POINTER(OrConfirm), vp, vp, vp, i64, vp, i64,
                                     i64, vp, vp, vp]
            L.or_confirm_assign.argtypes = [vp, vp, i64, i64, vp]
            _lib = L
        return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _threads(threads):
    return max(1, threads if threads else (os.cpu_count() or 1))


def _chunks(n, parts):
    parts = max(1, min(parts, n)) if n > 0 else 1
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def tables(g):
    """(phi0, sin phi0, cos phi0, rho) float64 axis tables."""
    G = _geom(g)
    phi0 = np.empty(g["n_phi0"]); sn = np.empty_like(phi0); cs = np.empty_like(phi0)
    rho = np.empty(g["n_rho"])
    lib().or_tables(ctypes.byref(G), _p(phi0), _p(sn), _p(cs), _p(rho))
    return phi0, sn, cs, rho


def vote(g, x, y, threads=None, rows=None):
    """Accumulator int64 [n_rho, n_d0, n_phi0] and stats {votes, edge}.

    rows=(a, b) computes only rho rows [a, b) and returns acc[a:b] (each row
    of the vote depends only on that row)."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    r0, r1 = (0, g["n_rho"]) if rows is None else rows
    acc = np.zeros((g["n_rho"], g["n_d0"], g["n_phi0"]), np.int64) if rows is None else \
        np.zeros((r1 - r0, g["n_d0"], g["n_phi0"]), np.int64)
    base = 0 if rows is None else r0 * g["n_d0"] * g["n_phi0"] * 8
    parts = [(a + r0, b + r0) for a, b in _chunks(r1 - r0, _threads(threads) * 2)]
    stats = np.zeros((len(parts), 2), np.int64)
    accp = acc.ctypes.data - base

    def run(t):
        a, b = parts[t]
        lib().or_vote(ctypes.byref(G), _p(x), _p(y), x.shape[0], a, b,
                      ctypes.c_void_p(accp), _p(stats[t]))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, range(len(parts))))
    tot = stats.sum(0)
    return acc, {"votes": int(tot[0]), "edge": int(tot[1])}


def vote_hitmask(g, x, y, masks, threads=None, rows=None):
    """The vote with hit h's votes kept only in cells allowed by masks[h]
    (uint64 per hit: a region set on the 8 x 8 region grid, plus a one-cell
    halo; see or_vote_hitmask).  Returns (acc, {votes, edge}) like vote;
    rows=(a, b) computes only rho rows [a, b) and returns acc[a:b]."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    m = np.ascontiguousarray(np.asarray(masks, np.uint64))
    assert m.shape[0] == x.shape[0]
    r0, r1 = (0, g["n_rho"]) if rows is None else rows
    acc = np.zeros((r1 - r0, g["n_d0"], g["n_phi0"]), np.int64)
    base = r0 * g["n_d0"] * g["n_phi0"] * 8
    parts = [(a + r0, b + r0) for a, b in _chunks(r1 - r0, _threads(threads) * 2)]
    stats = np.zeros((len(parts), 2), np.int64)
    accp = acc.ctypes.data - base

    def run(t):
        a, b = parts[t]
        lib().or_vote_hitmask(ctypes.byref(G), _p(x), _p(y), _p(m), x.shape[0], a, b,
                              ctypes.c_void_p(accp), _p(stats[t]))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, range(len(parts))))
    tot = stats.sum(0)
    return acc, {"votes": int(tot[0]), "edge": int(tot[1])}


def edge_tables(g):
    """(sin, cos) of the column lower edges e_k = (2k - N) pi / N, float64."""
    G = _geom(g)
    sn = np.empty(g["n_phi0"]); cs = np.empty_like(sn)
    lib().or_edge_tables(ctypes.byref(G), _p(sn), _p(cs))
    return sn, cs


def vote_swept(g, x, y, threads=None, rows=None):
    """Swept-interval vote (or_vote_swept): each hit marks, in every (rho
    row, phi0 column), the d0 bins its roots sweep between the column's
    edges and centre.  Returns (acc, {votes}); rows=(a, b) computes only
    rho rows [a, b) and returns acc[a:b]."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    r0, r1 = (0, g["n_rho"]) if rows is None else rows
    acc = np.zeros((r1 - r0, g["n_d0"], g["n_phi0"]), np.int64)
    base = r0 * g["n_d0"] * g["n_phi0"] * 8
    parts = [(a + r0, b + r0) for a, b in _chunks(r1 - r0, _threads(threads) * 2)]
    stats = np.zeros((len(parts), 2), np.int64)
    accp = acc.ctypes.data - base

    def run(t):
        a, b = parts[t]
        lib().or_vote_swept(ctypes.byref(G), _p(x), _p(y), x.shape[0], a, b,
                            ctypes.c_void_p(accp), _p(stats[t]))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, range(len(parts))))
    return acc, {"votes": int(stats[:, 0].sum())}


def peaks(g, acc, cap=None, threads=None):
    """Peaks sorted by logical index: (int32 [min(count, cap), 4], count)."""
    G = _geom(g)
    acc = np.ascontiguousarray(acc, np.int64)
    rows = _chunks(g["n_rho"], _threads(threads) * 2)
    outs = [None] * len(rows)

    def run(t):
        a, b = rows[t]
        n = lib().or_peaks(ctypes.byref(G), _p(acc), a, b, None, 0)
        buf = np.zeros((max(n, 1), 4), np.int32)
        lib().or_peaks(ctypes.byref(G), _p(acc), a, b, _p(buf), n)
        outs[t] = buf[:n]

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, range(len(rows))))
    allp = np.concatenate(outs) if outs else np.zeros((0, 4), np.int32)
    count = allp.shape[0]
    if cap is not None:
        allp = allp[:cap]
    return np.ascontiguousarray(allp), count


def associate(g, x, y, pk, hit_idx=None, threads=None):
    """Assignment int32 per selected hit (all hits if hit_idx is None)."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    pk = np.ascontiguousarray(pk, np.int32).reshape(-1, 4)
    if hit_idx is None:
        hit_idx = np.arange(x.shape[0], dtype=np.int64)
    hit_idx = np.ascontiguousarray(hit_idx, np.int64)
    out = np.full(hit_idx.shape[0], -1, np.int32)
    parts = _chunks(hit_idx.shape[0], _threads(threads) * 4)

    def run(ab):
        a, b = ab
        sub = hit_idx[a:b].copy()
        o = np.empty(b - a, np.int32)
        lib().or_associate(ctypes.byref(G), _p(x), _p(y), _p(sub), b - a, _p(pk),
                           pk.shape[0], _p(o))
        out[a:b] = o

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, parts))
    return out


def associate_dense(g, x, y, pk, hit_idx=None, threads=None):
    """Association by enumerating each hit's votes against a cell -> candidate
    map (same rule as associate(); the route used for full-size events)."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    pk = np.ascontiguousarray(pk, np.int32).reshape(-1, 4)
    cand_at = np.full(g["n_rho"] * g["n_d0"] * g["n_phi0"], -1, np.int32)
    lidx = (pk[:, 0].astype(np.int64) * g["n_d0"] + pk[:, 1]) * g["n_phi0"] + pk[:, 2]
    cand_at[lidx] = np.arange(pk.shape[0], dtype=np.int32)
    if hit_idx is None:
        hit_idx = np.arange(x.shape[0], dtype=np.int64)
    hit_idx = np.ascontiguousarray(hit_idx, np.int64)
    out = np.full(hit_idx.shape[0], -1, np.int32)
    parts = _chunks(hit_idx.shape[0], _threads(threads) * 4)

    def run(ab):
        a, b = ab
        sub = hit_idx[a:b].copy()
        o = np.empty(b - a, np.int32)
        lib().or_associate_dense(ctypes.byref(G), _p(x), _p(y), _p(sub), b - a, _p(pk),
                                 _p(cand_at), _p(o))
        out[a:b] = o

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, parts))
    return out


def vote_z(g, x, y, z, assign, pk, cand=None, threads=None):
    """Per-candidate (z0, cot theta) argmax: int32 [n_cand, 3] = {n, q, count}."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    assign = np.ascontiguousarray(assign, np.int32)
    pk = np.ascontiguousarray(pk, np.int32).reshape(-1, 4)
    if cand is None:
        cand = np.arange(pk.shape[0], dtype=np.int64)
    cand = np.ascontiguousarray(cand, np.int64)
    # group hit indices by assigned candidate (marshalling, no arithmetic)
    order = np.argsort(assign, kind="stable").astype(np.int64)
    sa = assign[order]
    lo = np.searchsorted(sa, cand, side="left")
    hi = np.searchsorted(sa, cand, side="right")
    out = np.zeros((cand.shape[0], 3), np.int32)
    parts = _chunks(cand.shape[0], _threads(threads) * 4)

    def run(ab):
        a, b = ab
        c_sub = cand[a:b].copy()
        lists = [order[lo[t]:hi[t]] for t in range(a, b)]
        off = np.zeros(b - a + 1, np.int64)
        off[1:] = np.cumsum([len(v) for v in lists])
        lst = np.concatenate(lists) if lists else np.zeros(0, np.int64)
        lst = np.ascontiguousarray(lst, np.int64)
        o = np.zeros((b - a, 3), np.int32)
        lib().or_vote_z(ctypes.byref(G), _p(x), _p(y), _p(z), _p(pk), _p(c_sub), b - a,
                        _p(off), _p(lst), _p(o))
        out[a:b] = o

    if cand.shape[0]:
        with ThreadPoolExecutor(_threads(threads)) as ex:
            list(ex.map(run, parts))
    return out


def atan2(y, x):
    """The oracle's basic-operation atan2, elementwise over float64 arrays."""
    y = np.ascontiguousarray(y, np.float64); x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(y)
    lib().or_atan2_array(_p(y), _p(x), y.shape[0], _p(out))
    return out


def vote_layers(g, x, y, layer, masks=None, threads=None, rows=None):
    """Distinct-layer accumulator int64 [n_rho, n_d0, n_phi0] (or rows
    [a, b) only) and stats {votes, edge}: a cell counts the distinct layers
    of the hits voting in it (or_vote_layers).  masks: None or one uint64
    region set per hit (the per-hit proposal's halo rule)."""
    G = _geom(g)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    layer = np.ascontiguousarray(layer, np.uint8)
    assert layer.shape[0] == x.shape[0] and (layer.size == 0 or int(layer.max()) < 16)
    m = None if masks is None else np.ascontiguousarray(np.asarray(masks, np.uint64))
    if m is not None:
        assert m.shape[0] == x.shape[0]
    r0, r1 = (0, g["n_rho"]) if rows is None else rows
    acc = np.zeros((r1 - r0, g["n_d0"], g["n_phi0"]), np.int64)
    base = r0 * g["n_d0"] * g["n_phi0"] * 8
    parts = [(a + r0, b + r0) for a, b in _chunks(r1 - r0, _threads(threads) * 2)]
    stats = np.zeros((len(parts), 2), np.int64)
    accp = acc.ctypes.data - base

    def run(t):
        a, b = parts[t]
        lib().or_vote_layers(ctypes.byref(G), _p(x), _p(y), _p(layer),
                             None if m is None else _p(m), x.shape[0], a, b,
                             ctypes.c_void_p(accp), _p(stats[t]))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, range(len(parts))))
    tot = stats.sum(0)
    return acc, {"votes": int(tot[0]), "edge": int(tot[1])}


def circle3(p1, p2, p3):
    """(xc, yc, R) of the circle through three points, or None if collinear."""
    xc, yc, R = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = lib().or_circle3(float(p1[0]), float(p1[1]), float(p2[0]), float(p2[1]),
                          float(p3[0]), float(p3[1]), ctypes.byref(xc), ctypes.byref(yc),
                          ctypes.byref(R))
    return (xc.value, yc.value, R.value) if ok else None


def _confirm_struct(cp):
    c = dict(CONFIRM_DEFAULT)
    c.update(cp or {})
    assert 1 <= c["n_layers"] <= 16
    return OrConfirm(c["pool"], c["min_layers"], c["n_layers"], 0, c["tol"])


def confirm(g, x, y, layer, pk, cp=None, threads=None):
    """Confirmation of every candidate (or_confirm): (score int32 [m],
    seeds int32 [m, 3], inliers int32 [m, 16])."""
    G = _geom(g)
    C = _confirm_struct(cp)
    x = np.ascontiguousarray(x, np.float32); y = np.ascontiguousarray(y, np.float32)
    layer = np.ascontiguousarray(layer, np.uint8)
    assert layer.shape[0] == x.shape[0] and (layer.size == 0 or int(layer.max()) < C.n_layers)
    pk = np.ascontiguousarray(pk, np.int32).reshape(-1, 4)
    npk = pk.shape[0]
    score = np.zeros(npk, np.int32)
    seeds = np.full((npk, 3), -1, np.int32)
    inl = np.full((npk, 16), -1, np.int32)
    parts = _chunks(npk, _threads(threads) * 4)

    def run(ab):
        a, b = ab
        lib().or_confirm(ctypes.byref(G), ctypes.byref(C), _p(x), _p(y), _p(layer), x.shape[0],
                         _p(pk), a, b, _p(score), _p(seeds), _p(inl))

    if npk:
        with ThreadPoolExecutor(_threads(threads)) as ex:
            list(ex.map(run, parts))
    return score, seeds, inl


def confirm_assign(score, inl, n_hits):
    """Hit -> confirmed candidate (or_confirm_assign): int32 [n_hits]."""
    score = np.ascontiguousarray(score, np.int32)
    inl = np.ascontiguousarray(inl, np.int32).reshape(-1, 16)
    out = np.full(n_hits, -1, np.int32)
    lib().or_confirm_assign(_p(score), _p(inl), score.shape[0], n_hits, _p(out))
    return out


def run_event_tracks(g, x, y, z, layer, cp=None, cap=None, masks=None, threads=None):
    """The track-finding path on one event: distinct-layer vote, peaks,
    confirmation, final assignment and the (z0, cot theta) vote."""
    acc, st = vote_layers(g, x, y, layer, masks, threads)
    pk, cnt = peaks(g, acc, cap, threads)
    score, seeds, inl = confirm(g, x, y, layer, pk, cp, threads)
    asg = confirm_assign(score, inl, x.shape[0])
    zr = vote_z(g, x, y, z, asg, pk, threads=threads)
    return dict(acc=acc, stats=st, peaks=pk, count=cnt, score=score, seeds=seeds, inliers=inl,
                assign=asg, zres=zr)


def run_event(g, x, y, z, cap=None, threads=None):
    """The whole path on one event: acc, stats, peaks, count, assign, zres."""
    acc, st = vote(g, x, y, threads)
    pk, cnt = peaks(g, acc, cap, threads)
    asg = associate_dense(g, x, y, pk, threads=threads)
    zr = vote_z(g, x, y, z, asg, pk, threads=threads)
    return dict(acc=acc, stats=st, peaks=pk, count=cnt, assign=asg, zres=zr)
