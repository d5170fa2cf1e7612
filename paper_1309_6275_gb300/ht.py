"""Thin Python binding of libht (include/ht.h), argument marshalling only.

Every function here forwards torch CUDA tensors (device pointers) or pinned
host tensors to the C ABI of the same name; all arithmetic runs in libht's
CUDA kernels.  There is no CPU or PyTorch fallback: if the library cannot be
built or loaded, importing this module raises.

Tensor conventions:
  hits          float32 [n] each (x, y, z), contiguous, on the geometry's GPU
  accumulator   int16 (viewed as uint16) or int32 [n_rho, n_d0, n_phi0]
  peaks         int32 [cap, 4] = {i_rho, j_d0, k_phi0, count}
  d_count       int32 [1]
  assign        int32 [n]
  zres          int32 [cap, 3] = {n_z0, m_cot, count}
  stats         int64 [2] (uint64 counters: votes, float64 redos)
  workspace     uint8, at least the size the matching *_workspace_size gives
  mask          int64 [1] per event (uint64 region bits, see ht_vote_masked)
  hit_masks     int64 [n] per hit (uint64 region bits, see ht_vote_hit_masked)
  MLP params    float32 master / int16 (BF16 bits) copy [ht_mlp_param_count()]
  layer         uint8 [n] per hit
"""
import ctypes
import os

import torch

from . import build as _build

_lib = None


class HTError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [("n_rho", ctypes.c_int32), ("n_d0", ctypes.c_int32),
                ("n_phi0", ctypes.c_int32), ("n_z0", ctypes.c_int32),
                ("n_cot", ctypes.c_int32), ("threshold", ctypes.c_int32),
                ("count_bits", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rho_max", ctypes.c_double), ("d0_half", ctypes.c_double),
                ("z0_max", ctypes.c_double), ("cot_max", ctypes.c_double)]


class _VertexDesc(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
                ("threshold", ctypes.c_int32), ("min_count", ctypes.c_int32),
                ("r_max", ctypes.c_double), ("r_keep", ctypes.c_double)]


class _Proposal(ctypes.Structure):
    _fields_ = [("params_bf16", ctypes.c_void_p), ("layer", ctypes.c_void_p),
                ("tau", ctypes.c_float), ("fmax", ctypes.c_float),
                ("grow", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _HitProposal(ctypes.Structure):
    _fields_ = [("params_bf16", ctypes.c_void_p), ("layer", ctypes.c_void_p),
                ("topk", ctypes.c_int32), ("pmin", ctypes.c_float)]


class _ConfirmDesc(ctypes.Structure):
    _fields_ = [("pool", ctypes.c_int32), ("min_layers", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("n_bands", ctypes.c_int32),
                ("tol", ctypes.c_double), ("band_max_hits", ctypes.c_int32 * 8),
                ("band_threshold", ctypes.c_int32 * 8)]


def confirm_desc(c):
    """ht_confirm_desc from a dict {pool, min_layers, n_layers, tol, bands}
    (bands: [(max_hits, threshold), ...] in increasing max_hits)."""
    bands = list(c.get("bands", ()))
    assert len(bands) <= 8
    d = _ConfirmDesc(int(c["pool"]), int(c["min_layers"]), int(c["n_layers"]), len(bands),
                     float(c["tol"]))
    for q, (mh, t) in enumerate(bands):
        d.band_max_hits[q] = int(mh)
        d.band_threshold[q] = int(t)
    return d


# (name, restype, argtypes) of every exported function, as in include/ht.h
_P, _I32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
SIGNATURES = [
    ("ht_last_error", ctypes.c_char_p, []),
    ("ht_geometry_create", _I32, [ctypes.POINTER(_Desc), ctypes.POINTER(_P)]),
    ("ht_geometry_destroy", _I32, [_P]),
    ("ht_accumulator_bytes", _SZ, [_P]),
    ("ht_vote", _I32, [_P, _P, _P, _I32, _P, _P, _P]),
    ("ht_find_peaks_workspace_size", _SZ, [_P]),
    ("ht_find_peaks", _I32, [_P, _P, _P, _I32, _P, _P, _SZ, _P]),
    ("ht_find_peaks_noalloc", _I32, [_P, _P, _P, _I32, _P, _P]),
    ("ht_associate_workspace_size", _SZ, [_P, _I32, _I32]),
    ("ht_associate", _I32, [_P, _P, _P, _I32, _P, _P, _I32, _P, _P, _SZ, _P]),
    ("ht_vote_z_workspace_size", _SZ, [_P, _I32, _I32]),
    ("ht_vote_z", _I32, [_P, _P, _P, _P, _I32, _P, _P, _P, _I32, _P, _P, _SZ, _P]),
    ("ht_event_workspace_size", _SZ, [_P, _I32, _I32]),
    ("ht_run_event", _I32, [_P, _P, _P, _P, _I32, _P, _SZ, _P, _I32, _P, _P, _P, _P, _P]),
    ("ht_batch_create", _I32, [_P, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    ("ht_batch_destroy", _I32, [_P]),
    ("ht_batch_set_graphs", _I32, [_P, _I32]),
    ("ht_batch_run", _I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P]),
    ("ht_batch_stage_ms", _I32, [_P, _P]),
    ("ht_batch_autotune", _I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _P,
                                  ctypes.POINTER(_I32), _P]),
    ("ht_vote_masked", _I32, [_P, _P, _P, _I32, _P, _P, _P, _P]),
    ("ht_find_peaks_masked", _I32, [_P, _P, _P, _P, _I32, _P, _P, _SZ, _P]),
    ("ht_vote_hit_masked", _I32, [_P, _P, _P, _I32, _P, _P, _P, _P]),
    ("ht_vote_swept", _I32, [_P, _P, _P, _I32, _P, _P, _P]),
    ("ht_mlp_param_count", _I32, []),
    ("ht_mlp_timeouts", ctypes.c_int64, []),
    ("ht_mlp_forward", _I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P]),
    ("ht_mlp_region_mask", _I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, ctypes.c_float,
                                  ctypes.c_float, _I32, _P, _P, _P]),
    ("ht_mlp_hit_masks", _I32, [_P, _P, _P, _P, _P, _I32, _I32, ctypes.c_float, _P, _P]),
    ("ht_mlp_backward_workspace_size", _SZ, [_I32]),
    ("ht_mlp_backward", _I32, [_P, _P, _I32, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("ht_mlp_adam", _I32, [_P, _P, _P, _P, _I32, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, ctypes.c_float, _P, _P]),
    ("ht_batch_run_masked", _I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    ("ht_batch_run_learned", _I32, [_P, _P, _P, _P, _P, _I32, ctypes.POINTER(_Proposal), _P,
                                    _P, _P, _P, _P, _P, _P]),
    ("ht_batch_run_hit_masked", _I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P,
                                       _P]),
    ("ht_batch_run_learned_hits", _I32, [_P, _P, _P, _P, _P, _I32,
                                         ctypes.POINTER(_HitProposal), _P, _P, _P, _P, _P, _P,
                                         _P]),
    ("ht_fit_workspace_size", _SZ, [_I32, _I32, _I32]),
    ("ht_fit_tracks", _I32, [_P, _P, _P, _P, _I32, _I32, _P, _P, _P, _I32, _I32, _I32,
                             ctypes.c_double, ctypes.c_double, ctypes.c_double, _I32, _P, _P,
                             _SZ, _P]),
    ("ht_vertex_create", _I32, [_P, ctypes.POINTER(_VertexDesc), ctypes.POINTER(_P)]),
    ("ht_vertex_destroy", _I32, [_P]),
    ("ht_vertex_accumulator_bytes", _SZ, [_P]),
    ("ht_vertex_workspace_size", _SZ, [_P]),
    ("ht_vertex_vote", _I32, [_P, _P, _P, _I32, _I32, _P, _P, _P]),
    ("ht_vertex_find", _I32, [_P, _P, _I32, _P, _I32, _P, _P, _P, _SZ, _P]),
    ("ht_vote_layers", _I32, [_P, _P, _P, _P, _I32, _P, _P, _P]),
    ("ht_confirm_workspace_size", _SZ, [_P, _I32, _I32]),
    ("ht_confirm", _I32, [_P, ctypes.POINTER(_ConfirmDesc), _P, _P, _P, _I32, _P, _P, _I32,
                          _P, _P, _P, _P, _SZ, _P]),
    ("ht_batch_set_confirm", _I32, [_P, ctypes.POINTER(_ConfirmDesc)]),
    ("ht_batch_run_tracks", _I32, [_P, _P, _P, _P, _P, _P, _I32, ctypes.POINTER(_HitProposal),
                                   _P, _P, _P, _P, _P, _P, _P, _P]),
    ("ht_batch_run_tracks_host", _I32, [_P, _P, _P, _P, _P, _P, _I32,
                                        ctypes.POINTER(_HitProposal), _P, _I32, _P, _P, _P, _P]),
]


def library_path():
    return _build.LIB


def lib():
    """Load libht (building it first if its sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise HTError(f"libht not found at {path}")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, what):
    if status != 0:
        msg = lib().ht_last_error().decode(errors="replace")
        raise HTError(f"{what} failed (status {status}): {msg}")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Geometry:
    """Owns an ht_geometry handle created on the current CUDA device."""

    def __init__(self, g):
        self.desc = dict(g)
        d = _Desc(g["n_rho"], g["n_d0"], g["n_phi0"], g["n_z0"], g["n_cot"],
                  g["threshold"], g.get("count_bits", 32), 0, g["rho_max"],
                  g["d0_half"], g["z0_max"], g["cot_max"])
        h = ctypes.c_void_p()
        _check(lib().ht_geometry_create(ctypes.byref(d), ctypes.byref(h)),
               "ht_geometry_create")
        self.handle = h
        self.shape = (g["n_rho"], g["n_d0"], g["n_phi0"])
        self.acc_dtype = torch.int16 if g.get("count_bits", 32) == 16 else torch.int32

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ht_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def accumulator_bytes(self):
        return lib().ht_accumulator_bytes(self.handle)

    def find_peaks_workspace_size(self):
        return lib().ht_find_peaks_workspace_size(self.handle)

    def associate_workspace_size(self, n_hits, cap):
        return lib().ht_associate_workspace_size(self.handle, n_hits, cap)

    def vote_z_workspace_size(self, n_hits, cap):
        return lib().ht_vote_z_workspace_size(self.handle, n_hits, cap)

    def event_workspace_size(self, n_hits, cap):
        return lib().ht_event_workspace_size(self.handle, n_hits, cap)

    def new_accumulator(self, device="cuda"):
        return torch.empty(self.shape, dtype=self.acc_dtype, device=device)


def ht_vote(g, x, y, acc, stats=None, stream=None):
    n = x.numel()
    _check(lib().ht_vote(g.handle, _ptr(x), _ptr(y), n, _ptr(acc), _ptr(stats),
                         _stream(stream)), "ht_vote")


def ht_vote_layers(g, x, y, layer, acc, stats=None, stream=None):
    """Distinct-layer vote: a cell counts the layers of the hits voting in it."""
    _check(lib().ht_vote_layers(g.handle, _ptr(x), _ptr(y), _ptr(layer), x.numel(), _ptr(acc),
                                _ptr(stats), _stream(stream)), "ht_vote_layers")


def ht_confirm_workspace_size(g, n_hits, cap):
    return lib().ht_confirm_workspace_size(g.handle, n_hits, cap)


def ht_confirm(g, c, x, y, layer, peaks, d_count, cap, score, inliers, assign, workspace,
               stream=None):
    """Confirmation of the candidates and the final assignment (c: a dict
    for confirm_desc); score int32 [cap], inliers int32 [cap, 16]."""
    d = confirm_desc(c)
    _check(lib().ht_confirm(g.handle, ctypes.byref(d), _ptr(x), _ptr(y), _ptr(layer),
                            x.numel(), _ptr(peaks), _ptr(d_count), cap, _ptr(score),
                            _ptr(inliers), _ptr(assign), _ptr(workspace), workspace.numel(),
                            _stream(stream)), "ht_confirm")


def ht_find_peaks(g, acc, peaks, cap, d_count, workspace, stream=None):
    _check(lib().ht_find_peaks(g.handle, _ptr(acc), _ptr(peaks), cap, _ptr(d_count),
                               _ptr(workspace), workspace.numel(), _stream(stream)),
           "ht_find_peaks")


def ht_vote_masked(g, x, y, mask, acc, stats=None, stream=None):
    """Vote restricted to the regions of mask (device int64 [1])."""
    _check(lib().ht_vote_masked(g.handle, _ptr(x), _ptr(y), x.numel(), _ptr(mask), _ptr(acc),
                                _ptr(stats), _stream(stream)), "ht_vote_masked")


def ht_vote_hit_masked(g, x, y, hit_masks, acc, stats=None, stream=None):
    """Vote with hit h restricted to the regions of hit_masks[h] (device int64 [n])."""
    _check(lib().ht_vote_hit_masked(g.handle, _ptr(x), _ptr(y), x.numel(), _ptr(hit_masks),
                                    _ptr(acc), _ptr(stats), _stream(stream)),
           "ht_vote_hit_masked")


def ht_vote_swept(g, x, y, acc, stats=None, stream=None):
    """Swept-interval vote: each column votes the d0 bins swept across it."""
    _check(lib().ht_vote_swept(g.handle, _ptr(x), _ptr(y), x.numel(), _ptr(acc), _ptr(stats),
                               _stream(stream)), "ht_vote_swept")


def ht_find_peaks_masked(g, acc, mask, peaks, cap, d_count, workspace, stream=None):
    _check(lib().ht_find_peaks_masked(g.handle, _ptr(acc), _ptr(mask), _ptr(peaks), cap,
                                      _ptr(d_count), _ptr(workspace), workspace.numel(),
                                      _stream(stream)), "ht_find_peaks_masked")


def ht_mlp_param_count():
    return lib().ht_mlp_param_count()


def ht_mlp_timeouts():
    """Forward passes that gave up waiting on their tensor-core work."""
    return lib().ht_mlp_timeouts()


def ht_mlp_forward(params_bf16, x, y, z, layer, prob=None, h1=None, h2=None, feat=None,
                   stream=None):
    _check(lib().ht_mlp_forward(_ptr(params_bf16), _ptr(x), _ptr(y), _ptr(z), _ptr(layer),
                                x.numel(), _ptr(prob), _ptr(h1), _ptr(h2), _ptr(feat),
                                _stream(stream)), "ht_mlp_forward")


def ht_mlp_region_mask(params_bf16, x, y, z, layer, off, tau, fmax, grow, mass, masks,
                       stream=None):
    """off: device int32 [n_events + 1]; mass float32 [n_events, 64]; masks int64."""
    _check(lib().ht_mlp_region_mask(_ptr(params_bf16), _ptr(x), _ptr(y), _ptr(z), _ptr(layer),
                                    _ptr(off), off.numel() - 1, x.numel(), tau, fmax,
                                    int(grow), _ptr(mass), _ptr(masks), _stream(stream)),
           "ht_mlp_region_mask")


def ht_mlp_hit_masks(params_bf16, x, y, z, layer, topk, pmin, hit_masks, stream=None):
    """hit_masks (device int64 [n]) receives each hit's top-k region set."""
    _check(lib().ht_mlp_hit_masks(_ptr(params_bf16), _ptr(x), _ptr(y), _ptr(z), _ptr(layer),
                                  x.numel(), int(topk), float(pmin), _ptr(hit_masks),
                                  _stream(stream)), "ht_mlp_hit_masks")


def ht_mlp_backward_workspace_size(n):
    return lib().ht_mlp_backward_workspace_size(n)


def ht_mlp_backward(params_bf16, labels, prob, h1, h2, feat, grad, workspace, stream=None):
    _check(lib().ht_mlp_backward(_ptr(params_bf16), _ptr(labels), labels.numel(), _ptr(prob),
                                 _ptr(h1), _ptr(h2), _ptr(feat), _ptr(grad), _ptr(workspace),
                                 workspace.numel(), _stream(stream)), "ht_mlp_backward")


def ht_mlp_adam(params, m, v, grad, step, lr, beta1, beta2, eps, params_bf16, stream=None):
    _check(lib().ht_mlp_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), step, lr, beta1, beta2,
                             eps, _ptr(params_bf16), _stream(stream)), "ht_mlp_adam")


def ht_find_peaks_noalloc(g, acc, peaks, cap, d_count, stream=None):
    """ht_find_peaks with the library's fixed internal scratch (no workspace)."""
    _check(lib().ht_find_peaks_noalloc(g.handle, _ptr(acc), _ptr(peaks), cap, _ptr(d_count),
                                       _stream(stream)), "ht_find_peaks_noalloc")


def ht_associate(g, x, y, peaks, d_count, cap, assign, workspace, stream=None):
    _check(lib().ht_associate(g.handle, _ptr(x), _ptr(y), x.numel(), _ptr(peaks),
                              _ptr(d_count), cap, _ptr(assign), _ptr(workspace),
                              workspace.numel(), _stream(stream)), "ht_associate")


def ht_vote_z(g, x, y, z, assign, peaks, d_count, cap, out, workspace, stream=None):
    _check(lib().ht_vote_z(g.handle, _ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(assign),
                           _ptr(peaks), _ptr(d_count), cap, _ptr(out), _ptr(workspace),
                           workspace.numel(), _stream(stream)), "ht_vote_z")


def ht_run_event(g, hx, hy, hz, workspace, h_peaks, cap, h_count, h_assign, h_zres,
                 h_stats=None, stream=None):
    """Host-buffer path: hx, hy, hz and the outputs are CPU tensors."""
    _check(lib().ht_run_event(g.handle, _ptr(hx), _ptr(hy), _ptr(hz), hx.numel(),
                              _ptr(workspace), workspace.numel(), _ptr(h_peaks), cap,
                              _ptr(h_count), _ptr(h_assign), _ptr(h_zres), _ptr(h_stats),
                              _stream(stream)), "ht_run_event")


TRACK_FIELDS = ["rho", "d0", "phi0", "sig_rho", "sig_d0", "sig_phi0"]


def ht_fit_tracks(G, x, y, d_off, assign, peaks, d_count, cap, out, workspace, min_hits=4,
                  iters=5, sigma=20e-4, road=0.0, cut=0.0, iters2=3, stream=None):
    """Refit candidates.  out: uint8 tensor of n_events * cap * 64 bytes (one
    ht_track each); d_off: device int32 [n_events + 1]."""
    _check(lib().ht_fit_tracks(G.handle, _ptr(x), _ptr(y), _ptr(d_off), d_off.numel() - 1,
                               x.numel(), _ptr(assign), _ptr(peaks), _ptr(d_count), cap, min_hits,
                               iters, sigma, road, cut, iters2, _ptr(out), _ptr(workspace),
                               workspace.numel(), _stream(stream)), "ht_fit_tracks")


def ht_fit_workspace_size(n_events, cap, n_hits):
    return lib().ht_fit_workspace_size(n_events, cap, n_hits)


def tracks_to_numpy(buf, n):
    """The first n ht_track records of a uint8 tensor as a numpy record array."""
    import numpy as np
    dt = np.dtype([(f, "<f8") for f in TRACK_FIELDS] +
                  [("chi2", "<f4"), ("n_hits", "<i4"), ("status", "<i4"), ("reserved", "<i4")])
    assert dt.itemsize == 64
    return np.frombuffer(buf[:n * 64].cpu().numpy().tobytes(), dtype=dt)


class Vertex:
    """Second transform (ht_vertex_*) for candidates of geometry G; vd is a
    dict with n_r, n_theta, threshold, r_max, r_keep and optional min_count."""

    def __init__(self, G, vd, max_events, cap, device="cuda"):
        self.G, self.vd, self.cap = G, dict(vd), cap
        d = _VertexDesc(vd["n_r"], vd["n_theta"], vd["threshold"], vd.get("min_count", 0),
                        vd["r_max"], vd["r_keep"])
        h = ctypes.c_void_p()
        _check(lib().ht_vertex_create(G.handle, ctypes.byref(d), ctypes.byref(h)),
               "ht_vertex_create")
        self.handle = h
        dev = torch.device(device)
        self.acc = torch.empty((max_events, vd["n_r"], vd["n_theta"]), dtype=torch.int32,
                               device=dev)
        self.peaks = torch.empty((max_events * cap, 4), dtype=torch.int32, device=dev)
        self.counts = torch.zeros(max_events, dtype=torch.int32, device=dev)
        self.first = torch.zeros(max_events, dtype=torch.int32, device=dev)
        self.stats = torch.zeros(2 * max_events, dtype=torch.int64, device=dev)
        self.ws = torch.empty(max(lib().ht_vertex_workspace_size(h), 256), dtype=torch.uint8,
                              device=dev)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ht_vertex_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, cands, d_count, cand_cap, n_events, stream=None):
        """Vote and find for n_events events of candidates (device peaks laid
        out e * cand_cap, counts d_count)."""
        s = _stream(stream)
        _check(lib().ht_vertex_vote(self.handle, _ptr(cands), _ptr(d_count), cand_cap, n_events,
                                    _ptr(self.acc), _ptr(self.stats), s), "ht_vertex_vote")
        _check(lib().ht_vertex_find(self.handle, _ptr(self.acc), n_events, _ptr(self.peaks),
                                    self.cap, _ptr(self.counts), _ptr(self.first),
                                    _ptr(self.ws), self.ws.numel(), s), "ht_vertex_find")

    def event_results(self, e):
        cnt = int(self.counts[e].item())
        k = min(cnt, self.cap)
        return dict(acc=self.acc[e].cpu().numpy(), count=cnt,
                    peaks=self.peaks[e * self.cap:e * self.cap + k].cpu().numpy(),
                    first=int(self.first[e].item()), votes=int(self.stats[2 * e].item()),
                    redo=int(self.stats[2 * e + 1].item()))


class EventPipeline:
    """Device buffers for one event of up to `max_hits` hits and `cap`
    candidates, and the four calls of the path in order."""

    def __init__(self, g, max_hits, cap, device="cuda"):
        self.g, self.cap, self.max_hits = g, cap, max_hits
        dev = torch.device(device)
        self.acc = g.new_accumulator(dev)
        self.peaks = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.assign = torch.empty(max(max_hits, 1), dtype=torch.int32, device=dev)
        self.zres = torch.empty((max(cap, 1), 3), dtype=torch.int32, device=dev)
        self.stats = torch.zeros(2, dtype=torch.int64, device=dev)
        ws = max(g.find_peaks_workspace_size(), g.associate_workspace_size(max_hits, cap),
                 g.vote_z_workspace_size(max_hits, cap))
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=dev)

    def run(self, x, y, z, stream=None, swept=False):
        """swept: the swept-interval vote (ht_vote_swept) instead of ht_vote."""
        n = x.numel()
        assert n <= self.max_hits
        g = self.g
        (ht_vote_swept if swept else ht_vote)(g, x, y, self.acc, self.stats, stream)
        ht_find_peaks(g, self.acc, self.peaks, self.cap, self.count, self.workspace, stream)
        ht_associate(g, x, y, self.peaks, self.count, self.cap, self.assign[:n],
                     self.workspace, stream)
        ht_vote_z(g, x, y, z, self.assign[:n], self.peaks, self.count, self.cap, self.zres,
                  self.workspace, stream)

    def results(self, n):
        """Copy results to numpy (synchronises)."""
        import numpy as np
        cnt = int(self.count.item())
        k = min(cnt, self.cap)
        acc = self.acc.cpu().numpy()
        if acc.dtype == np.int16:
            acc = acc.view(np.uint16)
        return dict(acc=acc, count=cnt, peaks=self.peaks[:k].cpu().numpy(),
                    assign=self.assign[:n].cpu().numpy(), zres=self.zres[:k].cpu().numpy(),
                    stats=self.stats.cpu().numpy().astype(np.uint64))


class Batch:
    """Batched runtime (ht_batch_*): caller-owned device outputs for up to
    `max_events` events, `max_hits` hits in total, `cap` candidates each."""

    def __init__(self, g, max_events, max_hits, cap, device="cuda"):
        import numpy as np
        self.g, self.max_events, self.max_hits, self.cap = g, max_events, max_hits, cap
        h = ctypes.c_void_p()
        _check(lib().ht_batch_create(g.handle, max_events, max_hits, cap, ctypes.byref(h)),
               "ht_batch_create")
        self.handle = h
        dev = torch.device(device)
        self.peaks = torch.empty((max_events * cap, 4), dtype=torch.int32, device=dev)
        self.zres = torch.empty((max_events * cap, 3), dtype=torch.int32, device=dev)
        self.counts = torch.zeros(max_events, dtype=torch.int32, device=dev)
        self.assign = torch.empty(max(max_hits, 1), dtype=torch.int32, device=dev)
        self.stats = torch.zeros(2 * max_events, dtype=torch.int64, device=dev)
        self._off = np.zeros(max_events + 1, np.int32)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ht_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graphs(self, enable):
        _check(lib().ht_batch_set_graphs(self.handle, int(bool(enable))), "ht_batch_set_graphs")

    def _offsets(self, offsets):
        import numpy as np
        off = np.ascontiguousarray(offsets, np.int32)
        return off, off.ctypes.data_as(ctypes.c_void_p)

    def run(self, x, y, z, offsets, stream=None):
        """x, y, z: device float32 (concatenated hits); offsets: host ints."""
        off, p = self._offsets(offsets)
        self._keep = off
        _check(lib().ht_batch_run(self.handle, _ptr(x), _ptr(y), _ptr(z), p, off.shape[0] - 1,
                                  _ptr(self.peaks), _ptr(self.counts), _ptr(self.assign),
                                  _ptr(self.zres), _ptr(self.stats), _stream(stream)),
               "ht_batch_run")

    def run_masked(self, x, y, z, offsets, masks, stream=None):
        """run() with event e's vote and peaks restricted to masks[e]
        (device int64 [n_events])."""
        off, p = self._offsets(offsets)
        self._keep = off
        _check(lib().ht_batch_run_masked(self.handle, _ptr(x), _ptr(y), _ptr(z), p,
                                         off.shape[0] - 1, _ptr(masks), _ptr(self.peaks),
                                         _ptr(self.counts), _ptr(self.assign), _ptr(self.zres),
                                         _ptr(self.stats), _stream(stream)),
               "ht_batch_run_masked")

    def run_learned(self, x, y, z, layer, offsets, params_bf16, masks, tau, fmax, grow=0,
                    stream=None):
        """run() with the masks proposed by the MLP inside the same graph;
        masks (device int64 [n_events]) receives them."""
        off, p = self._offsets(offsets)
        self._keep = off
        self._prop = _Proposal(params_bf16.data_ptr(), layer.data_ptr(), tau, fmax, int(grow), 0)
        _check(lib().ht_batch_run_learned(self.handle, _ptr(x), _ptr(y), _ptr(z), p,
                                          off.shape[0] - 1, ctypes.byref(self._prop),
                                          _ptr(masks), _ptr(self.peaks), _ptr(self.counts),
                                          _ptr(self.assign), _ptr(self.zres), _ptr(self.stats),
                                          _stream(stream)), "ht_batch_run_learned")

    def run_hit_masked(self, x, y, z, offsets, hit_masks, stream=None):
        """run() with each hit's vote restricted to hit_masks[h] (device
        int64 [total hits], indexed like x)."""
        off, p = self._offsets(offsets)
        self._keep = off
        _check(lib().ht_batch_run_hit_masked(self.handle, _ptr(x), _ptr(y), _ptr(z), p,
                                             off.shape[0] - 1, _ptr(hit_masks),
                                             _ptr(self.peaks), _ptr(self.counts),
                                             _ptr(self.assign), _ptr(self.zres),
                                             _ptr(self.stats), _stream(stream)),
               "ht_batch_run_hit_masked")

    def run_learned_hits(self, x, y, z, layer, offsets, params_bf16, hit_masks, topk, pmin=0.0,
                         stream=None):
        """run() with each hit's region set (its top-k regions) proposed by
        the MLP inside the same graph; hit_masks (device int64 [total hits])
        receives them."""
        off, p = self._offsets(offsets)
        self._keep = off
        self._hprop = _HitProposal(params_bf16.data_ptr(), layer.data_ptr(), int(topk),
                                   float(pmin))
        _check(lib().ht_batch_run_learned_hits(self.handle, _ptr(x), _ptr(y), _ptr(z), p,
                                               off.shape[0] - 1, ctypes.byref(self._hprop),
                                               _ptr(hit_masks), _ptr(self.peaks),
                                               _ptr(self.counts), _ptr(self.assign),
                                               _ptr(self.zres), _ptr(self.stats),
                                               _stream(stream)), "ht_batch_run_learned_hits")

    def set_confirm(self, c):
        """Switch on the track path with confirmation parameters c (a dict
        for confirm_desc); allocates the per-candidate score output."""
        self._conf = confirm_desc(c)
        _check(lib().ht_batch_set_confirm(self.handle, ctypes.byref(self._conf)),
               "ht_batch_set_confirm")
        if getattr(self, "score", None) is None:
            self.score = torch.zeros(self.max_events * self.cap, dtype=torch.int32,
                                     device=self.peaks.device)

    def run_tracks(self, x, y, z, layer, offsets, params_bf16=None, hit_masks=None, topk=8,
                   pmin=0.0, stream=None):
        """The track path (ht_batch_run_tracks): distinct-layer vote, peaks at
        each event's band threshold, confirmation, z vote.  With params_bf16
        the proposal's per-hit top-k sets restrict the vote (written to
        hit_masks, device int64 [total hits]); with hit_masks alone, the given
        sets do."""
        off, p = self._offsets(offsets)
        self._keep = off
        prop = None
        if params_bf16 is not None:
            assert hit_masks is not None
            self._hprop = _HitProposal(params_bf16.data_ptr(), layer.data_ptr(), int(topk),
                                       float(pmin))
            prop = ctypes.byref(self._hprop)
        _check(lib().ht_batch_run_tracks(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(layer), p,
                                         off.shape[0] - 1, prop, _ptr(hit_masks),
                                         _ptr(self.peaks), _ptr(self.counts), _ptr(self.score),
                                         _ptr(self.assign), _ptr(self.zres), _ptr(self.stats),
                                         _stream(stream)), "ht_batch_run_tracks")

    def run_tracks_host(self, hx, hy, hz, hlayer, offsets, tracks, ntracks, assign,
                        params_bf16=None, topk=8, pmin=0.0, stats=None, stream=None):
        """ht_batch_run_tracks_host: host (numpy or pinned torch) hit arrays
        in; tracks (int32 [track_cap, 8] host: i, j, k, count, score, n_z0,
        m_cot, zcount), ntracks (int32 [n_events]) and assign (int32 [hits])
        host outputs written; synchronous.  Returns False when the tracks
        exceeded track_cap (the first track_cap were written)."""
        off, p = self._offsets(offsets)
        prop = None
        if params_bf16 is not None:
            self._hprop = _HitProposal(params_bf16.data_ptr(), None, int(topk), float(pmin))
            prop = ctypes.byref(self._hprop)

        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)

        st = lib().ht_batch_run_tracks_host(self.handle, hp(hx), hp(hy), hp(hz), hp(hlayer), p,
                                            off.shape[0] - 1, prop, hp(tracks),
                                            int(tracks.shape[0]), hp(ntracks), hp(assign),
                                            hp(stats), _stream(stream))
        if st == 2:   # HT_ERR_CAPACITY: counts still written
            return False
        _check(st, "ht_batch_run_tracks_host")
        return True

    def stage_ms(self):
        """[proposal, vote, peaks + candidate lists, association (track path:
        confirmation and assignment), decode + z vote] ms of the last
        completed run (synchronise first)."""
        arr = (ctypes.c_float * 5)()
        _check(lib().ht_batch_stage_ms(self.handle, ctypes.cast(arr, ctypes.c_void_p)),
               "ht_batch_stage_ms")
        return list(arr)

    def autotune(self, x, y, z, offsets, stream=None):
        off, p = self._offsets(offsets)
        c = ctypes.c_int32()
        _check(lib().ht_batch_autotune(self.handle, _ptr(x), _ptr(y), _ptr(z), p,
                                       off.shape[0] - 1, _ptr(self.peaks), _ptr(self.counts),
                                       _ptr(self.assign), _ptr(self.zres), ctypes.byref(c),
                                       _stream(stream)), "ht_batch_autotune")
        v = c.value
        return dict(kt_pack=v & 255, kt_unpacked=(v >> 8) & 255, kt_assoc=(v >> 16) & 255)

    def event_results(self, offsets, e):
        """Results of event e as numpy arrays (synchronises)."""
        cnt = int(self.counts[e].item())
        k = min(cnt, self.cap)
        a, b = int(offsets[e]), int(offsets[e + 1])
        base = e * self.cap
        r = dict(count=cnt, peaks=self.peaks[base:base + k].cpu().numpy(),
                 zres=self.zres[base:base + k].cpu().numpy(),
                 assign=self.assign[a:b].cpu().numpy(),
                 votes=int(self.stats[2 * e].item()))
        if getattr(self, "score", None) is not None:
            r["score"] = self.score[base:base + k].cpu().numpy()
        return r
