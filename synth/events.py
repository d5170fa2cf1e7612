"""Monte Carlo event generator for a barrel silicon tracker in a solenoid.

Track model (transverse plane, perigee parametrisation):
  t = (cos phi0, sin phi0), n = (-sin phi0, cos phi0), P = d0 * n,
  X(theta) = P + (sin theta / rho) t + ((1 - cos theta) / rho) n,
where rho is the signed curvature (> 0 counter-clockwise) and theta = rho * L
the turning angle after transverse arc length L >= 0.  Along z:
z(L) = z0 + L * cot(theta_polar).

A track leaves one hit on each layer of radius r > |d0| that it reaches on
its first half turn: |X(theta)|^2 = r^2 gives
  1 - cos theta = rho^2 (r^2 - d0^2) / (2 (1 + rho d0)),
and a layer is crossed iff that value lies in [0, 2).  Hits are smeared along
the layer (r stays on the layer) and in z.  Positions are computed in float64
and rounded to float32 once.

Random numbers come from numpy's Philox4x32-10 counter-based generator, one
stream per event seed.
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .configs import (KAPPA, B_FIELD, LAYER_R, ETA_MAX, HIT_SIGMA, Z0_SIGMA,
                      CONFIGS)


@dataclass
class Event:
    x: np.ndarray          # float32 [n_hits]
    y: np.ndarray          # float32 [n_hits]
    z: np.ndarray          # float32 [n_hits]
    layer: np.ndarray      # int8    [n_hits]
    track: np.ndarray      # int32   [n_hits], -1 for noise hits
    # truth per track
    rho: np.ndarray = field(default_factory=lambda: np.zeros(0))
    d0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    phi0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    z0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    cot: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pt: np.ndarray = field(default_factory=lambda: np.zeros(0))
    n_track_hits: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    # displaced-jet truth (jet events only): jet of each track (-1 prompt),
    # vertex radius and azimuth of each jet
    jet: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    vr: np.ndarray = field(default_factory=lambda: np.zeros(0))
    vtheta: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_hits(self):
        return int(self.x.shape[0])


def _rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def helix_hits(rho, d0, phi0, z0=0.0, cot=0.0, radii=LAYER_R):
    """Exact (unsmeared) float64 hits of one track on the given layer radii.

    Returns (x, y, z, layer_index, L) for the layers the track reaches on its
    first half turn.  rho must be nonzero or the track is a straight line
    (rho == 0 handled as the limit: X = P + L t).
    """
    radii = np.asarray(radii, dtype=np.float64)
    lay = np.arange(radii.shape[0])
    t = np.array([math.cos(phi0), math.sin(phi0)])
    nv = np.array([-math.sin(phi0), math.cos(phi0)])
    ok = radii > abs(d0)
    if rho == 0.0:
        L = np.sqrt(np.maximum(radii ** 2 - d0 * d0, 0.0))
        X = d0 * nv[0] + L * t[0]
        Y = d0 * nv[1] + L * t[1]
    else:
        A = rho * rho * (radii ** 2 - d0 * d0) / (2.0 * (1.0 + rho * d0))
        ok &= (A >= 0.0) & (A < 2.0) & (1.0 + rho * d0 > 0.0)
        A = np.where(ok, A, 0.0)
        tha = np.arccos(1.0 - A)
        th = math.copysign(1.0, rho) * tha
        L = tha / abs(rho)
        X = d0 * nv[0] + (np.sin(th) / rho) * t[0] + ((1.0 - np.cos(th)) / rho) * nv[0]
        Y = d0 * nv[1] + (np.sin(th) / rho) * t[1] + ((1.0 - np.cos(th)) / rho) * nv[1]
    Z = z0 + L * cot
    return X[ok], Y[ok], Z[ok], lay[ok], L[ok]


def _draw_tracks(rng, gen, n):
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    u = rng.random(n)
    if gen["pt_kind"] == "trunc_exp":
        lo, sc, hi = gen["pt_min"], gen["pt_scale"], gen["pt_max"]
        pt = lo - sc * np.log1p(-u * (1.0 - math.exp(-(hi - lo) / sc)))
    else:  # shifted exponential, capped
        pt = np.minimum(gen["pt_min"] - gen["pt_scale"] * np.log1p(-u), gen["pt_max"])
    rho = -q * KAPPA * B_FIELD / pt
    phi0 = rng.uniform(-math.pi, math.pi, n)
    eta = rng.uniform(-ETA_MAX, ETA_MAX, n)
    cot = np.sinh(eta)
    z0 = rng.normal(0.0, Z0_SIGMA, n)
    return rho, phi0, cot, z0, pt


def _tracks_to_hits(rng, rho, d0, phi0, z0, cot):
    """Vectorised helix_hits over tracks x layers, with smearing."""
    r = np.asarray(LAYER_R)[None, :]
    rho_ = rho[:, None]
    d0_ = d0[:, None]
    A = rho_ * rho_ * (r * r - d0_ * d0_) / (2.0 * (1.0 + rho_ * d0_))
    ok = (r > np.abs(d0_)) & (A >= 0.0) & (A < 2.0) & (1.0 + rho_ * d0_ > 0.0)
    A = np.where(ok, A, 0.0)
    tha = np.arccos(1.0 - A)
    th = np.sign(rho_) * tha
    L = tha / np.abs(rho_)
    c0, s0 = np.cos(phi0)[:, None], np.sin(phi0)[:, None]
    a = np.sin(th) / rho_
    b = (1.0 - np.cos(th)) / rho_
    X = -d0_ * s0 + a * c0 - b * s0
    Y = d0_ * c0 + a * s0 + b * c0
    Z = z0[:, None] + L * cot[:, None]
    tr, lay = np.nonzero(ok)
    X, Y, Z = X[tr, lay], Y[tr, lay], Z[tr, lay]
    rl = np.asarray(LAYER_R)[lay]
    phi = np.arctan2(Y, X) + rng.normal(0.0, HIT_SIGMA, X.shape[0]) / rl
    Z = Z + rng.normal(0.0, HIT_SIGMA, X.shape[0])
    return rl * np.cos(phi), rl * np.sin(phi), Z, lay, tr


def make_event(gen, seed, target_hits=None):
    """Generate one event from a generator mix dict (see configs.CONFIGS)."""
    rng = _rng(seed)
    if target_hits is None:
        target_hits = gen.get("target_hits")
    if target_hits is None and gen.get("hits_loguniform"):
        lo, hi = gen["hits_loguniform"]
        target_hits = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    nf = gen["noise_frac"]
    if target_hits is None:
        n = gen["n_tracks"]
        rho, phi0, cot, z0, pt = _draw_tracks(rng, gen, n)
        d0 = np.zeros(n)
        nd = gen.get("n_displaced", 0)
        d0[n - nd:] = rng.uniform(-gen["d0_disp"], gen["d0_disp"], nd)
        hx, hy, hz, lay, tr = _tracks_to_hits(rng, rho, d0, phi0, z0, cot)
    else:
        want = target_hits / (1.0 + nf)
        parts, total, ntr = [], 0, 0
        batch = max(64, int(want / 8))
        while total < want:
            rho, phi0, cot, z0, pt = _draw_tracks(rng, gen, batch)
            disp = rng.random(batch) < gen["disp_frac"]
            d0 = np.where(disp, rng.uniform(-gen["d0_disp"], gen["d0_disp"], batch), 0.0)
            hx, hy, hz, lay, tr = _tracks_to_hits(rng, rho, d0, phi0, z0, cot)
            per = np.bincount(tr, minlength=batch)
            cum = total + np.cumsum(per)
            stop = int(np.searchsorted(cum, want, side="left"))
            keep_tracks = batch if stop >= batch else stop + 1
            sel = tr < keep_tracks
            parts.append((rho[:keep_tracks], d0[:keep_tracks], phi0[:keep_tracks],
                          z0[:keep_tracks], cot[:keep_tracks], pt[:keep_tracks],
                          hx[sel], hy[sel], hz[sel], lay[sel], tr[sel] + ntr))
            total += int(per[:keep_tracks].sum())
            ntr += keep_tracks
        rho, d0, phi0, z0, cot, pt = (np.concatenate([p[i] for p in parts]) for i in range(6))
        hx, hy, hz, lay, tr = (np.concatenate([p[i] for p in parts]) for i in range(6, 11))
    n_track_hits = np.bincount(tr, minlength=rho.shape[0]).astype(np.int32)
    nn = int(round(nf * hx.shape[0]))
    nl = rng.integers(0, len(LAYER_R), nn)
    rl = np.asarray(LAYER_R)[nl]
    nphi = rng.uniform(-math.pi, math.pi, nn)
    nz = rng.uniform(-1.0, 1.0, nn) * rl * math.sinh(ETA_MAX)
    X = np.concatenate([hx, rl * np.cos(nphi)])
    Y = np.concatenate([hy, rl * np.sin(nphi)])
    Z = np.concatenate([hz, nz])
    LAY = np.concatenate([lay, nl]).astype(np.int8)
    TR = np.concatenate([tr, np.full(nn, -1)]).astype(np.int32)
    perm = rng.permutation(X.shape[0])
    return Event(x=X[perm].astype(np.float32), y=Y[perm].astype(np.float32),
                 z=Z[perm].astype(np.float32), layer=LAY[perm], track=TR[perm],
                 rho=rho, d0=d0, phi0=phi0, z0=z0, cot=cot, pt=pt,
                 n_track_hits=n_track_hits)


def perigee_of(vx, vy, psi, rho):
    """Perigee parameters (d0, phi0) of the circle of signed curvature rho
    through (vx, vy) with direction psi there (rho == 0: the straight line).

    The centre is C = V + n_psi / rho with n_psi = (-sin psi, cos psi); the
    perigee is the circle's point closest to the origin, where the left
    normal is n = sign(rho) C / |C|, so phi0 = atan2(-n_x, n_y) and
    d0 = sign(rho) (|C| - 1/|rho|)."""
    vx, vy, psi, rho = (np.asarray(a, np.float64) for a in (vx, vy, psi, rho))
    straight = rho == 0.0
    rs = np.where(straight, 1.0, rho)
    R = 1.0 / rs
    cx = vx - R * np.sin(psi)
    cy = vy + R * np.cos(psi)
    cn = np.hypot(cx, cy)
    sg = np.sign(rs)
    nx, ny = sg * cx / cn, sg * cy / cn
    d0 = np.where(straight, -vx * np.sin(psi) + vy * np.cos(psi), sg * (cn - np.abs(R)))
    phi0 = np.where(straight, psi, np.arctan2(-nx, ny))
    return d0, phi0


def make_jet_event(gen, seed):
    """Displaced-jet event: n_jets jets of tracks_per_jet tracks from vertices
    at radius uniform in r_vertex and uniform azimuth, track directions
    uniform within half the jet's dispersion angle (uniform in
    dispersion_deg) of the vertex's radial direction, plus n_prompt tracks
    from the origin; hits only on layers outside the vertex; noise hits as
    in make_event."""
    rng = _rng(seed)
    nj, tpj = gen["n_jets"], gen["tracks_per_jet"]
    vr = rng.uniform(*gen["r_vertex"], nj)
    vth = rng.uniform(-math.pi, math.pi, nj)
    disp = np.radians(rng.uniform(*gen["dispersion_deg"], nj))
    nt_j = nj * tpj
    jet_of = np.repeat(np.arange(nj), tpj)
    psi = vth[jet_of] + rng.uniform(-0.5, 0.5, nt_j) * disp[jet_of]
    q = np.where(rng.random(nt_j) < 0.5, -1.0, 1.0)
    u = rng.random(nt_j)
    lo, sc, hi = gen["jet_pt_min"], gen["jet_pt_scale"], gen["jet_pt_max"]
    pt_j = lo - sc * np.log1p(-u * (1.0 - math.exp(-(hi - lo) / sc)))
    rho_j = -q * KAPPA * B_FIELD / pt_j
    vx, vy = vr[jet_of] * np.cos(vth[jet_of]), vr[jet_of] * np.sin(vth[jet_of])
    d0_j, phi0_j = perigee_of(vx, vy, psi, rho_j)
    cot_j = np.sinh(rng.uniform(-ETA_MAX, ETA_MAX, nt_j))
    z0_j = np.repeat(rng.normal(0.0, Z0_SIGMA, nj), tpj)
    npr = gen.get("n_prompt", 0)
    rho_p, phi0_p, cot_p, z0_p, pt_p = _draw_tracks(rng, gen, npr)
    rho = np.concatenate([rho_j, rho_p])
    d0 = np.concatenate([d0_j, np.zeros(npr)])
    phi0 = np.concatenate([phi0_j, phi0_p])
    cot = np.concatenate([cot_j, cot_p])
    z0 = np.concatenate([z0_j, z0_p])
    pt = np.concatenate([pt_j, pt_p])
    jet = np.concatenate([jet_of, np.full(npr, -1)]).astype(np.int32)
    hx, hy, hz, lay, tr = _tracks_to_hits(rng, rho, d0, phi0, z0, cot)
    # a jet track starts at its vertex: drop the layers inside it
    rv_tr = np.where(jet >= 0, vr[np.maximum(jet, 0)], 0.0)
    keep = np.asarray(LAYER_R)[lay] > rv_tr[tr]
    hx, hy, hz, lay, tr = hx[keep], hy[keep], hz[keep], lay[keep], tr[keep]
    n_track_hits = np.bincount(tr, minlength=rho.shape[0]).astype(np.int32)
    nf = gen["noise_frac"]
    nn = int(round(nf * hx.shape[0]))
    nl = rng.integers(0, len(LAYER_R), nn)
    rl = np.asarray(LAYER_R)[nl]
    nphi = rng.uniform(-math.pi, math.pi, nn)
    nz = rng.uniform(-1.0, 1.0, nn) * rl * math.sinh(ETA_MAX)
    X = np.concatenate([hx, rl * np.cos(nphi)])
    Y = np.concatenate([hy, rl * np.sin(nphi)])
    Z = np.concatenate([hz, nz])
    LAY = np.concatenate([lay, nl]).astype(np.int8)
    TR = np.concatenate([tr, np.full(nn, -1)]).astype(np.int32)
    perm = rng.permutation(X.shape[0])
    return Event(x=X[perm].astype(np.float32), y=Y[perm].astype(np.float32),
                 z=Z[perm].astype(np.float32), layer=LAY[perm], track=TR[perm],
                 rho=rho, d0=d0, phi0=phi0, z0=z0, cot=cot, pt=pt,
                 n_track_hits=n_track_hits, jet=jet, vr=vr, vtheta=vth)


def make_stream(name, n_events=None, seed0=None):
    """Yield the events of a named workload (seed = seed0 + event index)."""
    cfg = CONFIGS[name]
    n_events = cfg["events"] if n_events is None else n_events
    seed0 = cfg["seed0"] if seed0 is None else seed0
    for e in range(n_events):
        yield generate(cfg["gen"], seed0 + e)


def generate(gen, seed):
    """One event of a generator mix (jet mixes go to make_jet_event)."""
    if gen.get("kind") == "jets":
        return make_jet_event(gen, seed)
    return make_event(gen, seed)
