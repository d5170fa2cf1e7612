"""Workload definitions: detector, generator mix and accumulator geometry.

Units are cm, GeV and tesla throughout.  The detector follows the simple
transverse-plane model of Section 5 of the paper (a beam pipe of 3.0 cm and
ten evenly spaced barrel layers out to 110 cm); the workloads below override
the innermost radius (4 cm), the hit resolution (20 um) and add z.

Each workload is a plain dict with two parts:
  ``geom``  the Hough-transform geometry (accumulator axes and ranges);
  ``gen``   the event-generator mix.

The four workloads are the single-event case (64^3 int32 accumulator, one
event of ~275 hits), the 100-event case (~10k hits per event, 256x128x512
uint16), the pile-up-like case (~50k hits per event, 512x256x1024 uint16) and
the batched stream (2000 events, hit counts log-uniform on [2k, 60k], the
100-event case's geometry and mix).
"""
import math

# Curvature per unit field over transverse momentum: rho[1/cm] = KAPPA * B[T] / pT[GeV].
KAPPA = 0.299792458e-2
B_FIELD = 3.8
# Ten barrel layers, evenly spaced from 4 cm to 110 cm.
LAYER_R = tuple(4.0 + l * 106.0 / 9.0 for l in range(10))
ETA_MAX = 2.5
HIT_SIGMA = 20e-4      # 20 um r-phi and z smear
Z0_SIGMA = 5.0


def _track(threshold, pool=4, min_layers=8, tol=0.01, bands=()):
    """Parameters of the dense-event track path (distinct-layer vote, peak
    threshold T counted in layers, confirmation; bands give the batched
    stream each event's T from its hit count: [(max_hits, T), ...])."""
    return dict(threshold=threshold, pool=pool, min_layers=min_layers, n_layers=10, tol=tol,
                bands=list(bands))


def _geom(n_rho, n_d0, n_phi0, pt_min, d0_half, count_bits, threshold=7,
          n_z0=128, n_cot=128, z0_max=32.0, cot_max=6.5):
    return dict(n_rho=n_rho, n_d0=n_d0, n_phi0=n_phi0,
                rho_max=KAPPA * B_FIELD / pt_min, d0_half=d0_half,
                n_z0=n_z0, n_cot=n_cot, z0_max=z0_max, cot_max=cot_max,
                threshold=threshold, count_bits=count_bits)


CONFIGS = {
    # One event: 25 tracks (20 prompt, 5 displaced with |d0| < 10 cm),
    # pT = 1 GeV + exponential(1 GeV) truncated at 20 GeV, +10% noise hits.
    "single_64": dict(
        geom=_geom(64, 64, 64, pt_min=1.0, d0_half=10.0, count_bits=32),
        gen=dict(n_tracks=25, n_displaced=5, d0_disp=10.0, pt_kind="trunc_exp",
                 pt_min=1.0, pt_scale=1.0, pt_max=20.0, noise_frac=0.10),
        # a column spans 10.8 cm at 110 cm: a wide pool, 6 layers, T = 3
        track=_track(3, pool=20, min_layers=6),
        events=1, seed0=0),
    # 100 events of ~10k hits: 5% displaced (|d0| < 20 cm), 15% noise.
    "event100_256": dict(
        geom=_geom(256, 128, 512, pt_min=1.0, d0_half=20.0, count_bits=16),
        gen=dict(target_hits=10000, disp_frac=0.05, d0_disp=20.0,
                 pt_kind="trunc_exp", pt_min=1.0, pt_scale=1.0, pt_max=20.0,
                 noise_frac=0.15),
        track=_track(9),
        events=100, seed0=0),
    # Pile-up-like: 20 events of ~50k hits, pT = 0.5 GeV + exponential(0.7 GeV)
    # capped at 100 GeV, 2% displaced (|d0| < 30 cm), 20% noise.
    "pileup_512": dict(
        geom=_geom(512, 256, 1024, pt_min=0.5, d0_half=30.0, count_bits=16),
        gen=dict(target_hits=50000, disp_frac=0.02, d0_disp=30.0,
                 pt_kind="shifted_exp", pt_min=0.5, pt_scale=0.7, pt_max=100.0,
                 noise_frac=0.20),
        track=_track(10, tol=0.006),
        events=20, seed0=0),
    # Batched stream: 2000 events, hit counts log-uniform on [2k, 60k],
    # generator mix and geometry of the 100-event case.
    "stream2000_256": dict(
        geom=_geom(256, 128, 512, pt_min=1.0, d0_half=20.0, count_bits=16),
        gen=dict(target_hits=None, hits_loguniform=(2000, 60000), disp_frac=0.05,
                 d0_disp=20.0, pt_kind="trunc_exp", pt_min=1.0, pt_scale=1.0,
                 pt_max=20.0, noise_frac=0.15),
        # per-event T by hit count; 60 um (3 sigma) inliers against the
        # random coincidences of the 20k-60k-hit events
        track=_track(10, tol=0.006, bands=[(4000, 7), (7000, 8), (12000, 9)]),
        # the learned proposal on this stream: each hit's top-8 regions; its
        # restricted vote lacks most background votes, so its thresholds sit
        # one layer lower
        learned=dict(topk=8, track=_track(10, tol=0.006, bands=[(4000, 6), (7000, 7),
                                                                  (12000, 8), (1 << 30, 9)])),
        events=2000, seed0=0),
    # Displaced jets (the scenario of Figs. 6 and 8-9): 4 jets of 10 tracks
    # from vertices at 5-25 cm, dispersion 15-60 degrees, jet tracks
    # pT = 5 GeV + exponential(10 GeV) truncated at 50 GeV, no prompt tracks,
    # 5% noise; the 100-event case's track geometry.  Vertex space: 16 radius
    # bins of 2 cm x 64 azimuth bins, T2 = 5, candidates with >= 9 votes,
    # beam pipe 3.0 cm.
    "jets4_256": dict(
        geom=_geom(256, 128, 512, pt_min=1.0, d0_half=20.0, count_bits=16),
        gen=dict(kind="jets", n_jets=4, tracks_per_jet=10, r_vertex=(5.0, 25.0),
                 dispersion_deg=(15.0, 60.0), jet_pt_min=5.0, jet_pt_scale=10.0,
                 jet_pt_max=50.0, n_prompt=0, pt_kind="trunc_exp", pt_min=1.0,
                 pt_scale=1.0, pt_max=20.0, noise_frac=0.05),
        vertex=dict(n_r=16, n_theta=64, r_max=32.0, threshold=5, min_count=9, r_keep=3.0),
        events=100, seed0=0),
    # The same with 2960 prompt tracks: 3000 tracks in all (Fig. 10's event).
    "jets3000_256": dict(
        geom=_geom(256, 128, 512, pt_min=1.0, d0_half=20.0, count_bits=16),
        gen=dict(kind="jets", n_jets=4, tracks_per_jet=10, r_vertex=(5.0, 25.0),
                 dispersion_deg=(15.0, 60.0), jet_pt_min=5.0, jet_pt_scale=10.0,
                 jet_pt_max=50.0, n_prompt=2960, pt_kind="trunc_exp", pt_min=1.0,
                 pt_scale=1.0, pt_max=20.0, noise_frac=0.05),
        vertex=dict(n_r=16, n_theta=64, r_max=32.0, threshold=5, min_count=9, r_keep=3.0),
        events=20, seed0=0),
}


def track_of(name):
    """The track path's parameters of a workload (None if it has none)."""
    t = CONFIGS[name].get("track")
    return None if t is None else dict(t, bands=list(t["bands"]))


def learned_of(name):
    """The learned proposal's parameters on a workload (None if none):
    {topk, track}."""
    l = CONFIGS[name].get("learned")
    return None if l is None else dict(topk=l["topk"], track=dict(l["track"], bands=list(l["track"]["bands"])))


def track_geometry(name, n_hits=None):
    """The workload's geometry with the track path's peak threshold (the
    band's for an event of n_hits hits, when bands are set)."""
    t = CONFIGS[name]["track"]
    g = geometry_of(name)
    g["threshold"] = t["threshold"]
    if n_hits is not None:
        for mh, thr in t["bands"]:
            if n_hits <= mh:
                g["threshold"] = thr
                break
    return g


def geometry_of(name, **overrides):
    """Return a copy of a workload's geometry dict with optional overrides."""
    g = dict(CONFIGS[name]["geom"])
    g.update(overrides)
    return g


def sinh_eta_max():
    return math.sinh(ETA_MAX)
