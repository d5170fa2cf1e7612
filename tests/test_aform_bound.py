"""The vote tile's A-form error bound, checked on the CPU.

The vote evaluates most (hit, column) items in the A-form: the root with
|w| < c of rho w^2 + 2 w + rho c^2 = 0 (w = d0 + s), written as
u = A0 - rho c2d / (1 + sqrt(1 - rho^2 c^2)) with A0 = off - s / delta and
c2d = c^2 / delta precomputed per item in float32, and a bin is voted only
when the floors of u - e and u + e agree, with e = eA + |rho| eB a
first-order bound derived in tiles.cuh.  These tests restate the kernel's
float32 steps with numpy (each operation rounded to float32 once; the fused
multiply-adds formed in float64 and rounded once; the approximate rsqrt and
rcp pushed to both ends of their error bounds) and check, on the geometries
of every workload and of the extreme-geometry GPU tests, that the float32
coordinate lies within e of the coordinate the float64 definition gives
(b = 1 + rho s, q = -(b + sgn(b) sqrt(D)), root C / q, u = root / delta + off),
on tiles of 32 and of 64 rows.
A bound a twentieth as large fails, so the check has teeth, and dropping the
b > 0 condition of the A-form (the item's one root is then the other branch)
is caught too.
"""
import math
import zlib

import numpy as np
import pytest

F32 = np.float32
U = 2.0 ** -24
KAPPA_B = 0.299792458e-2 * 3.8

# geometry (n_rho, n_d0, n_phi0, rho_max, d0_half) and the hit radius range (cm)
GEOMS = {
    "single_64": ((64, 64, 64, KAPPA_B, 10.0), (4.0, 110.0)),
    "event100_256": ((256, 128, 512, KAPPA_B, 20.0), (4.0, 110.0)),
    "pileup_512": ((512, 256, 1024, KAPPA_B / 0.5, 30.0), (4.0, 110.0)),
    "fine_bins_far_hits": ((64, 256, 256, 0.002, 0.05), (0.6, 3000.0)),
    "tight_curls": ((48, 64, 96, 0.15, 3.0), (1.0, 12.0)),
    "straight_far": ((32, 64, 128, 2e-5, 1.0), (1000.0, 20000.0)),
}


def fma32(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def items(geom, rr, n, seed, TR=32):
    """Random hits x random columns x random TR-row tiles of a geometry."""
    NR, ND, NP, rmax, dh = geom
    rng = np.random.default_rng(seed)
    r = np.exp(rng.uniform(math.log(rr[0]), math.log(rr[1]), n))
    ph = rng.uniform(-math.pi, math.pi, n)
    x = (r * np.cos(ph)).astype(F32)
    y = (r * np.sin(ph)).astype(F32)
    k = rng.integers(0, NP, n)
    t0 = rng.integers(0, (NR + TR - 1) // TR, n) * TR
    i = np.minimum(t0 + rng.integers(0, TR, n), NR - 1)
    return x, y, k, t0, i, TR


def emulate(geom, x, y, k, t0, i, TR, scale=1.0, need_b_positive=True, rsq_err=0.0,
            rcp_err=0.0):
    """Float32 A-form coordinate, its bound and the float64 definition's
    coordinate for the items the kernel would put in A-form."""
    NR, ND, NP, rmax, dh = geom
    delta = 2.0 * dh / ND
    off = ND / 2 + 0.5
    invd, off_f = F32(1.0 / delta), F32(off)
    rho64 = (2 * np.arange(NR) + 1 - NR) * (rmax / NR)
    phi = (2 * np.arange(NP) + 1 - NP) * (math.pi / NP)
    sn64, cs64 = np.sin(phi), np.cos(phi)
    sn32, cs32 = sn64.astype(F32), cs64.astype(F32)
    ilast = np.minimum(t0 + TR - 1, NR - 1)
    rt = np.maximum(np.abs(rho64[t0]), np.abs(rho64[ilast])).astype(F32) * F32(1.0001)
    s = fma32(x, sn32[k], -(y * cs32[k]))
    c = fma32(x, cs32[k], y * sn32[k])
    R1 = np.abs(x) + np.abs(y)
    eS = F32(4e-7) * R1
    # root B out of the axis (the vote's sB / cB tests), then the A-form tests
    dext = dh + delta
    sB = (1.0 / rt - dext) * (1 - 1e-6) - 0.01
    cB = np.sqrt(np.maximum(1.0 / rt ** 2 - dext * dext, 0.0)) * (1 - 1e-6) - 0.05
    plain = ~((np.abs(s) + eS >= sB) & (c + eS >= cB)) & (c > F32(12 * U) * R1)
    t = rt * rt * (c * c) * F32(1.001)
    ok = plain & (c >= F32(4e-4) * R1) & (R1 >= F32(1e-20)) & (1 - t >= 0.015625)
    ok &= (R1 + rt * c * c) * invd + off_f + 1 < 2e6
    if need_b_positive:
        ok &= rt * (F32(4e-7) * R1 + np.abs(s)) < 0.99
    sel = np.nonzero(ok)[0]
    s, c, R1, eS, t, rt, i, k = (a[sel] for a in (s, c, R1, eS, t, rt, i, k))
    X, Y = x[sel].astype(np.float64), y[sel].astype(np.float64)
    # the record (make_aform)
    c2 = c * c
    A0 = fma32(-s, invd, off_f)
    c2d = F32(c2 * invd)
    rc = F32(2.0) * eS * F32(1.0 / c) * F32(1.001)
    dD = fma32(t, rc + F32(5 * U), F32(U))
    isD = F32(1.0 / np.sqrt(1.0 - t)) * F32(1.001)
    aA = np.abs(A0)
    e64 = 1.6e-14 * (rt * R1 * R1 + 2 * R1) * invd + 4e-15 * (aA + rt * c2d + off_f)
    eA = F32(4.004 * ((U * np.abs(s) + eS) * invd + 2 * U * aA) + e64)
    eB = F32(4.004 * c2d * (rc + 14.3 * U + dD * isD))
    # the lane's row (aform_bin)
    rho32 = rho64[i].astype(F32)
    D = fma32(-(rho32 * rho32), c2, F32(1.0))
    rs = F32(1.0 / np.sqrt(np.float64(D)) * (1.0 + rsq_err))
    den = fma32(D, rs, F32(1.0))
    ir = F32(1.0 / np.float64(den) * (1.0 + rcp_err))
    u32 = fma32(-(rho32 * c2d), ir, A0)
    e = fma32(np.abs(rho32), eB, eA) * F32(scale)
    # the float64 definition
    rho = rho64[i]
    s64 = X * sn64[k] - Y * cs64[k]
    c64 = X * cs64[k] + Y * sn64[k]
    b = 1.0 + rho * s64
    q = -(b + np.where(b >= 0, 1.0, -1.0) * np.sqrt(1.0 - (rho * c64) ** 2))
    C = rho * (X * X + Y * Y) + 2.0 * s64
    u64 = (C / q) / delta + off
    return np.float64(u32), np.float64(e), u64


@pytest.mark.parametrize("TR", [32, 64])
@pytest.mark.parametrize("name", sorted(GEOMS))
def test_float32_coordinate_within_the_bound(name, TR):
    """Tiles of 32 rows (the masked and per-hit votes) and 64 rows (the
    distinct-layer vote)."""
    geom, rr = GEOMS[name]
    it = items(geom, rr, 60000, seed=zlib.crc32(name.encode()) & 0xffff, TR=TR)
    worst = 0.0
    n = 0
    for rsq in (-2 ** -22.9, 2 ** -22.9):
        for rcp in (-2 ** -23.0, 2 ** -23.0):
            u32, e, u64 = emulate(geom, *it, rsq_err=rsq, rcp_err=rcp)
            n = u32.size
            assert np.all(np.isfinite(u32)) and np.all(e > 0)
            worst = max(worst, float(np.max(np.abs(u32 - u64) / e)))
    assert n > 1000, f"too few A-form items ({n})"
    assert worst <= 1.0, f"float32 coordinate outside its bound: |u32 - u64| / e = {worst}"


def test_bound_has_teeth():
    """A twentieth of the bound is exceeded on the 10k-hit geometry."""
    geom, rr = GEOMS["event100_256"]
    it = items(geom, rr, 60000, seed=7)
    u32, e, u64 = emulate(geom, *it, scale=0.05, rsq_err=2 ** -22.9)
    assert np.any(np.abs(u32 - u64) > e)


def test_b_positive_condition_is_needed():
    """Without b > 0 on the tile, tight curls put items in A-form whose one
    root is the other branch: the coordinates then differ by whole bins."""
    geom, rr = GEOMS["tight_curls"]
    it = items(geom, rr, 60000, seed=11)
    u32, e, u64 = emulate(geom, *it, need_b_positive=False)
    assert np.max(np.abs(u32 - u64)) > 1.0
    u32, e, u64 = emulate(geom, *it)
    assert np.max(np.abs(u32 - u64) / e) <= 1.0
