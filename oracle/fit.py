"""Oracle of the candidate refinement: a track fit of each candidate to its
assigned hits.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; it shares no code with the
CUDA path.

Section 5 says costlier computations confirm the candidates, and Section 6
names a Kalman filter for that step (run on the CPU there, with a GPU version
suggested).  With no material and no process noise a Kalman filter
over a track's hits computes the weighted least-squares estimate, which is
what this reading fits directly:

* Parameters p = (rho, d0, phi0), started at the candidate's cell centre
  (rho_i, d0_j = (j - n_d0/2) delta, phi0_k).
* Residual of hit (x, y): F / 2 with F = rho d0^2 + 2 (1 + rho s) d0 +
  rho r^2 + 2 s, s = x sin phi0 - y cos phi0 (F / 2 is the signed distance
  of the hit from the circle to first order; equal hit weights).
* Jacobian of F / 2: (d0^2 + 2 s d0 + r^2) / 2, rho d0 + 1 + rho s,
  (1 + rho d0) c with c = x cos phi0 + y sin phi0.
* `iters` Gauss-Newton steps: solve (J^T J) dp = -J^T r by Cholesky,
  p += dp (a non-positive pivot stops the fit with status -1).  chi2 =
  sum r^2 / sigma^2 and the covariance sigma^2 (J^T J)^-1 at the final p.
Only candidates with at least `min_hits` assigned hits are fitted.
Optional hit selection (the road of a track finder, the outlier cut of a
Kalman filter): fit only the hits within `road` cm of the cell-centre
circle, then refit the hits within `cut` sigma of the fitted one.
All arithmetic float64.
"""
import math

import numpy as np

from . import oracle as O


def residuals(p, x, y):
    rho, d0, phi0 = p
    sn, cs = math.sin(phi0), math.cos(phi0)
    s = x * sn - y * cs
    c = x * cs + y * sn
    r2 = x * x + y * y
    F = rho * d0 * d0 + 2.0 * (1.0 + rho * s) * d0 + rho * r2 + 2.0 * s
    J = np.stack([(d0 * d0 + 2.0 * s * d0 + r2) * 0.5,
                  rho * d0 + 1.0 + rho * s,
                  (1.0 + rho * d0) * c], axis=1)
    return 0.5 * F, J


def cholesky3(A):
    """Lower Cholesky factor of a 3 x 3 matrix, or None if a pivot is not
    positive (the normal matrix is singular to working precision)."""
    L = np.zeros((3, 3))
    for i in range(3):
        for j in range(i + 1):
            v = A[i, j] - sum(L[i, k] * L[j, k] for k in range(j))
            if i == j:
                if not v > 0.0:
                    return None
                L[i, i] = math.sqrt(v)
            else:
                L[i, j] = v / L[j, j]
    return L


def fit_one(p0, x, y, iters=5, sigma=20e-4):
    """(p, chi2, covariance, status) of one track: status 1 fitted, -1 the
    normal matrix lost positive definiteness (p is the last good one)."""
    p = np.array(p0, np.float64)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    status = 1
    for _ in range(iters):
        r, J = residuals(p, x, y)
        L = cholesky3(J.T @ J)
        if L is None:
            status = -1
            break
        g = J.T @ r
        p = p - np.linalg.solve(L.T, np.linalg.solve(L, g))
    r, J = residuals(p, x, y)
    L = cholesky3(J.T @ J)
    if L is None:
        return p, float(np.sum(r * r) / (sigma * sigma)), np.full((3, 3), np.nan), -1
    Li = np.linalg.inv(L)
    cov = (Li.T @ Li) * sigma * sigma
    return p, float(np.sum(r * r) / (sigma * sigma)), cov, status


def cell_start(g, pk, tables=None):
    """Fit start at the cell centre of candidate pk = (i, j, k, count)."""
    phi0, _, _, rho = O.tables(g) if tables is None else tables
    delta = 2.0 * g["d0_half"] / g["n_d0"]
    return (rho[pk[0]], (pk[1] - 0.5 * g["n_d0"]) * delta, phi0[pk[2]])


def select(p, x, y, width):
    """Hits whose residual at p is at most width (cm) in magnitude."""
    r, _ = residuals(p, x, y)
    return np.abs(r) <= width


def fit_candidates(g, x, y, assign, peaks, min_hits=4, iters=5, sigma=20e-4, road=None,
                   cut=None, iters2=3):
    """Per candidate m: dict(p, chi2, n, cov, status) or None when fewer
    than min_hits hits are assigned to it.

    With road (cm): only hits within road of the cell-centre circle are
    fitted; with cut (in sigma): after the fit, the assigned hits within
    cut * sigma of the fitted circle are refitted with iters2 more steps
    from the first fit.  n is the number of hits in the last fit; fewer
    than min_hits there gives status 0 (p is the last start)."""
    assign = np.asarray(assign)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    tables = O.tables(g)
    out = []
    for m, pk in enumerate(np.asarray(peaks)):
        sel = np.nonzero(assign == m)[0]
        if sel.shape[0] < min_hits:
            out.append(None)
            continue
        xs, ys = x[sel], y[sel]
        p0 = np.array(cell_start(g, pk, tables), np.float64)
        keep = select(p0, xs, ys, road) if road is not None else np.ones(sel.shape[0], bool)
        if keep.sum() < min_hits:
            out.append(dict(p=p0, chi2=np.nan, n=int(keep.sum()), cov=None, status=0))
            continue
        p, chi2, cov, st = fit_one(p0, xs[keep], ys[keep], iters, sigma)
        n = int(keep.sum())
        if cut is not None and st == 1:
            keep = select(p, xs, ys, cut * sigma)
            n = int(keep.sum())
            if n < min_hits:
                out.append(dict(p=p, chi2=np.nan, n=n, cov=None, status=0))
                continue
            p, chi2, cov, st = fit_one(p, xs[keep], ys[keep], iters2, sigma)
        out.append(dict(p=p, chi2=chi2, n=n, cov=cov, status=st))
    return out
