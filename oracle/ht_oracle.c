/*
 * ht_oracle.c -- plain, slow CPU oracle for Hough-transform track finding.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library and its binding) never calls it and shares no code with it.
 *
 * Method: Halyo, LeGresley, Lujan, "Massively Parallel Computing and the
 * Search for Jets and Black Holes at the LHC", arXiv:1309.6275.
 *   Section 5   the Hough transform: every instance of a parametrised feature
 *               starts at zero votes; each input adds one vote to every
 *               instance that would contain it; local maxima of the vote
 *               space are the candidate features, which costlier steps then
 *               confirm.
 *   Section 6   (Fig. 5) hits -> transform -> peak finding -> refinement.
 *   Section 7   the peak finder is tuned for tracks of at least seven hits.
 * The paper gives no formulas, bin layout or tie rules.  The readings used
 * here (each marked "reading") are stated where they are applied.
 *
 * Arithmetic: IEEE binary64, round to nearest.  Compile with -O2
 * -ffp-contract=off and without fast-math, so that every + - * / sqrt below is
 * one correctly rounded operation in the order written.
 *
 * Parametrisation (reading; the paper says only that the transform measures
 * the transverse momentum of prompt or displaced tracks):
 *   signed curvature rho (> 0 counter-clockwise), transverse impact
 *   parameter d0 and azimuth phi0 at the perigee.  A circle with these
 *   parameters passes through hit (x, y) iff
 *     F(d0) = rho d0^2 + 2 (1 + rho s) d0 + (rho r^2 + 2 s) = 0,
 *   s = x sin phi0 - y cos phi0,  c = x cos phi0 + y sin phi0,  r^2 = x^2 + y^2,
 *   with discriminant / 4   D = 1 - (rho c)^2.
 *   rho and phi0 are sampled at bin centres; d0 is solved and binned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_rho, n_d0, n_phi0;
    int32_t n_z0, n_cot;
    int32_t threshold;
    int64_t count_max;  /* saturation value of a cell: 65535 (uint16) or 2^31-1 */
    double rho_max, d0_half, z0_max, cot_max;
} or_geom;

static const double OR_PI = 3.141592653589793;        /* nearest double to pi */
static const double OR_HALF_PI = 1.5707963267948966;  /* OR_PI / 2, exact */

/* Axis tables (reading): phi0_k = (2k + 1 - N) pi / N covers [-pi, pi);
 * rho_i = (2i + 1 - N) rho_max / N covers [-rho_max, rho_max). */
void or_tables(const or_geom *g, double *phi0, double *sn, double *cs, double *rho)
{
    for (int32_t k = 0; k < g->n_phi0; ++k) {
        double p = (double)(2 * k + 1 - g->n_phi0) * (OR_PI / (double)g->n_phi0);
        phi0[k] = p;
        sn[k] = sin(p);
        cs[k] = cos(p);
    }
    for (int32_t i = 0; i < g->n_rho; ++i)
        rho[i] = (double)(2 * i + 1 - g->n_rho) * (g->rho_max / (double)g->n_rho);
}

/* Column edges (reading): e_k = (2k - N) pi / N, the lower edge of column k
 * (its centre phi0_k minus pi / N); sin/cos via libm. */
void or_edge_tables(const or_geom *g, double *sn, double *cs)
{
    for (int32_t k = 0; k < g->n_phi0; ++k) {
        const double e = (double)(2 * k - g->n_phi0) * (OR_PI / (double)g->n_phi0);
        sn[k] = sin(e);
        cs[k] = cos(e);
    }
}

/* d0 binning (reading): width delta = 2 d0_half / n_d0, bin coordinate
 * u = d0 / delta + (n_d0 / 2 + 0.5), bin j = floor(u), valid iff 0 <= u < n_d0.
 * So d0 = 0 is the centre of bin n_d0 / 2 (prompt tracks do not straddle an
 * edge) and the axis covers [-d0_half - delta/2, d0_half - delta/2). */
static double d0_delta(const or_geom *g) { return 2.0 * g->d0_half / (double)g->n_d0; }
static double d0_offset(const or_geom *g) { return (double)g->n_d0 * 0.5 + 0.5; }

/* The d0 bins voted by one hit in one (rho_i, phi0_k) column.
 * Forward condition (reading): only c > 0 votes -- the hit lies on the first
 * half turn.  Without it every circle would also appear as its mirror
 * (-rho, -d0, phi0 + pi) and every track would give two peaks.
 * Both real roots of F vote (both can be physical: the second is a hit past a
 * quarter turn).  A double root (D == 0) votes once.
 * Stable roots: q = -(b + sgn(b) sqrt(D)), b = 1 + rho s, sgn(0) = +1;
 * roots q / rho (rho != 0) and (rho r^2 + 2 s) / q (q != 0).
 * Returns the number of in-range roots written to j[]; *n_edge counts those
 * whose bin coordinate lies within 1e-5 of an integer. */
static int cell_bins(const or_geom *g, float xf, float yf, double sn, double cs,
                     double rho, int32_t j[2], int64_t *n_edge)
{
    const double delta = d0_delta(g), off = d0_offset(g);
    const double x = (double)xf, y = (double)yf;
    const double s = x * sn - y * cs;
    const double c = x * cs + y * sn;
    if (!(c > 0.0))
        return 0;
    const double r2 = x * x + y * y;
    const double b = 1.0 + rho * s;
    const double pc = rho * c;
    const double D = 1.0 - pc * pc;
    if (D < 0.0)
        return 0;
    const double sq = sqrt(D);
    const double q = -(b + (b >= 0.0 ? sq : -sq));
    const double C = rho * r2 + 2.0 * s;
    double root[2];
    int nr = 0;
    if (rho != 0.0)
        root[nr++] = q / rho;
    if (q != 0.0 && !(D == 0.0 && rho != 0.0))
        root[nr++] = C / q;
    int nv = 0;
    for (int t = 0; t < nr; ++t) {
        const double u = root[t] / delta + off;
        if (u >= 0.0 && u < (double)g->n_d0) {
            const double fl = floor(u);
            const double fr = u - fl;
            j[nv++] = (int32_t)fl;
            if (fr < 1e-5 || fr > 1.0 - 1e-5)
                ++*n_edge;
        }
    }
    return nv;
}

/* Section 5 vote.  acc[(i n_d0 + j) n_phi0 + k] for rows i in [i_begin, i_end)
 * (the caller zeroes acc; rows outside the range are not touched, so callers
 * may split rows across threads).  Each vote adds one, saturating at
 * count_max (reading).  stats[0] += votes cast, stats[1] += edge votes. */
void or_vote(const or_geom *g, const float *x, const float *y, int64_t n,
             int32_t i_begin, int32_t i_end, int64_t *acc, int64_t *stats)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    int64_t votes = 0, edge = 0;
    for (int64_t h = 0; h < n; ++h)
        for (int32_t i = i_begin; i < i_end; ++i)
            for (int32_t k = 0; k < g->n_phi0; ++k) {
                int32_t j[2];
                const int nv = cell_bins(g, x[h], y[h], sn[k], cs[k], rho[i], j, &edge);
                for (int t = 0; t < nv; ++t) {
                    int64_t *cell = &acc[((int64_t)i * g->n_d0 + j[t]) * g->n_phi0 + k];
                    if (*cell < g->count_max)
                        ++*cell;
                    ++votes;
                }
            }
    stats[0] += votes;
    stats[1] += edge;
    free(phi0); free(sn); free(cs); free(rho);
}

/* Per-hit region proposals (the learned proposal's per-hit variant; the paper
 * has no learned part).  Regions (reading): an 8 x 8 grid over the rho rows
 * and d0 bins, cell (i, j) in region 8 (i 8 / n_rho) + (j 8 / n_d0) (integer
 * division).  A hit may vote in cell (i, j) iff some cell (i', j') with
 * |i - i'| <= 1 and |j - j'| <= 1 (inside the axes) lies in one of the
 * regions of its mask: its regions plus a one-cell halo, so that a track
 * whose peak sits on a region edge keeps the votes around it. */
static int in_hit_halo(const or_geom *g, uint64_t mask, int32_t i, int32_t j)
{
    for (int32_t di = -1; di <= 1; ++di)
        for (int32_t dj = -1; dj <= 1; ++dj) {
            const int32_t ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= g->n_rho || jj < 0 || jj >= g->n_d0)
                continue;
            const int32_t r = (ii * 8 / g->n_rho) * 8 + jj * 8 / g->n_d0;
            if ((mask >> r) & 1u)
                return 1;
        }
    return 0;
}

/* or_vote with every vote of hit h dropped unless its cell is allowed by
 * mask[h] (in_hit_halo).  stats[0] counts the votes cast, stats[1] the
 * in-range roots near a bin edge, allowed or not (as cell_bins counts them). */
void or_vote_hitmask(const or_geom *g, const float *x, const float *y, const uint64_t *mask,
                     int64_t n, int32_t i_begin, int32_t i_end, int64_t *acc, int64_t *stats)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    int64_t votes = 0, edge = 0;
    for (int64_t h = 0; h < n; ++h)
        for (int32_t i = i_begin; i < i_end; ++i)
            for (int32_t k = 0; k < g->n_phi0; ++k) {
                int32_t j[2];
                int64_t e = 0;
                const int nv = cell_bins(g, x[h], y[h], sn[k], cs[k], rho[i], j, &e);
                for (int t = 0; t < nv; ++t) {
                    if (!in_hit_halo(g, mask[h], i, j[t]))
                        continue;
                    int64_t *cell = &acc[((int64_t)i * g->n_d0 + j[t]) * g->n_phi0 + k];
                    if (*cell < g->count_max)
                        ++*cell;
                    ++votes;
                }
                edge += e;
            }
    stats[0] += votes;
    stats[1] += edge;
    free(phi0); free(sn); free(cs); free(rho);
}

/* Swept-interval vote (reading; the paper samples phi0 at bin centres and
 * notes that the transform tolerates data the discretisation cannot
 * represent exactly).  Column k covers phi0 from its lower edge
 * e_k = (2k - N) pi / N to e_{(k+1) mod N} (the same angle as e_k + 2 pi / N,
 * taken from the same table).  The hit's roots are sampled at the lower edge,
 * the centre phi0_k and the upper edge.  At each sample t the roots exist
 * when c > 0 and D >= 0; they are labelled by branch, + = (-b + sqrt D) / rho
 * and - = (-b - sqrt D) / rho (rho == 0: only +, = -s; D == 0: both equal),
 * and each gets a code: floor(u) inside the axis, -1 below it, n_d0 above.
 * Per branch, two consecutive samples that both have the root give every
 * bin between their codes (clamped to the axis; nothing if both are on the
 * same side outside); a sample whose neighbours lack the root gives its own
 * bin.  The cell (i, j, k) gets one vote when bin j is in the union of these
 * ranges over both branches. */
typedef struct {
    int ok[2];      /* branch + / - has a root at this sample */
    int64_t code[2];
} sweep_sample;

static int64_t u_code(const or_geom *g, double u)
{
    if (u < 0.0)
        return -1;
    if (u >= (double)g->n_d0)
        return g->n_d0;
    return (int64_t)floor(u);
}

static sweep_sample sweep_at(const or_geom *g, float xf, float yf, double sn, double cs,
                             double rho)
{
    sweep_sample r = {{0, 0}, {0, 0}};
    const double delta = d0_delta(g), off = d0_offset(g);
    const double x = (double)xf, y = (double)yf;
    const double s = x * sn - y * cs;
    const double c = x * cs + y * sn;
    if (!(c > 0.0))
        return r;
    const double r2 = x * x + y * y;
    const double b = 1.0 + rho * s;
    const double pc = rho * c;
    const double D = 1.0 - pc * pc;
    if (D < 0.0)
        return r;
    const double sq = sqrt(D);
    const double q = -(b + (b >= 0.0 ? sq : -sq));
    const double C = rho * r2 + 2.0 * s;
    if (rho == 0.0) {               /* one root, C / q = -s */
        r.ok[0] = 1;
        r.code[0] = u_code(g, (C / q) / delta + off);
        return r;
    }
    if (D == 0.0) {                 /* double root */
        r.ok[0] = r.ok[1] = 1;
        r.code[0] = r.code[1] = u_code(g, (q / rho) / delta + off);
        return r;
    }
    const int64_t cA = u_code(g, (C / q) / delta + off);
    const int64_t cB = u_code(g, (q / rho) / delta + off);
    /* b >= 0: C / q is the + root and q / rho the - root; b < 0: swapped */
    r.ok[0] = r.ok[1] = 1;
    r.code[0] = b >= 0.0 ? cA : cB;
    r.code[1] = b >= 0.0 ? cB : cA;
    return r;
}

/* Marks bins [lo, hi] (clamped) in mark[] and widens the touched span
 * [*t_lo, *t_hi]. */
static void mark_range(const or_geom *g, int64_t lo, int64_t hi, unsigned char *mark,
                       int64_t *t_lo, int64_t *t_hi)
{
    if (hi < 0 || lo > g->n_d0 - 1)
        return;
    if (lo < 0)
        lo = 0;
    if (hi > g->n_d0 - 1)
        hi = g->n_d0 - 1;
    for (int64_t j = lo; j <= hi; ++j)
        mark[j] = 1;
    if (lo < *t_lo)
        *t_lo = lo;
    if (hi > *t_hi)
        *t_hi = hi;
}

/* Bins swept by one hit in one (rho_i, column k): mark[j] = 1 (mark has
 * n_d0 entries, clear on entry) for j in the touched span [*t_lo, *t_hi]
 * (empty when *t_lo > *t_hi).  sn/cs: the three samples' tables. */
static void swept_bins(const or_geom *g, float x, float y, const double sn[3],
                       const double cs[3], double rho, unsigned char *mark, int64_t *t_lo,
                       int64_t *t_hi)
{
    *t_lo = g->n_d0;
    *t_hi = -1;
    sweep_sample t[3];
    for (int a = 0; a < 3; ++a)
        t[a] = sweep_at(g, x, y, sn[a], cs[a], rho);
    for (int br = 0; br < 2; ++br) {
        for (int a = 0; a < 2; ++a)
            if (t[a].ok[br] && t[a + 1].ok[br]) {
                const int64_t c0 = t[a].code[br], c1 = t[a + 1].code[br];
                mark_range(g, c0 < c1 ? c0 : c1, c0 < c1 ? c1 : c0, mark, t_lo, t_hi);
            }
        for (int a = 0; a < 3; ++a) {
            const int left = a > 0 && t[a - 1].ok[br];
            const int right = a < 2 && t[a + 1].ok[br];
            if (t[a].ok[br] && !left && !right)
                mark_range(g, t[a].code[br], t[a].code[br], mark, t_lo, t_hi);
        }
    }
}

/* Swept vote of rows [i_begin, i_end): acc as or_vote (caller zeroes it,
 * saturating at count_max); stats[0] += votes cast. */
void or_vote_swept(const or_geom *g, const float *x, const float *y, int64_t n,
                   int32_t i_begin, int32_t i_end, int64_t *acc, int64_t *stats)
{
    const int32_t NP = g->n_phi0, ND = g->n_d0;
    double *phi0 = malloc(sizeof(double) * NP);
    double *sn = malloc(sizeof(double) * NP);
    double *cs = malloc(sizeof(double) * NP);
    double *esn = malloc(sizeof(double) * NP);
    double *ecs = malloc(sizeof(double) * NP);
    double *rho = malloc(sizeof(double) * g->n_rho);
    unsigned char *mark = calloc((size_t)ND, 1);
    or_tables(g, phi0, sn, cs, rho);
    or_edge_tables(g, esn, ecs);
    int64_t votes = 0;
    for (int64_t h = 0; h < n; ++h)
        for (int32_t i = i_begin; i < i_end; ++i)
            for (int32_t k = 0; k < NP; ++k) {
                const int32_t k1 = (k + 1) % NP;
                const double s3[3] = {esn[k], sn[k], esn[k1]};
                const double c3[3] = {ecs[k], cs[k], ecs[k1]};
                int64_t t_lo, t_hi;
                swept_bins(g, x[h], y[h], s3, c3, rho[i], mark, &t_lo, &t_hi);
                for (int64_t j = t_lo; j <= t_hi; ++j)
                    if (mark[j]) {
                        mark[j] = 0;
                        int64_t *cell = &acc[((int64_t)i * ND + j) * NP + k];
                        if (*cell < g->count_max)
                            ++*cell;
                        ++votes;
                    }
            }
    stats[0] += votes;
    free(phi0); free(sn); free(cs); free(esn); free(ecs); free(rho); free(mark);
}

/* Peak finding (Sections 5 and 6: local maxima of the vote space; Section 7:
 * tuned for tracks of at least seven hits).  Reading: cell
 * l = (i n_d0 + j) n_phi0 + k
 * is a peak iff acc[l] >= threshold and, for every existing one of its 26
 * neighbours l' (rho and d0 do not wrap, phi0 wraps modulo n_phi0),
 * acc[l] > acc[l'] when l' < l and acc[l] >= acc[l'] when l' > l -- so of a
 * plateau only the cell of smallest index can be a peak.
 * Rows i in [i_begin, i_end) are scanned in increasing l.  The first `cap`
 * peaks are written as {i, j, k, count}; the number found is returned. */
int64_t or_peaks(const or_geom *g, const int64_t *acc, int32_t i_begin, int32_t i_end,
                 int32_t *out, int64_t cap)
{
    const int32_t NR = g->n_rho, ND = g->n_d0, NP = g->n_phi0;
    int64_t cnt = 0;
    for (int32_t i = i_begin; i < i_end; ++i)
        for (int32_t j = 0; j < ND; ++j)
            for (int32_t k = 0; k < NP; ++k) {
                const int64_t l = ((int64_t)i * ND + j) * NP + k;
                const int64_t v = acc[l];
                if (v < g->threshold)
                    continue;
                int peak = 1;
                for (int di = -1; di <= 1 && peak; ++di)
                    for (int dj = -1; dj <= 1 && peak; ++dj)
                        for (int dk = -1; dk <= 1 && peak; ++dk) {
                            if (di == 0 && dj == 0 && dk == 0)
                                continue;
                            const int32_t ii = i + di, jj = j + dj;
                            if (ii < 0 || ii >= NR || jj < 0 || jj >= ND)
                                continue;
                            const int32_t kk = (k + dk + NP) % NP;
                            const int64_t l2 = ((int64_t)ii * ND + jj) * NP + kk;
                            const int64_t v2 = acc[l2];
                            if (l2 < l ? !(v > v2) : !(v >= v2))
                                peak = 0;
                        }
                if (!peak)
                    continue;
                if (cnt < cap) {
                    out[4 * cnt + 0] = i;
                    out[4 * cnt + 1] = j;
                    out[4 * cnt + 2] = k;
                    out[4 * cnt + 3] = (int32_t)v;
                }
                ++cnt;
            }
    return cnt;
}

/* Candidate confirmation (Section 5: "more expensive computations" confirm a
 * candidate).  Reading: hit h is compatible with candidate m = (i_m, j_m, k_m)
 * iff one of its votes lies in a cell with |i - i_m| <= 1, |j - j_m| <= 1 and
 * circular |k - k_m| <= 1.  The hit goes to the compatible candidate of
 * largest count, ties to the smallest m; -1 if none.
 * Hits hit_idx[0..n_sel) are processed (all n hits when hit_idx is NULL). */
void or_associate(const or_geom *g, const float *x, const float *y,
                  const int64_t *hit_idx, int64_t n_sel,
                  const int32_t *peaks, int64_t npk, int32_t *assign)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    int64_t edge = 0;
    for (int64_t t = 0; t < n_sel; ++t) {
        const int64_t h = hit_idx ? hit_idx[t] : t;
        int32_t best = -1, best_count = -1;
        for (int64_t m = 0; m < npk; ++m) {
            const int32_t im = peaks[4 * m], jm = peaks[4 * m + 1], km = peaks[4 * m + 2];
            const int32_t cm = peaks[4 * m + 3];
            int compat = 0;
            for (int a = -1; a <= 1 && !compat; ++a) {
                const int32_t ii = im + a;
                if (ii < 0 || ii >= g->n_rho)
                    continue;
                for (int dk = -1; dk <= 1 && !compat; ++dk) {
                    const int32_t kk = (km + dk + g->n_phi0) % g->n_phi0;
                    int32_t j[2];
                    const int nv = cell_bins(g, x[h], y[h], sn[kk], cs[kk], rho[ii], j, &edge);
                    for (int v = 0; v < nv; ++v)
                        if (abs(j[v] - jm) <= 1)
                            compat = 1;
                }
            }
            if (compat && cm > best_count) {
                best = (int32_t)m;
                best_count = cm;
            }
        }
        assign[t] = best;
    }
    free(phi0); free(sn); free(cs); free(rho);
}

/* The same association rule by a second route, for full-size events: hit h
 * casts its votes (the vote's own cell_bins); each vote cell and its 26
 * neighbours are looked up in cand_at[] (candidate index of every cell, -1
 * if none), and the compatible candidate of largest count, smallest index
 * wins.  Hits hit_idx[0..n_sel). */
void or_associate_dense(const or_geom *g, const float *x, const float *y,
                        const int64_t *hit_idx, int64_t n_sel, const int32_t *peaks,
                        const int32_t *cand_at, int32_t *assign)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    const int32_t NR = g->n_rho, ND = g->n_d0, NP = g->n_phi0;
    int64_t edge = 0;
    for (int64_t t = 0; t < n_sel; ++t) {
        const int64_t h = hit_idx[t];
        int32_t best = -1, best_count = -1;
        for (int32_t i = 0; i < NR; ++i)
            for (int32_t k = 0; k < NP; ++k) {
                int32_t j[2];
                const int nv = cell_bins(g, x[h], y[h], sn[k], cs[k], rho[i], j, &edge);
                for (int v = 0; v < nv; ++v)
                    for (int di = -1; di <= 1; ++di)
                        for (int dj = -1; dj <= 1; ++dj)
                            for (int dk = -1; dk <= 1; ++dk) {
                                const int32_t ii = i + di, jj = j[v] + dj;
                                if (ii < 0 || ii >= NR || jj < 0 || jj >= ND)
                                    continue;
                                const int32_t kk = (k + dk + NP) % NP;
                                const int32_t m = cand_at[((int64_t)ii * ND + jj) * NP + kk];
                                if (m < 0)
                                    continue;
                                const int32_t cm = peaks[4 * m + 3];
                                if (cm > best_count || (cm == best_count && m < best)) {
                                    best = m;
                                    best_count = cm;
                                }
                            }
            }
        assign[t] = best;
    }
    free(phi0); free(sn); free(cs); free(rho);
}

/* atan2 from basic operations only, so that a second implementation that
 * follows the same steps reproduces it bit for bit.  Method: reduce to
 * t = min(|y|, |x|) / max(|y|, |x|) in [0, 1]; apply the half-angle identity
 * atan(t) = 2 atan(t / (1 + sqrt(1 + t^2))) three times (|t| <= tan(pi/32));
 * sum the Maclaurin series atan(t) = sum_n (-1)^n t^(2n+1) / (2n+1) to n = 10
 * by Horner's rule; undo the reductions.  Error: a few ulp.
 * Returns 0 for (0, 0); atan2(-0.0, x < 0) returns +pi (sign of zero ignored). */
static double atan_unit(double t)
{
    for (int h = 0; h < 3; ++h)
        t = t / (1.0 + sqrt(1.0 + t * t));
    const double t2 = t * t;
    double p = 1.0 / 21.0;
    for (int k = 9; k >= 0; --k)
        p = 1.0 / (double)(2 * k + 1) - t2 * p;
    return 8.0 * (t * p);
}

double or_atan2(double y, double x)
{
    if (x == 0.0 && y == 0.0)
        return 0.0;
    const double ax = fabs(x), ay = fabs(y);
    double a;
    if (ay <= ax)
        a = atan_unit(ay / ax);
    else
        a = OR_HALF_PI - atan_unit(ax / ay);
    if (x < 0.0)
        a = OR_PI - a;
    return y < 0.0 ? -a : a;
}

void or_atan2_array(const double *y, const double *x, int64_t n, double *out)
{
    for (int64_t t = 0; t < n; ++t)
        out[t] = or_atan2(y[t], x[t]);
}

/* Second vote in (z0, cot theta) per candidate (reading; the paper is
 * transverse-plane only).  For candidate m at cell centres
 * (rho_i, d0_j = (j - n_d0/2) delta, phi0_k) and each hit assigned to it:
 * turning angle theta = atan2(rho c, 1 + rho (s + d0_j)), arc length
 * L = theta / rho (L = c when rho == 0); for each cot-theta centre
 * t_q = (2q + 1 - n_cot) cot_max / n_cot: z0 = z - L t_q, bin
 * u = (z0 + z0_max) / dz with dz = 2 z0_max / n_z0, n = floor(u), valid iff
 * 0 <= u < n_z0.  Output per candidate: argmax {n, q, count} over the
 * n_z0 x n_cot histogram, ties to the smallest n n_cot + q; {-1, -1, 0} when
 * no vote was cast.
 * Candidates cand[0..n_cand) are processed; the hits assigned to cand[t] are
 * list[off[t] .. off[t + 1]) (grouped by the caller); out has 3 int32 per
 * listed candidate. */
void or_vote_z(const or_geom *g, const float *x, const float *y, const float *z,
               const int32_t *peaks, const int64_t *cand, int64_t n_cand,
               const int64_t *off, const int64_t *list, int32_t *out)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    const int32_t NZ = g->n_z0, NC = g->n_cot;
    const double delta = d0_delta(g);
    const double dz = 2.0 * g->z0_max / (double)NZ;
    const double cstep = g->cot_max / (double)NC;
    int64_t *hist = malloc(sizeof(int64_t) * (size_t)NZ * NC);
    for (int64_t t = 0; t < n_cand; ++t) {
        const int64_t m = cand[t];
        const int32_t im = peaks[4 * m], jm = peaks[4 * m + 1], km = peaks[4 * m + 2];
        memset(hist, 0, sizeof(int64_t) * (size_t)NZ * NC);
        const double r = rho[im];
        const double d0c = ((double)jm - 0.5 * (double)g->n_d0) * delta;
        for (int64_t e = off[t]; e < off[t + 1]; ++e) {
            const int64_t h = list[e];
            const double xd = x[h], yd = y[h], zd = z[h];
            const double s = xd * sn[km] - yd * cs[km];
            const double c = xd * cs[km] + yd * sn[km];
            double L;
            if (r == 0.0)
                L = c;
            else
                L = or_atan2(r * c, 1.0 + r * (s + d0c)) / r;
            for (int32_t q = 0; q < NC; ++q) {
                const double tq = (double)(2 * q + 1 - NC) * cstep;
                const double z0 = zd - L * tq;
                const double u = (z0 + g->z0_max) / dz;
                if (u >= 0.0 && u < (double)NZ)
                    ++hist[(int64_t)floor(u) * NC + q];
            }
        }
        int64_t best = -1, bc = 0;
        for (int64_t b = 0; b < (int64_t)NZ * NC; ++b)
            if (hist[b] > bc) {
                bc = hist[b];
                best = b;
            }
        out[3 * t + 0] = best < 0 ? -1 : (int32_t)(best / NC);
        out[3 * t + 1] = best < 0 ? -1 : (int32_t)(best % NC);
        out[3 * t + 2] = (int32_t)bc;
    }
    free(hist);
    free(phi0); free(sn); free(cs); free(rho);
}

/* ------------------------------------------------------------------------
 * Track finding in dense events: the distinct-layer vote and the candidate
 * confirmation.
 *
 * Reading (the paper's detector has ten layers and its peak finder expects
 * tracks of seven or more hits, Sections 5 and 7; a track leaves at most one
 * hit per layer): a cell's count is the number of DISTINCT detector layers
 * among the hits that vote in it, instead of the number of votes.  Inner
 * layers are the densest (about a thousand hits on a circle of 25 cm at
 * 10k hits per event), and with plain counts their hits pile up tens of
 * votes in every cell of the d0 band they reach, which buries the 10-hit
 * tracks; counting each layer once removes that pile-up.  The votes are the
 * plain vote's (cell_bins), hit by hit. */

/* Distinct-layer vote.  layer[h] in [0, 16) is hit h's detector layer;
 * mask (NULL: every cell allowed) restricts hit h's votes to the cells that
 * in_hit_halo(mask[h]) allows, as in or_vote_hitmask.  acc holds rows
 * [i_begin, i_end) (the caller zeroes it): acc[cell] = number of distinct
 * layers among the hits voting in the cell.  stats[0] += votes cast,
 * stats[1] += in-range roots near a bin edge (as or_vote counts them). */
void or_vote_layers(const or_geom *g, const float *x, const float *y, const uint8_t *layer,
                    const uint64_t *mask, int64_t n, int32_t i_begin, int32_t i_end,
                    int64_t *acc, int64_t *stats)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    const int64_t row_cells = (int64_t)g->n_d0 * g->n_phi0;
    uint32_t *seen = calloc((size_t)((i_end - i_begin) * row_cells), sizeof(uint32_t));
    int64_t votes = 0, edge = 0;
    for (int64_t h = 0; h < n; ++h)
        for (int32_t i = i_begin; i < i_end; ++i)
            for (int32_t k = 0; k < g->n_phi0; ++k) {
                int32_t j[2];
                int64_t e = 0;
                const int nv = cell_bins(g, x[h], y[h], sn[k], cs[k], rho[i], j, &e);
                for (int t = 0; t < nv; ++t) {
                    if (mask && !in_hit_halo(g, mask[h], i, j[t]))
                        continue;
                    seen[(int64_t)(i - i_begin) * row_cells + (int64_t)j[t] * g->n_phi0 + k] |=
                        1u << layer[h];
                    ++votes;
                }
                edge += e;
            }
    for (int32_t i = i_begin; i < i_end; ++i)
        for (int64_t c = 0; c < row_cells; ++c) {
            const uint32_t bits = seen[(int64_t)(i - i_begin) * row_cells + c];
            int64_t nl = 0;
            for (int l = 0; l < 16; ++l)
                nl += (bits >> l) & 1u;
            acc[(int64_t)i * row_cells + c] = nl;
        }
    stats[0] += votes;
    stats[1] += edge;
    free(seen);
    free(phi0); free(sn); free(cs); free(rho);
}

typedef struct {
    int32_t pool;        /* inlier pool: bins within pool of the candidate's bin */
    int32_t min_layers;  /* a candidate is confirmed with at least this many inlier layers */
    int32_t n_layers;    /* layers are 0 .. n_layers - 1 (<= 16) */
    int32_t reserved;
    double tol;          /* inlier distance to the seed circle, cm */
} or_confirm_params;

/* Circle through three points (the circumcentre, from coordinates relative
 * to the first point): with a = P2 - P1, b = P3 - P1 and
 * d = 2 (a_x b_y - a_y b_x), the centre is P1 + ((b_y |a|^2 - a_y |b|^2) / d,
 * (a_x |b|^2 - b_x |a|^2) / d) and the radius its distance from P1.
 * Returns 0 when the points are collinear (d == 0). */
int or_circle3(double x1, double y1, double x2, double y2, double x3, double y3,
               double *xc, double *yc, double *R)
{
    const double ax = x2 - x1, ay = y2 - y1, bx = x3 - x1, by = y3 - y1;
    const double d = 2.0 * (ax * by - ay * bx);
    if (d == 0.0)
        return 0;
    const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
    const double ux = (by * a2 - ay * b2) / d;
    const double uy = (ax * b2 - bx * a2) / d;
    *xc = x1 + ux;
    *yc = y1 + uy;
    *R = sqrt(ux * ux + uy * uy);
    return 1;
}

/* Candidate confirmation (Section 5: costlier computations confirm a
 * candidate; Fig. 5 refines candidates by a fit).  Reading, for candidate
 * m = (i, j, k) and every hit h of the event, with the bins b of h's roots
 * in column (rho_i, phi0_k) exactly as the vote casts them (cell_bins):
 *   own(h)   some b == j             (h votes in the candidate's cell)
 *   pool(h)  some |b - j| <= pool    (h is near the cell in this column)
 * 1. Seed layers: the layers holding exactly one own hit, in increasing
 *    layer order; fewer than three: not confirmed.  la = the first, lc =
 *    the last, lb = the one between them whose index is closest to
 *    (la + lc) / 2 (smaller index on a tie).
 * 2. Seed circle: through the own hits of la, lb and lc (or_circle3);
 *    collinear seeds: not confirmed.
 * 3. Inliers: for each layer, the pool hit of that layer closest to the
 *    circle, |sqrt((x - xc)^2 + (y - yc)^2) - R| (smaller hit index on a
 *    tie), if that distance is below tol.
 * 4. score = the number of inlier layers; confirmed iff score >= min_layers.
 * Candidates m_begin .. m_end - 1 of peaks[0 .. npk); per candidate:
 * score[m] (0 when not confirmed), seeds[3 m .. 3 m + 2] (hit indices, -1
 * when there is no seed) and inl[16 m + l] (the inlier hit of layer l, -1
 * none; all -1 when not confirmed). */
void or_confirm(const or_geom *g, const or_confirm_params *p, const float *x, const float *y,
                const uint8_t *layer, int64_t n, const int32_t *peaks, int64_t m_begin,
                int64_t m_end, int32_t *score, int32_t *seeds, int32_t *inl)
{
    double *phi0 = malloc(sizeof(double) * g->n_phi0);
    double *sn = malloc(sizeof(double) * g->n_phi0);
    double *cs = malloc(sizeof(double) * g->n_phi0);
    double *rho = malloc(sizeof(double) * g->n_rho);
    or_tables(g, phi0, sn, cs, rho);
    unsigned char *own = malloc((size_t)(n > 0 ? n : 1));
    unsigned char *pool = malloc((size_t)(n > 0 ? n : 1));
    int64_t edge = 0;
    for (int64_t m = m_begin; m < m_end; ++m) {
        const int32_t im = peaks[4 * m], jm = peaks[4 * m + 1], km = peaks[4 * m + 2];
        score[m] = 0;
        seeds[3 * m] = seeds[3 * m + 1] = seeds[3 * m + 2] = -1;
        for (int l = 0; l < 16; ++l)
            inl[16 * m + l] = -1;
        int32_t n_own[16] = {0}, own_hit[16];
        for (int64_t h = 0; h < n; ++h) {
            int32_t j[2];
            const int nv = cell_bins(g, x[h], y[h], sn[km], cs[km], rho[im], j, &edge);
            own[h] = pool[h] = 0;
            for (int v = 0; v < nv; ++v) {
                if (j[v] == jm)
                    own[h] = 1;
                if (abs(j[v] - jm) <= p->pool)
                    pool[h] = 1;
            }
            if (own[h]) {
                ++n_own[layer[h]];
                own_hit[layer[h]] = (int32_t)h;
            }
        }
        int32_t sl[16], ns = 0;
        for (int l = 0; l < p->n_layers; ++l)
            if (n_own[l] == 1)
                sl[ns++] = l;
        if (ns < 3)
            continue;
        const int32_t la = sl[0], lc = sl[ns - 1];
        int32_t lb = -1, best_gap = 1 << 30;
        for (int t = 1; t < ns - 1; ++t) {
            const int32_t gap = abs(2 * sl[t] - (la + lc));
            if (gap < best_gap) {
                best_gap = gap;
                lb = sl[t];
            }
        }
        const int32_t ha = own_hit[la], hb = own_hit[lb], hc = own_hit[lc];
        seeds[3 * m] = ha;
        seeds[3 * m + 1] = hb;
        seeds[3 * m + 2] = hc;
        double xc, yc, R;
        if (!or_circle3((double)x[ha], (double)y[ha], (double)x[hb], (double)y[hb],
                        (double)x[hc], (double)y[hc], &xc, &yc, &R))
            continue;
        double best_d[16];
        int32_t best_h[16];
        for (int l = 0; l < 16; ++l) {
            best_d[l] = 0.0;
            best_h[l] = -1;
        }
        for (int64_t h = 0; h < n; ++h) {
            if (!pool[h])
                continue;
            const double dx = (double)x[h] - xc, dy = (double)y[h] - yc;
            const double d = fabs(sqrt(dx * dx + dy * dy) - R);
            const int l = layer[h];
            if (best_h[l] < 0 || d < best_d[l]) {
                best_d[l] = d;
                best_h[l] = (int32_t)h;
            }
        }
        int32_t sc = 0;
        for (int l = 0; l < p->n_layers; ++l)
            if (best_h[l] >= 0 && best_d[l] < p->tol)
                ++sc;
        if (sc < p->min_layers)
            continue;
        score[m] = sc;
        for (int l = 0; l < p->n_layers; ++l)
            if (best_h[l] >= 0 && best_d[l] < p->tol)
                inl[16 * m + l] = best_h[l];
    }
    free(own); free(pool);
    free(phi0); free(sn); free(cs); free(rho);
}

/* Final assignment after confirmation (reading): hit h goes to the confirmed
 * candidate that lists it as an inlier with the largest score, ties to the
 * smallest candidate index; -1 when no confirmed candidate lists it.
 * assign[0 .. n) is written. */
void or_confirm_assign(const int32_t *score, const int32_t *inl, int64_t npk, int64_t n,
                       int32_t *assign)
{
    int32_t *best = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t h = 0; h < n; ++h) {
        assign[h] = -1;
        best[h] = 0;
    }
    for (int64_t m = 0; m < npk; ++m) {
        if (score[m] <= 0)
            continue;
        for (int l = 0; l < 16; ++l) {
            const int32_t h = inl[16 * m + l];
            if (h < 0)
                continue;
            if (score[m] > best[h]) {   /* candidates in increasing m: ties keep the first */
                best[h] = score[m];
                assign[h] = (int32_t)m;
            }
        }
    }
    free(best);
}
