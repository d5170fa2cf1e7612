// k_fit.cu -- refinement of the candidates (ht_fit_tracks in include/ht.h):
// a least-squares circle fit of each candidate to its assigned hits.
// Section 5 has costlier computations confirm the candidates and Section 6
// names a Kalman filter for it (run on the CPU there, with a GPU version
// suggested); without material or process noise a Kalman filter over
// the hits computes the weighted least-squares estimate, fitted here
// directly.
//
// Reading: p = (rho, d0, phi0) starts at the candidate's cell centre; the
// residual of hit (x, y) is F / 2 with F = rho d0^2 + 2 (1 + rho s) d0 +
// rho r^2 + 2 s (the signed distance to the circle to first order); `iters`
// Gauss-Newton steps solve (J^T J) dp = -J^T r by Cholesky (a non-positive
// pivot stops with status -1); chi2 and sigma^2 (J^T J)^-1 at the final p.
// Optional hit selection: only hits within `road` of the cell-centre circle
// are fitted; then the hits within `cut` sigma of the fitted circle are
// fitted again with `iters2` steps (the outlier rejection of a track fit).
//
// Design (GB300): candidates' hit lists by counting sort (count, scan,
// scatter); one warp per candidate, lanes over its hits, the normal
// equations summed with warp shuffles in float64 (a few dozen flops per
// hit: the float64 rate is no bottleneck) and solved by lane 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

__device__ __forceinline__ int event_of(const int *off, int n_ev, int h)
{
    int lo = 0, hi = n_ev;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= h) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Count (list null) or scatter the hits of every candidate: candidate m of
// event e is slot e * cap + m.
__global__ void k_fit_lists(const int *__restrict__ off, int n_ev,
                            const int *__restrict__ assign, const int *__restrict__ counts,
                            int cap, int *__restrict__ cnt, int *__restrict__ cur,
                            int *__restrict__ list)
{
    const int total = off[n_ev];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < total; h += gridDim.x * blockDim.x) {
        const int m = assign[h];
        if (m < 0) continue;
        const int e = event_of(off, n_ev, h);
        if (m >= min(counts[e], cap)) continue;
        const size_t slot = (size_t)e * cap + m;
        if (list) list[atomicAdd(&cur[slot], 1)] = h;
        else atomicAdd(&cnt[slot], 1);
    }
}

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double half_f(double rho, double d0, double s, double r2)
{
    return 0.5 * (rho * d0 * d0 + 2.0 * (1.0 + rho * s) * d0 + rho * r2 + 2.0 * s);
}

// A hit selection: the hits whose residual at q is at most w in magnitude
// (w = infinity: every hit).
struct Sel {
    double q[3];
    double w;
};

// Normal equations of the selected hits of list[b .. b + nh) at p: A (6
// unique entries), J^T r, sum r^2 and their number; every lane gets them.
__device__ __forceinline__ void normal_eq(const float *__restrict__ x,
                                          const float *__restrict__ y,
                                          const int *__restrict__ list, int b, int nh,
                                          const double p[3], const Sel &S, int lane,
                                          double A[6], double g[3], double &rr, int &nk)
{
    double sn, cs, qs, qc;
    sincos(p[2], &sn, &cs);
    sincos(S.q[2], &qs, &qc);
    double a[6] = {0, 0, 0, 0, 0, 0}, gg[3] = {0, 0, 0}, s2 = 0;
    int k = 0;
    for (int t = lane; t < nh; t += 32) {
        const int h = list[b + t];
        const double xh = (double)x[h], yh = (double)y[h];
        if (S.w < 1e300) {
            const double sq = xh * qs - yh * qc;
            if (!(fabs(half_f(S.q[0], S.q[1], sq, xh * xh + yh * yh)) <= S.w)) continue;
        }
        ++k;
        const double s = xh * sn - yh * cs, c = xh * cs + yh * sn;
        const double r2 = xh * xh + yh * yh;
        const double rho = p[0], d0 = p[1];
        const double r = half_f(rho, d0, s, r2);
        const double j0 = 0.5 * (d0 * d0 + 2.0 * s * d0 + r2);
        const double j1 = rho * d0 + 1.0 + rho * s;
        const double j2 = (1.0 + rho * d0) * c;
        a[0] += j0 * j0; a[1] += j0 * j1; a[2] += j0 * j2;
        a[3] += j1 * j1; a[4] += j1 * j2; a[5] += j2 * j2;
        gg[0] += j0 * r; gg[1] += j1 * r; gg[2] += j2 * r;
        s2 += r * r;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) A[i] = wsum(a[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] = wsum(gg[i]);
    rr = wsum(s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    nk = k;
}

// Cholesky of the symmetric 3 x 3 matrix {A0 A1 A2; . A3 A4; . . A5}:
// L = {l0; l1 l2; l3 l4 l5}; false if a pivot is not positive.
__device__ __forceinline__ bool chol3(const double A[6], double L[6])
{
    if (!(A[0] > 0.0)) return false;
    L[0] = sqrt(A[0]);
    L[1] = A[1] / L[0];
    const double d1 = A[3] - L[1] * L[1];
    if (!(d1 > 0.0)) return false;
    L[2] = sqrt(d1);
    L[3] = A[2] / L[0];
    L[4] = (A[4] - L[3] * L[1]) / L[2];
    const double d2 = A[5] - L[3] * L[3] - L[4] * L[4];
    if (!(d2 > 0.0)) return false;
    L[5] = sqrt(d2);
    return true;
}

struct FitArgs {
    double delta, half_nd, pi_over_np, sigma, road, cut;
    const double *rho64;
    int n_phi0, min_hits, iters, iters2;
};

// Gauss-Newton steps on the hits that S selects; false (and p kept) when
// the normal matrix is not positive definite.
__device__ __forceinline__ bool gauss_newton(const float *__restrict__ x,
                                             const float *__restrict__ y,
                                             const int *__restrict__ list, int b, int nh,
                                             double p[3], const Sel &S, int iters, int lane)
{
    double A[6], g[3], rr, L[6];
    int nk;
    for (int it = 0; it < iters; ++it) {
        normal_eq(x, y, list, b, nh, p, S, lane, A, g, rr, nk);
        if (!chol3(A, L)) return false;               // same sums on every lane
        // forward then backward substitution: L z = g, L^T dp = z
        const double z0 = g[0] / L[0];
        const double z1 = (g[1] - L[1] * z0) / L[2];
        const double z2 = (g[2] - L[3] * z0 - L[4] * z1) / L[5];
        const double d2 = z2 / L[5];
        const double d1 = (z1 - L[4] * d2) / L[2];
        const double d0 = (z0 - L[1] * d1 - L[3] * d2) / L[0];
        p[0] -= d0;
        p[1] -= d1;
        p[2] -= d2;
    }
    return true;
}

// One warp per candidate (grid.y = event, warps stride over its candidates).
__global__ void __launch_bounds__(256)
k_fit_tracks(FitArgs F, const float *__restrict__ x, const float *__restrict__ y,
             const ht_peak *__restrict__ peaks, const int *__restrict__ counts, int cap,
             const int *__restrict__ cnt, const int *__restrict__ start,
             const int *__restrict__ list, ht_track *__restrict__ out)
{
    const int e = blockIdx.y, lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int nc = min(counts[e], cap);
    for (int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); m < nc; m += nwarps) {
        const size_t slot = (size_t)e * cap + m;
        const int nh = cnt[slot], b = start[slot];
        ht_track T;
        T.n_hits = nh;
        T.reserved = 0;
        const ht_peak pk = peaks[slot];
        double p[3] = {F.rho64[pk.i_rho], ((double)pk.j_d0 - F.half_nd) * F.delta,
                       (double)(2 * pk.k_phi0 + 1 - F.n_phi0) * F.pi_over_np};
        if (nh < F.min_hits) {
            T.rho = p[0]; T.d0 = p[1]; T.phi0 = p[2];
            T.sig_rho = T.sig_d0 = T.sig_phi0 = nan("");
            T.chi2 = nanf("");
            T.status = 0;
            if (lane == 0) out[slot] = T;
            continue;
        }
        int status = 1;
        double A[6], g[3], rr, L[6];
        int nk;
        Sel S;
        S.q[0] = p[0]; S.q[1] = p[1]; S.q[2] = p[2];
        S.w = F.road > 0.0 ? F.road : 1e308;
        // the road: hits near the cell-centre circle
        normal_eq(x, y, list, b, nh, p, S, lane, A, g, rr, nk);
        bool few = nk < F.min_hits;
        if (!few) {
            if (!gauss_newton(x, y, list, b, nh, p, S, F.iters, lane)) status = -1;
            if (status == 1 && F.cut > 0.0) {
                // the outlier cut: hits near the fitted circle, fitted again
                S.q[0] = p[0]; S.q[1] = p[1]; S.q[2] = p[2];
                S.w = F.cut * F.sigma;
                normal_eq(x, y, list, b, nh, p, S, lane, A, g, rr, nk);
                few = nk < F.min_hits;
                if (!few && !gauss_newton(x, y, list, b, nh, p, S, F.iters2, lane)) status = -1;
            }
        }
        T.rho = p[0]; T.d0 = p[1]; T.phi0 = p[2];
        if (few) {
            T.n_hits = nk;
            T.sig_rho = T.sig_d0 = T.sig_phi0 = nan("");
            T.chi2 = nanf("");
            T.status = 0;
            if (lane == 0) out[slot] = T;
            continue;
        }
        normal_eq(x, y, list, b, nh, p, S, lane, A, g, rr, nk);
        T.n_hits = nk;
        T.chi2 = (float)(rr / (F.sigma * F.sigma));
        if (chol3(A, L)) {
            // diagonal of (L L^T)^-1 = columns of L^-1 squared and summed
            const double i0 = 1.0 / L[0], i2 = 1.0 / L[2], i5 = 1.0 / L[5];
            const double i1 = -L[1] * i0 * i2;                       // (L^-1)[1][0]
            const double i4 = -L[4] * i2 * i5;                       // (L^-1)[2][1]
            const double i3 = -(L[3] * i0 + L[4] * i1) * i5;         // (L^-1)[2][0]
            const double s2 = F.sigma * F.sigma;
            T.sig_rho = sqrt(s2 * (i0 * i0 + i1 * i1 + i3 * i3));
            T.sig_d0 = sqrt(s2 * (i2 * i2 + i4 * i4));
            T.sig_phi0 = sqrt(s2 * (i5 * i5));
        } else {
            T.sig_rho = T.sig_d0 = T.sig_phi0 = nan("");
            status = -1;
        }
        T.status = status;
        if (lane == 0) out[slot] = T;
    }
}

}  // namespace
}  // namespace ht

extern "C" {

size_t ht_fit_workspace_size(int32_t n_events, int32_t cap, int32_t n_hits)
{
    const size_t ns = (size_t)(n_events > 0 ? n_events : 1) * (size_t)(cap > 0 ? cap : 1);
    return 3 * ht::align256((ns + 1) * 4) + ht::align256((size_t)(n_hits > 0 ? n_hits : 1) * 4) +
           ht::scan_tmp_bytes((int)ns);
}

ht_status ht_fit_tracks(const ht_geometry *g, const float *x, const float *y, const int32_t *d_off,
                        int32_t n_events, int32_t n_hits, const int32_t *assign,
                        const ht_peak *peaks, const int32_t *d_count, int32_t cap,
                        int32_t min_hits, int32_t iters, double sigma, double road, double cut,
                        int32_t iters2, ht_track *out, void *workspace, size_t workspace_bytes,
                        ht_stream stream)
{
    if (!g || !d_off || !d_count || !out || !workspace || n_events < 1 || n_hits < 0 || cap < 1 ||
        min_hits < 3 || iters < 0 || iters > 64 || iters2 < 0 || iters2 > 64 ||
        !(sigma > 0.0) || road != road || cut != cut ||
        (n_hits > 0 && (!x || !y || !assign)) || !peaks)
        return ht::set_error(HT_ERR_ARG, "ht_fit_tracks: bad argument");
    if ((int64_t)n_events * cap > 0x7fffffffLL)
        return ht::set_error(HT_ERR_CAPACITY, "ht_fit_tracks: n_events * cap above 2^31");
    if (workspace_bytes < ht_fit_workspace_size(n_events, cap, n_hits) ||
        reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return ht::set_error(HT_ERR_ARG, "ht_fit_tracks: workspace size or alignment");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int ns = n_events * cap;
    char *w = reinterpret_cast<char *>(workspace);
    int *cnt = reinterpret_cast<int *>(w);
    int *start = reinterpret_cast<int *>(w + ht::align256(((size_t)ns + 1) * 4));
    int *cur = reinterpret_cast<int *>(w + 2 * ht::align256(((size_t)ns + 1) * 4));
    int *list = reinterpret_cast<int *>(w + 3 * ht::align256(((size_t)ns + 1) * 4));
    void *tmp = w + 3 * ht::align256(((size_t)ns + 1) * 4) +
                ht::align256((size_t)(n_hits > 0 ? n_hits : 1) * 4);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)ns * 4, st);
    const int gb = n_hits > 0 ? min((n_hits + 255) / 256, 4096) : 1;
    if (e == cudaSuccess) {
        ht::k_fit_lists<<<gb, 256, 0, st>>>(d_off, n_events, assign, d_count, cap, cnt, nullptr,
                                            nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = ht::scan_exclusive(cnt, start, cur, ns, nullptr, nullptr, tmp, st);
    if (e == cudaSuccess) {
        ht::k_fit_lists<<<gb, 256, 0, st>>>(d_off, n_events, assign, d_count, cap, nullptr, cur,
                                            list);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ht::FitArgs F;
        F.delta = g->G.delta;
        F.half_nd = 0.5 * (double)g->G.n_d0;
        F.pi_over_np = ht::kPi / (double)g->G.n_phi0;
        F.sigma = sigma;
        F.road = road;
        F.cut = cut;
        F.iters2 = iters2;
        F.rho64 = g->G.rho64;
        F.n_phi0 = g->G.n_phi0;
        F.min_hits = min_hits;
        F.iters = iters;
        ht::k_fit_tracks<<<dim3(64, n_events), 256, 0, st>>>(F, x, y, peaks, d_count, cap, cnt,
                                                              start, list, out);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HT_OK : ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
