// k_swept.cu -- swept-interval phi0 vote (ht_vote_swept in include/ht.h): the
// Hough vote of Section 5 of arXiv:1309.6275 with every phi0 column voting
// the d0 range the hit's roots sweep across the column instead of the root
// at its centre.
//
// Reading (the paper samples phi0 at bin centres and notes that the
// transform tolerates data a discretisation cannot represent exactly): the
// roots are sampled at the column's lower edge e_k = (2k - N) pi / N, its
// centre phi0_k and its upper edge e_{(k+1) mod N}; at each sample they exist
// when c > 0 and D >= 0 and are labelled by branch, + = (-b + sqrt D) / rho
// and - = (-b - sqrt D) / rho (rho = 0: only +; D = 0: both equal), each with
// a code: floor(u) inside the axis, -1 below, n_d0 above.  Per branch, two
// consecutive samples that both have the root give every bin between their
// codes (clamped to the axis); a sample whose neighbours lack the root gives
// its own bin.  A cell gets one vote per hit when its bin is in the union.
//
// Kernel: one CTA per tile of 32 rho rows (lane = row) x KT columns with
// 32-bit counters in shared memory.  Phase 1 (thread = hit) keeps the
// (hit, column) pairs whose largest c over the column can reach the hit's
// angular window (section of ht_internal.cuh) and stores the three samples'
// s and c.  Phase 2 (warp = pair, lane = row) labels the six roots by guarded
// float32 arithmetic (the point vote's error bounds, per sample) and votes
// the union of at most four bin ranges; an undecided sample defers the whole
// (hit, row, column) to a float64 redo that repeats the definition's
// operations one rounding at a time.
#include "tiles.cuh"

namespace ht {
namespace {

constexpr int kSwMetaUnsure = 16, kSwMetaCol = 15;

struct SwList {
    float4 *s;   // s at lower edge, centre, upper edge; r2
    float4 *c;   // c at the same samples; R1
    int *meta;   // hit << 5 | unsure << 4 | column in tile
};

constexpr size_t kSwItemBytes = 36;

__device__ __forceinline__ SwList carve_sw(unsigned char *p, int cap)
{
    SwList w;
    w.s = reinterpret_cast<float4 *>(p);
    w.c = w.s + cap;
    w.meta = reinterpret_cast<int *>(w.c + cap);
    return w;
}

// Side-aware bin code of a root: floor(u) inside the axis, -1 certainly
// below, nd certainly above, -2 undecided.  For u in (-1, 0) the fraction
// u + 1 is rounded, so a root within e below the axis is undecided.
__device__ __forceinline__ int side_code(float u, float e, int nd)
{
    const float f = floorf(u);
    const float fr = u - f;
    if (u + e < 0.0f) return -1;
    if (u - e >= (float)nd) return nd;
    return (f >= 0.0f && fminf(fr, 1.0f - fr) > e) ? (int)f : -2;
}

// Root codes of one sample: ok[br] (branch + = 0, - = 1) and code[br].
struct SwSample {
    int ok[2], code[2];
};

// Guarded float32 sample; false when undecided (redo).  c_sure: c > 0 is
// proven (the caller skipped the sample if c <= 0 is proven).
__device__ __forceinline__ bool sample32(const DevGeom &G, float rho, float invrho,
                                         float invrho_es, bool has_b, float s, float c,
                                         float r2, float R1, float rt, SwSample &o)
{
    const Item it = make_item(G, s, c, r2, R1, rt);
    const float b = fmaf(rho, s, 1.0f);
    const float pc = rho * c;
    const float D = fmaf(-pc, pc, 1.0f);
    o.ok[0] = o.ok[1] = 0;
    if (D < -it.eD) return true;           // certainly no real root
    if (D <= it.eD) return false;          // sign of D not proven
    const float rs = rsqrt_approx(D);
    const float sq = D * rs;
    const float q = -(b + copysignf(sq, b));
    const float C = fmaf(rho, r2, s + s);
    const float iq = rcp_approx(q);
    const int nd = G.n_d0;
    const float uA = fmaf(C * iq, G.inv_delta_f, G.off_f);
    const float eA = fmaf(fabsf(iq), fmaf(it.E2, rs, it.E1), G.e3);
    const int cA = side_code(uA, eA, nd);
    if (cA == -2) return false;
    if (!has_b) {                          // rho == 0: the one root -s
        o.ok[0] = 1;
        o.code[0] = cA;
        return true;
    }
    const float uB = fmaf(q * invrho, G.inv_delta_f, G.off_f);
    const float eB = fmaf(invrho_es, fmaf(it.Qb, rs, it.Qa), G.e3);
    const int cB = side_code(uB, eB, nd);
    if (cB == -2) return false;
    // b >= 0: C / q is the + root; b < 0: q / rho is.  (Near b = 0 either
    // labelling computes the same two branches: no cancellation there.)
    o.ok[0] = o.ok[1] = 1;
    o.code[0] = b >= 0.0f ? cA : cB;
    o.code[1] = b >= 0.0f ? cB : cA;
    return true;
}

__device__ __forceinline__ int u_code64(const DevGeom &G, double root)
{
    const double u = __dadd_rn(__ddiv_rn(root, G.delta), G.off);
    if (u < 0.0) return -1;
    if (u >= (double)G.n_d0) return G.n_d0;
    return (int)floor(u);
}

// The definition's float64 sample, one correctly rounded operation at a time.
__device__ __noinline__ SwSample sample64(const DevGeom &G, float xf, float yf, double sn,
                                          double cs, double rho)
{
    SwSample o;
    o.ok[0] = o.ok[1] = 0;
    o.code[0] = o.code[1] = 0;
    const double x = (double)xf, y = (double)yf;
    const double s = __dsub_rn(__dmul_rn(x, sn), __dmul_rn(y, cs));
    const double c = __dadd_rn(__dmul_rn(x, cs), __dmul_rn(y, sn));
    if (!(c > 0.0)) return o;
    const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
    const double b = __dadd_rn(1.0, __dmul_rn(rho, s));
    const double pc = __dmul_rn(rho, c);
    const double D = __dsub_rn(1.0, __dmul_rn(pc, pc));
    if (D < 0.0) return o;
    const double sq = __dsqrt_rn(D);
    const double q = -__dadd_rn(b, b >= 0.0 ? sq : -sq);
    const double C = __dadd_rn(__dmul_rn(rho, r2), __dmul_rn(2.0, s));
    if (rho == 0.0) {
        o.ok[0] = 1;
        o.code[0] = u_code64(G, __ddiv_rn(C, q));
        return o;
    }
    if (D == 0.0) {
        o.ok[0] = o.ok[1] = 1;
        o.code[0] = o.code[1] = u_code64(G, __ddiv_rn(q, rho));
        return o;
    }
    const int cA = u_code64(G, __ddiv_rn(C, q));
    const int cB = u_code64(G, __ddiv_rn(q, rho));
    o.ok[0] = o.ok[1] = 1;
    o.code[0] = b >= 0.0 ? cA : cB;
    o.code[1] = b >= 0.0 ? cB : cA;
    return o;
}

// Vote the union of the swept bin ranges of three samples into one column
// of the tile (col points at the lane's row of column kl, stride 32).
__device__ __forceinline__ void vote_ranges(const SwSample t[3], int nd, uint32_t *col)
{
    int lo[4], hi[4], n = 0;
#pragma unroll
    for (int br = 0; br < 2; ++br) {
        const bool v0 = t[0].ok[br], v1 = t[1].ok[br], v2 = t[2].ok[br];
        const int c0 = t[0].code[br], c1 = t[1].code[br], c2 = t[2].code[br];
        if (v0 && v1 && v2) {
            lo[n] = min(c0, min(c1, c2));
            hi[n++] = max(c0, max(c1, c2));
        } else if (v0 && v1) {
            lo[n] = min(c0, c1);
            hi[n++] = max(c0, c1);
            // sample 2 lacks the root: nothing more on this branch
        } else if (v1 && v2) {
            lo[n] = min(c1, c2);
            hi[n++] = max(c1, c2);
        } else {
            // no consecutive pair: each sample with the root alone
            if (v0) { lo[n] = c0; hi[n++] = c0; }
            if (v1) { lo[n] = c1; hi[n++] = c1; }
            if (v2) { lo[n] = c2; hi[n++] = c2; }
        }
    }
    for (int a = 0; a < n; ++a) {
        const int l = max(lo[a], 0), h = min(hi[a], nd - 1);
        for (int j = l; j <= h; ++j) {
            bool seen = false;
            for (int p = 0; p < a; ++p) seen |= (j >= lo[p] && j <= hi[p]);
            if (!seen) atomicAdd(col + j * 32, 1u);
        }
    }
}

template <int KT, typename OutT>
__global__ void __launch_bounds__(kThreads, 2)
k_vote_swept(DevGeom G, const float *__restrict__ x, const float *__restrict__ y, int n,
             OutT *__restrict__ acc, unsigned long long *__restrict__ stats)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ND = G.n_d0, NP = G.n_phi0;
    constexpr int QCAP = kThreads * KT;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);   // [KT][ND][32]
    unsigned char *p = reinterpret_cast<unsigned char *>(cnt + KT * ND * 32);
    const SwList W = carve_sw(p, QCAP);
    const RedoQueue R = carve_redo(p + (size_t)QCAP * kSwItemBytes);
    __shared__ int qn, rn;
    __shared__ unsigned long long s_votes;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT> T;
    T.init(G, lane, blockIdx.x, blockIdx.y);
    // edges of the tile's columns: lower edge of k0 + kl for kl = 0 .. KT
    float es[KT + 1], ec[KT + 1];
#pragma unroll
    for (int kl = 0; kl <= KT; ++kl) {
        const int k = (T.k0 + kl) % NP;
        es[kl] = G.esn32[k];
        ec[kl] = G.ecs32[k];
    }
    // largest rise of c between samples half a column apart: r (1 - cos(pi / 2N))
    const float rise = 1.0f - cospif(0.5f / (float)NP) + 1e-6f;
    for (int t = threadIdx.x; t < KT * ND * 8; t += kThreads)
        reinterpret_cast<uint4 *>(cnt)[t] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        qn = 0;
        rn = 0;
        s_votes = 0ull;
    }
    __syncthreads();

    for (int base = 0; base < n; base += kThreads) {
        // ---- phase 1: thread = hit
        const int h = base + threadIdx.x;
        if (h < n) {
            const float xh = x[h], yh = y[h];
            const float r2 = fmaf(xh, xh, yh * yh);
            const float R1 = fabsf(xh) + fabsf(yh);
            const float r = sqrtf(r2);
            const float Ec = (kSafe * 3.0f * kEps) * R1;
            const float cmin = hit_cos_window(G, r2);
            // with r |rho| >= 1 a D < 0 gap inside a column can join roots on
            // both sides of the axis: no window test then
            const bool window = r * T.rt < 0.999f;
#pragma unroll
            for (int kl = 0; kl < KT; ++kl) {
                const float s0 = fmaf(xh, es[kl], -(yh * ec[kl]));
                const float c0 = fmaf(xh, ec[kl], yh * es[kl]);
                const float s1 = fmaf(xh, T.sk[kl], -(yh * T.ck[kl]));
                const float c1 = fmaf(xh, T.ck[kl], yh * T.sk[kl]);
                const float s2 = fmaf(xh, es[kl + 1], -(yh * ec[kl + 1]));
                const float c2 = fmaf(xh, ec[kl + 1], yh * es[kl + 1]);
                const float cmax = fmaxf(c0, fmaxf(c1, c2));
                if (cmax < -Ec) continue;                       // no sample has a root
                if (window && cmax + r * rise + 1e-3f * r < cmin) continue;
                const bool unsure = fabsf(c0) <= Ec || fabsf(c1) <= Ec || fabsf(c2) <= Ec;
                const int pos = atomicAdd(&qn, 1);
                W.s[pos] = make_float4(s0, s1, s2, r2);
                W.c[pos] = make_float4(c0, c1, c2, R1);
                W.meta[pos] = (h << 5) | (unsure ? kSwMetaUnsure : 0) | kl;
            }
        }
        __syncthreads();
        // ---- phase 2: warp = item, lane = row
        const int nq = qn;
        if (T.row_ok) {
            for (int t = warp; t < nq; t += nwarps) {
                const int m = W.meta[t];
                const int kl = m & kSwMetaCol;
                uint32_t *col = cnt + kl * ND * 32 + lane;
                bool redo = (m & kSwMetaUnsure) != 0;
                SwSample sm[3];
                if (!redo) {
                    const float4 S = W.s[t], Cc = W.c[t];
                    const float ss[3] = {S.x, S.y, S.z}, cc[3] = {Cc.x, Cc.y, Cc.z};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (cc[a] < 0.0f) {                  // proven c <= 0 (not unsure)
                            sm[a].ok[0] = sm[a].ok[1] = 0;
                            continue;
                        }
                        redo |= !sample32(G, T.rho, T.invrho, T.invrho_es, T.has_b, ss[a],
                                          cc[a], S.w, Cc.w, T.rt, sm[a]);
                    }
                }
                if (redo) {
                    if (push_redo(R, &rn, m >> 5, lane, kl)) continue;
                    const int hh = m >> 5, k = T.k0 + kl;
                    const double rho = G.rho64[T.irow];
                    sm[0] = sample64(G, x[hh], y[hh], G.esn64[k], G.ecs64[k], rho);
                    sm[1] = sample64(G, x[hh], y[hh], G.sn64[k], G.cs64[k], rho);
                    sm[2] = sample64(G, x[hh], y[hh], G.esn64[(k + 1) % NP],
                                     G.ecs64[(k + 1) % NP], rho);
                }
                vote_ranges(sm, ND, col);
            }
        }
        __syncthreads();
        const int nr = min(rn, kRedoCap);
        if (nr >= kRedoCap / 2 || base + kThreads >= n) {
            for (int t = threadIdx.x; t < nr; t += kThreads) {
                const int hh = R.hit[t], rc = R.rc[t];
                const int il = rc >> 4, kl = rc & 15, k = T.k0 + kl;
                const double rho = G.rho64[T.i0 + il];
                SwSample sm[3];
                sm[0] = sample64(G, x[hh], y[hh], G.esn64[k], G.ecs64[k], rho);
                sm[1] = sample64(G, x[hh], y[hh], G.sn64[k], G.cs64[k], rho);
                sm[2] = sample64(G, x[hh], y[hh], G.esn64[(k + 1) % NP], G.ecs64[(k + 1) % NP],
                                 rho);
                vote_ranges(sm, ND, cnt + kl * ND * 32 + il);
            }
            __syncthreads();
            if (threadIdx.x == 0) rn = 0;
        }
        if (threadIdx.x == 0) qn = 0;
        __syncthreads();
    }

    // write-back: thread = (row, d0 bin), the KT counts of a row as one vector
    unsigned long long my_votes = 0;
    for (int t = threadIdx.x; t < 32 * ND; t += kThreads) {
        const int il = t & 31, j = t >> 5;
        const int i = T.i0 + il;
        if (i >= G.n_rho) continue;
        __align__(16) OutT e[KT];
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            const uint32_t v = cnt[(kl * ND + j) * 32 + il];
            my_votes += v;
            e[kl] = saturate<OutT>(v);
        }
        OutT *dst = acc + ((size_t)i * ND + j) * NP + T.k0;
        if constexpr (KT * sizeof(OutT) == 8) {
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(e);
        } else if constexpr (KT * sizeof(OutT) == 4) {
            *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(e);
        } else {
#pragma unroll
            for (int kl = 0; kl < KT; ++kl) dst[kl] = e[kl];
        }
    }
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_votes += __shfl_xor_sync(0xffffffffu, my_votes, o);
        if (lane == 0) atomicAdd(&s_votes, my_votes);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&stats[0], s_votes);
    }
}

template <int KT>
size_t swept_smem(const DevGeom &G)
{
    return (size_t)KT * 32 * G.n_d0 * 4 + (size_t)kThreads * KT * kSwItemBytes + kRedoBytes;
}

template <int KT, typename OutT>
cudaError_t launch_swept_kt(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                            unsigned long long *stats, cudaStream_t st)
{
    dim3 grid(G.n_phi0 / KT, (G.n_rho + 31) / 32);
    k_vote_swept<KT, OutT><<<grid, kThreads, swept_smem<KT>(G), st>>>(
        G, x, y, n, reinterpret_cast<OutT *>(acc), stats);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_vote_swept(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                              unsigned long long *stats, cudaStream_t st)
{
    const bool two = swept_smem<2>(G) <= kSmemBudget2;
    if (G.count_bits == 16)
        return two ? launch_swept_kt<2, uint16_t>(G, x, y, n, acc, stats, st)
                   : launch_swept_kt<1, uint16_t>(G, x, y, n, acc, stats, st);
    return two ? launch_swept_kt<2, int32_t>(G, x, y, n, acc, stats, st)
               : launch_swept_kt<1, int32_t>(G, x, y, n, acc, stats, st);
}

size_t swept_smem_need(const DevGeom &G) { return swept_smem<1>(G); }

cudaError_t prepare_swept_kernels(int max_smem)
{
    const void *fns[] = {(const void *)k_vote_swept<2, uint16_t>,
                         (const void *)k_vote_swept<1, uint16_t>,
                         (const void *)k_vote_swept<2, int32_t>,
                         (const void *)k_vote_swept<1, int32_t>};
    return allow_smem(fns, 4, max_smem);
}

}  // namespace ht
