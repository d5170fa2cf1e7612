// ht_api.cu -- the C ABI of libht (declared in include/ht.h).
//
// Argument checking, the geometry handle (host-computed float64 tables and
// their float32 roundings, uploaded once), workspace carving and the
// synchronous host-buffer path.  All compute happens in the kernels of
// k_tiles.cu, k_peaks.cu and k_votez.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "ht_internal.cuh"

namespace ht {
cudaError_t prepare_tile_kernels(int max_smem);
size_t tile_smem_need(const DevGeom &G);
cudaError_t prepare_z_kernels(int max_smem);
cudaError_t prepare_mlp_kernels();
cudaError_t prepare_masked_vote_kernels(int max_smem);
cudaError_t prepare_swept_kernels(int max_smem);
size_t swept_smem_need(const DevGeom &G);
cudaError_t prepare_peaks_kernels();
size_t z_big_smem(const DevGeom &G);
cudaError_t prepare_layer_vote_kernels(int max_smem);
cudaError_t launch_vote_layers(const DevGeom &G, const float *x, const float *y,
                               const uint8_t *layer, int n, void *acc,
                               unsigned long long *stats, cudaStream_t st);
}  // namespace ht

namespace {

thread_local char g_err[512] = "";

ht_status fail(ht_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

ht_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(HT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t cell_count(const ht_geometry *g)
{
    return (size_t)g->desc.n_rho * g->desc.n_d0 * g->desc.n_phi0;
}

cudaStream_t S(ht_stream s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int32_t kMaxHits = 1 << 25;   // hit index must fit 25 bits in the work list

}  // namespace

namespace ht {
ht_status set_error(ht_status s, const char *msg)
{
    return fail(s, "%s", msg);
}
}  // namespace ht

extern "C" {

const char *ht_last_error(void) { return g_err; }

ht_status ht_geometry_create(const ht_geometry_desc *d, ht_geometry **out)
{
    if (!d || !out) return fail(HT_ERR_ARG, "ht_geometry_create: null argument");
    *out = nullptr;
    if (d->n_rho < 1 || d->n_rho > 65535 || d->n_d0 < 2 || d->n_d0 > 512 || d->n_phi0 < 8 ||
        d->n_phi0 % 8 != 0 || d->n_phi0 > (1 << 20) || d->n_z0 < 1 || d->n_z0 > 1024 ||
        d->n_cot < 1 || d->n_cot > 1024 || (int64_t)d->n_z0 * d->n_cot > 32768 ||
        d->threshold < 1 || (d->count_bits != 16 && d->count_bits != 32))
        return fail(HT_ERR_ARG, "ht_geometry_create: unsupported axis sizes "
                                "(n_rho %d, n_d0 %d, n_phi0 %d, n_z0 %d, n_cot %d, T %d, bits %d)",
                    d->n_rho, d->n_d0, d->n_phi0, d->n_z0, d->n_cot, d->threshold,
                    d->count_bits);
    if (!(d->rho_max > 0) || !(d->d0_half > 0) || !(d->z0_max > 0) || !(d->cot_max > 0))
        return fail(HT_ERR_ARG, "ht_geometry_create: ranges must be positive");
    if ((double)d->n_rho * d->n_d0 * d->n_phi0 > 2147483647.0)
        return fail(HT_ERR_ARG, "ht_geometry_create: more than 2^31-1 cells");

    ht_geometry *g = new (std::nothrow) ht_geometry();
    if (!g) return fail(HT_ERR_ARG, "ht_geometry_create: out of host memory");
    g->desc = *d;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaGetDevice"); }

    const int NP = d->n_phi0, NR = d->n_rho, ND = d->n_d0;
    // float64 tables, same expressions as the definition
    double *phi = new double[NP], *sn = new double[NP], *cs = new double[NP], *rho = new double[NR];
    for (int k = 0; k < NP; ++k) {
        phi[k] = (double)(2 * k + 1 - NP) * (ht::kPi / (double)NP);
        sn[k] = sin(phi[k]);
        cs[k] = cos(phi[k]);
    }
    for (int i = 0; i < NR; ++i) rho[i] = (double)(2 * i + 1 - NR) * (d->rho_max / (double)NR);

    // column lower edges e_k = (2k - N) pi / N (the swept-interval vote)
    double *esn = new double[NP], *ecs = new double[NP];
    for (int k = 0; k < NP; ++k) {
        const double ek = (double)(2 * k - NP) * (ht::kPi / (double)NP);
        esn[k] = sin(ek);
        ecs[k] = cos(ek);
    }

    // one device block: float64 sn, cs, rho, edge sn, edge cs | float32 sn,
    // cs, phi, rho, 1/rho, the float32 remainders sn - (float)sn,
    // cs - (float)cs, rho - (float)rho, and float32 edge sn, cs
    const size_t b64 = sizeof(double) * (4 * (size_t)NP + NR);
    const size_t b32 = sizeof(float) * (7 * (size_t)NP + 3 * (size_t)NR);
    const size_t bytes = ht::align256(b64) + ht::align256(b32);
    char *h = new char[bytes];
    memset(h, 0, bytes);
    double *h64 = reinterpret_cast<double *>(h);
    float *h32 = reinterpret_cast<float *>(h + ht::align256(b64));
    memcpy(h64, sn, sizeof(double) * NP);
    memcpy(h64 + NP, cs, sizeof(double) * NP);
    memcpy(h64 + 2 * NP, rho, sizeof(double) * NR);
    memcpy(h64 + 2 * NP + NR, esn, sizeof(double) * NP);
    memcpy(h64 + 3 * NP + NR, ecs, sizeof(double) * NP);
    for (int k = 0; k < NP; ++k) {
        h32[k] = (float)sn[k];
        h32[NP + k] = (float)cs[k];
        h32[2 * NP + k] = (float)phi[k];
    }
    for (int i = 0; i < NR; ++i) {
        h32[3 * NP + i] = (float)rho[i];
        h32[3 * NP + NR + i] = rho[i] != 0.0 ? (float)(1.0 / rho[i]) : 0.0f;
    }
    float *hlo = h32 + 3 * NP + 2 * NR;
    for (int k = 0; k < NP; ++k) {
        hlo[k] = (float)(sn[k] - (double)(float)sn[k]);
        hlo[NP + k] = (float)(cs[k] - (double)(float)cs[k]);
    }
    for (int i = 0; i < NR; ++i) hlo[2 * NP + i] = (float)(rho[i] - (double)(float)rho[i]);
    float *hedge = hlo + 2 * NP + NR;
    for (int k = 0; k < NP; ++k) {
        hedge[k] = (float)esn[k];
        hedge[NP + k] = (float)ecs[k];
    }
    e = cudaMalloc(&g->d_tables, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tables, h, bytes, cudaMemcpyHostToDevice);
    delete[] phi; delete[] sn; delete[] cs; delete[] rho; delete[] h;
    delete[] esn; delete[] ecs;
    if (e != cudaSuccess) {
        if (g->d_tables) cudaFree(g->d_tables);
        delete g;
        return cuda_fail(e, "ht_geometry_create: table upload");
    }
    const double *d64 = reinterpret_cast<const double *>(g->d_tables);
    const float *d32 = reinterpret_cast<const float *>(
        reinterpret_cast<const char *>(g->d_tables) + ht::align256(b64));

    ht::DevGeom &G = g->G;
    G.n_rho = NR; G.n_d0 = ND; G.n_phi0 = NP; G.n_z0 = d->n_z0; G.n_cot = d->n_cot;
    G.threshold = d->threshold; G.count_bits = d->count_bits;
    G.delta = 2.0 * d->d0_half / (double)ND;
    G.off = (double)ND * 0.5 + 0.5;
    G.delta_f = (float)G.delta;
    G.inv_delta_f = (float)(1.0 / G.delta);
    G.inv_delta_lo = (float)(1.0 / G.delta - (double)G.inv_delta_f);
    G.off_f = (float)G.off;
    G.d0lo_f = (float)(-G.off * G.delta) - 0.01f;
    G.d0hi_f = (float)(((double)ND - G.off) * G.delta) + 0.01f;
    G.err_scale = (float)(ht::kSafe * (double)ht::kEps / G.delta);
    G.dext_f = (float)((G.off + 0.5) * G.delta * 1.0001 + 0.01);
    G.e3 = G.err_scale * 6.0f * G.dext_f + ht::kSafe * ht::kEps * (float)(ND + 1);
    G.rho_max_f = (float)d->rho_max * 1.0001f;
    G.drho_f = (float)(2.0 * d->rho_max / (double)NR);
    G.dmax_f = (float)(G.off * G.delta) + 0.01f;
    G.sn64 = d64; G.cs64 = d64 + NP; G.rho64 = d64 + 2 * NP;
    G.sn32 = d32; G.cs32 = d32 + NP; G.phi32 = d32 + 2 * NP;
    G.rho32 = d32 + 3 * NP; G.invrho32 = d32 + 3 * NP + NR;
    G.snlo = d32 + 3 * NP + 2 * NR; G.cslo = G.snlo + NP; G.rholo = G.cslo + NP;
    G.esn64 = d64 + 2 * NP + NR; G.ecs64 = G.esn64 + NP;
    G.esn32 = G.rholo + NR; G.ecs32 = G.esn32 + NP;
    G.dz = 2.0 * d->z0_max / (double)d->n_z0;
    G.z0_max = d->z0_max;
    G.cstep = d->cot_max / (double)d->n_cot;
    G.inv_dz_f = (float)(1.0 / G.dz);
    G.z0_max_f = (float)d->z0_max;
    G.cstep_f = (float)G.cstep;

    int max_smem = 0;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
    if (e == cudaSuccess && (ht::tile_smem_need(G) + 1024 > (size_t)max_smem ||
                             ht::z_big_smem(G) + 8192 > (size_t)max_smem)) {
        cudaFree(g->d_tables);
        delete g;
        return fail(HT_ERR_ARG, "ht_geometry_create: tiles need more than %d B shared memory",
                    max_smem);
    }
    if (e == cudaSuccess) e = ht::prepare_tile_kernels(max_smem);
    if (e == cudaSuccess) e = ht::prepare_z_kernels(max_smem);
    if (e == cudaSuccess) e = ht::prepare_masked_vote_kernels(max_smem);
    if (e == cudaSuccess) e = ht::prepare_layer_vote_kernels(max_smem);
    if (e == cudaSuccess) e = ht::prepare_confirm_kernels();
    if (e == cudaSuccess) e = ht::prepare_swept_kernels(max_smem);
    if (e == cudaSuccess) e = ht::prepare_peaks_kernels();
    if (e == cudaSuccess) e = ht::prepare_mlp_kernels();
    if (e != cudaSuccess) {
        cudaFree(g->d_tables);
        delete g;
        return cuda_fail(e, "ht_geometry_create: kernel attributes");
    }
    *out = g;
    return HT_OK;
}

ht_status ht_geometry_destroy(ht_geometry *g)
{
    if (!g) return HT_OK;
    cudaError_t e = cudaFree(g->d_tables);
    delete g;
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_geometry_destroy");
}

size_t ht_accumulator_bytes(const ht_geometry *g)
{
    return g ? cell_count(g) * (g->desc.count_bits / 8) : 0;
}

ht_status ht_vote(const ht_geometry *g, const float *x, const float *y, int32_t n_hits,
                  void *acc, uint64_t *stats, ht_stream stream)
{
    if (!g || !acc) return fail(HT_ERR_ARG, "ht_vote: null geometry or accumulator");
    if (n_hits < 0 || n_hits > kMaxHits)
        return fail(HT_ERR_ARG, "ht_vote: n_hits %d outside [0, %d]", n_hits, kMaxHits);
    if (n_hits > 0 && (!x || !y)) return fail(HT_ERR_ARG, "ht_vote: null hit arrays");
    if (!aligned(acc, 16) || (x && !aligned(x, 16)) || (y && !aligned(y, 16)))
        return fail(HT_ERR_ARG, "ht_vote: pointers must be 16-byte aligned");
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), S(stream));
    if (e == cudaSuccess)
        e = ht::launch_vote(g->G, x, y, n_hits, acc,
                            reinterpret_cast<unsigned long long *>(stats), S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote");
}

ht_status ht_vote_masked(const ht_geometry *g, const float *x, const float *y, int32_t n_hits,
                         const uint64_t *mask, void *acc, uint64_t *stats, ht_stream stream)
{
    if (!g || !acc || !mask) return fail(HT_ERR_ARG, "ht_vote_masked: null geometry, mask or accumulator");
    if (n_hits < 0 || n_hits > kMaxHits)
        return fail(HT_ERR_ARG, "ht_vote_masked: n_hits %d outside [0, %d]", n_hits, kMaxHits);
    if (n_hits > 0 && (!x || !y)) return fail(HT_ERR_ARG, "ht_vote_masked: null hit arrays");
    if (!aligned(acc, 16) || (x && !aligned(x, 16)) || (y && !aligned(y, 16)) ||
        !aligned(mask, 8))
        return fail(HT_ERR_ARG, "ht_vote_masked: pointer alignment");
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), S(stream));
    if (e == cudaSuccess)
        e = ht::launch_vote_masked(g->G, x, y, n_hits, acc,
                                   reinterpret_cast<unsigned long long *>(stats),
                                   reinterpret_cast<const unsigned long long *>(mask), S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote_masked");
}

ht_status ht_vote_hit_masked(const ht_geometry *g, const float *x, const float *y,
                             int32_t n_hits, const uint64_t *hit_masks, void *acc,
                             uint64_t *stats, ht_stream stream)
{
    if (!g || !acc) return fail(HT_ERR_ARG, "ht_vote_hit_masked: null geometry or accumulator");
    if (n_hits < 0 || n_hits > kMaxHits)
        return fail(HT_ERR_ARG, "ht_vote_hit_masked: n_hits %d outside [0, %d]", n_hits,
                    kMaxHits);
    if (n_hits > 0 && (!x || !y || !hit_masks))
        return fail(HT_ERR_ARG, "ht_vote_hit_masked: null hit arrays");
    if (!aligned(acc, 16) || (x && !aligned(x, 16)) || (y && !aligned(y, 16)) ||
        (hit_masks && !aligned(hit_masks, 8)))
        return fail(HT_ERR_ARG, "ht_vote_hit_masked: pointer alignment");
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), S(stream));
    if (e == cudaSuccess)
        e = ht::launch_vote_hitmask(g->G, x, y, n_hits, acc,
                                    reinterpret_cast<unsigned long long *>(stats),
                                    reinterpret_cast<const unsigned long long *>(hit_masks),
                                    S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote_hit_masked");
}

ht_status ht_vote_swept(const ht_geometry *g, const float *x, const float *y, int32_t n_hits,
                        void *acc, uint64_t *stats, ht_stream stream)
{
    if (!g || !acc) return fail(HT_ERR_ARG, "ht_vote_swept: null geometry or accumulator");
    if (n_hits < 0 || n_hits > kMaxHits)
        return fail(HT_ERR_ARG, "ht_vote_swept: n_hits %d outside [0, %d]", n_hits, kMaxHits);
    if (n_hits > 0 && (!x || !y)) return fail(HT_ERR_ARG, "ht_vote_swept: null hit arrays");
    if (!aligned(acc, 16) || (x && !aligned(x, 16)) || (y && !aligned(y, 16)))
        return fail(HT_ERR_ARG, "ht_vote_swept: pointer alignment");
    if (ht::swept_smem_need(g->G) > 200 * 1024)
        return fail(HT_ERR_ARG, "ht_vote_swept: n_d0 %d too large for the swept tile",
                    g->G.n_d0);
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), S(stream));
    if (e == cudaSuccess)
        e = ht::launch_vote_swept(g->G, x, y, n_hits, acc,
                                  reinterpret_cast<unsigned long long *>(stats), S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote_swept");
}

ht_status ht_vote_layers(const ht_geometry *g, const float *x, const float *y,
                         const uint8_t *layer, int32_t n_hits, void *acc, uint64_t *stats,
                         ht_stream stream)
{
    if (!g || !acc) return fail(HT_ERR_ARG, "ht_vote_layers: null geometry or accumulator");
    if (n_hits < 0 || n_hits > kMaxHits)
        return fail(HT_ERR_ARG, "ht_vote_layers: n_hits %d outside [0, %d]", n_hits, kMaxHits);
    if (n_hits > 0 && (!x || !y || !layer))
        return fail(HT_ERR_ARG, "ht_vote_layers: null hit or layer arrays");
    if (g->desc.n_d0 % 2 != 0) return fail(HT_ERR_ARG, "ht_vote_layers: n_d0 must be even");
    if (!aligned(acc, 16) || (x && !aligned(x, 16)) || (y && !aligned(y, 16)))
        return fail(HT_ERR_ARG, "ht_vote_layers: pointers must be 16-byte aligned");
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), S(stream));
    if (e == cudaSuccess)
        e = ht::launch_vote_layers(g->G, x, y, layer, n_hits, acc,
                                   reinterpret_cast<unsigned long long *>(stats), S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote_layers");
}

size_t ht_confirm_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap)
{
    if (!g) return 0;
    return ht::confirm_workspace_bytes_single(g->G, n_hits > 0 ? n_hits : 0, cap > 0 ? cap : 0);
}

ht_status ht_confirm(const ht_geometry *g, const ht_confirm_desc *c, const float *x,
                     const float *y, const uint8_t *layer, int32_t n_hits, const ht_peak *peaks,
                     const int32_t *d_count, int32_t cap, int32_t *score, int32_t *inliers,
                     int32_t *assign, void *workspace, size_t workspace_bytes, ht_stream stream)
{
    if (!g || !c || !d_count || !workspace || (cap > 0 && (!peaks || !score || !inliers)))
        return fail(HT_ERR_ARG, "ht_confirm: null argument");
    if (n_hits < 0 || n_hits > kMaxHits || cap < 0)
        return fail(HT_ERR_ARG, "ht_confirm: n_hits %d or cap %d out of range", n_hits, cap);
    if (n_hits > 0 && (!x || !y || !layer || !assign))
        return fail(HT_ERR_ARG, "ht_confirm: null hit arrays");
    if (c->pool < 0 || c->min_layers < 1 || c->n_layers < 1 || c->n_layers > 16 ||
        !(c->tol > 0.0))
        return fail(HT_ERR_ARG, "ht_confirm: parameters out of range");
    if (workspace_bytes < ht::confirm_workspace_bytes_single(g->G, n_hits, cap) ||
        !aligned(workspace, 256))
        return fail(HT_ERR_ARG, "ht_confirm: workspace too small or misaligned");
    const ht::ConfirmDev P{c->pool, c->min_layers, c->n_layers, c->tol};
    cudaError_t e = ht::launch_confirm(g->G, P, x, y, layer, n_hits, peaks, d_count, cap, score,
                                       inliers, assign, workspace, S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_confirm");
}

// The workspace: the segment counts and offsets and the scan's scratch
// (peaks_workspace_bytes, enough), then the spill buffer that saves the
// second stencil pass when the workspace also holds it.
size_t ht_find_peaks_workspace_size(const ht_geometry *g)
{
    return g ? ht::align256(ht::peaks_workspace_bytes(g->G)) + ht::peak_spill_bytes(g->G) : 0;
}

static void *peak_spill_of(const ht::DevGeom &G, void *workspace, size_t workspace_bytes)
{
    const size_t a = ht::align256(ht::peaks_workspace_bytes(G));
    return workspace_bytes >= a + ht::peak_spill_bytes(G)
               ? reinterpret_cast<char *>(workspace) + a
               : nullptr;
}

ht_status ht_find_peaks(const ht_geometry *g, const void *acc, ht_peak *peaks, int32_t cap,
                        int32_t *d_count, void *workspace, size_t workspace_bytes,
                        ht_stream stream)
{
    if (!g || !acc || !d_count || !workspace || (cap > 0 && !peaks))
        return fail(HT_ERR_ARG, "ht_find_peaks: null argument");
    if (cap < 0) return fail(HT_ERR_ARG, "ht_find_peaks: cap < 0");
    if (workspace_bytes < ht::peaks_workspace_bytes(g->G))
        return fail(HT_ERR_ARG, "ht_find_peaks: workspace %zu B < %zu B", workspace_bytes,
                    ht::peaks_workspace_bytes(g->G));
    if (!aligned(workspace, 256) || !aligned(acc, 16))
        return fail(HT_ERR_ARG, "ht_find_peaks: workspace or accumulator alignment");
    cudaError_t e = ht::launch_peaks(g->G, acc, peaks, cap, d_count, workspace, S(stream),
                                     nullptr, nullptr,
                                     peak_spill_of(g->G, workspace, workspace_bytes));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_find_peaks");
}

ht_status ht_find_peaks_masked(const ht_geometry *g, const void *acc, const uint64_t *mask,
                               ht_peak *peaks, int32_t cap, int32_t *d_count, void *workspace,
                               size_t workspace_bytes, ht_stream stream)
{
    if (!g || !acc || !mask || !d_count || !workspace || (cap > 0 && !peaks))
        return fail(HT_ERR_ARG, "ht_find_peaks_masked: null argument");
    if (cap < 0) return fail(HT_ERR_ARG, "ht_find_peaks_masked: cap < 0");
    if (workspace_bytes < ht::peaks_workspace_bytes(g->G))
        return fail(HT_ERR_ARG, "ht_find_peaks_masked: workspace %zu B < %zu B", workspace_bytes,
                    ht::peaks_workspace_bytes(g->G));
    if (!aligned(workspace, 256) || !aligned(mask, 8) || !aligned(acc, 16))
        return fail(HT_ERR_ARG, "ht_find_peaks_masked: pointer alignment");
    cudaError_t e = ht::launch_peaks(g->G, acc, peaks, cap, d_count, workspace, S(stream),
                                     reinterpret_cast<const unsigned long long *>(mask), nullptr,
                                     peak_spill_of(g->G, workspace, workspace_bytes));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_find_peaks_masked");
}

size_t ht_associate_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap)
{
    return g ? ht::associate_workspace_bytes(g->G, n_hits, cap) : 0;
}

ht_status ht_associate(const ht_geometry *g, const float *x, const float *y, int32_t n_hits,
                       const ht_peak *peaks, const int32_t *d_count, int32_t cap,
                       int32_t *assign, void *workspace, size_t workspace_bytes,
                       ht_stream stream)
{
    if (!g || !d_count || !workspace || (cap > 0 && !peaks))
        return fail(HT_ERR_ARG, "ht_associate: null argument");
    if (n_hits < 0 || n_hits > kMaxHits || cap < 0)
        return fail(HT_ERR_ARG, "ht_associate: n_hits %d or cap %d out of range", n_hits, cap);
    if (n_hits > 0 && (!x || !y || !assign)) return fail(HT_ERR_ARG, "ht_associate: null hits");
    if (workspace_bytes < ht::associate_workspace_bytes(g->G, n_hits, cap) ||
        !aligned(workspace, 256))
        return fail(HT_ERR_ARG, "ht_associate: workspace too small or misaligned");
    cudaError_t e = ht::launch_associate(g->G, x, y, n_hits, peaks, d_count, cap, assign,
                                         workspace, S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_associate");
}

size_t ht_vote_z_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap)
{
    return g ? ht::vote_z_workspace_bytes(g->G, n_hits, cap) : 0;
}

ht_status ht_vote_z(const ht_geometry *g, const float *x, const float *y, const float *z,
                    int32_t n_hits, const int32_t *assign, const ht_peak *peaks,
                    const int32_t *d_count, int32_t cap, ht_zres *out, void *workspace,
                    size_t workspace_bytes, ht_stream stream)
{
    if (!g || !d_count || !workspace || (cap > 0 && (!peaks || !out)))
        return fail(HT_ERR_ARG, "ht_vote_z: null argument");
    if (n_hits < 0 || n_hits > kMaxHits || cap < 0)
        return fail(HT_ERR_ARG, "ht_vote_z: n_hits %d or cap %d out of range", n_hits, cap);
    if (n_hits > 0 && (!x || !y || !z || !assign)) return fail(HT_ERR_ARG, "ht_vote_z: null hits");
    if (workspace_bytes < ht::vote_z_workspace_bytes(g->G, n_hits, cap) ||
        !aligned(workspace, 256))
        return fail(HT_ERR_ARG, "ht_vote_z: workspace too small or misaligned");
    cudaError_t e = ht::launch_vote_z(g->G, x, y, z, n_hits, assign, peaks, d_count, cap, out,
                                      workspace, S(stream));
    return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_vote_z");
}

// ------------------------------------------------------------ host path
namespace {
struct EventWs {
    float *x, *y, *z;
    void *acc;
    ht_peak *peaks;
    int32_t *count, *assign;
    ht_zres *zres;
    uint64_t *stats;
    void *scratch;
    size_t scratch_bytes;
    size_t total;
};

EventWs carve_event(const ht_geometry *g, void *base, int32_t n, int32_t cap)
{
    using ht::align256;
    EventWs w{};
    char *p = reinterpret_cast<char *>(base);
    const size_t nh = (size_t)(n > 0 ? n : 1);
    w.x = reinterpret_cast<float *>(p); p += align256(nh * 4);
    w.y = reinterpret_cast<float *>(p); p += align256(nh * 4);
    w.z = reinterpret_cast<float *>(p); p += align256(nh * 4);
    w.acc = p; p += align256(ht_accumulator_bytes(g));
    w.peaks = reinterpret_cast<ht_peak *>(p); p += align256((size_t)(cap > 0 ? cap : 1) * 16);
    w.count = reinterpret_cast<int32_t *>(p); p += 256;
    w.assign = reinterpret_cast<int32_t *>(p); p += align256(nh * 4);
    w.zres = reinterpret_cast<ht_zres *>(p); p += align256((size_t)(cap > 0 ? cap : 1) * 12);
    w.stats = reinterpret_cast<uint64_t *>(p); p += 256;
    size_t s = ht_find_peaks_workspace_size(g);
    const size_t sa = ht::associate_workspace_bytes(g->G, n, cap);
    const size_t sz = ht::vote_z_workspace_bytes(g->G, n, cap);
    if (sa > s) s = sa;
    if (sz > s) s = sz;
    w.scratch = p;
    w.scratch_bytes = s;
    p += s;
    w.total = (size_t)(p - reinterpret_cast<char *>(base));
    return w;
}
}  // namespace

size_t ht_event_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap)
{
    if (!g) return 0;
    return carve_event(g, nullptr, n_hits, cap).total;
}

ht_status ht_run_event(const ht_geometry *g, const float *hx, const float *hy, const float *hz,
                       int32_t n_hits, void *workspace, size_t workspace_bytes, ht_peak *h_peaks,
                       int32_t cap, int32_t *h_count, int32_t *h_assign, ht_zres *h_zres,
                       uint64_t *h_stats, ht_stream stream)
{
    if (!g || !workspace || !h_count || (cap > 0 && (!h_peaks || !h_zres)))
        return fail(HT_ERR_ARG, "ht_run_event: null argument");
    if (n_hits < 0 || n_hits > kMaxHits || cap < 0)
        return fail(HT_ERR_ARG, "ht_run_event: n_hits %d or cap %d out of range", n_hits, cap);
    if (n_hits > 0 && (!hx || !hy || !hz || !h_assign))
        return fail(HT_ERR_ARG, "ht_run_event: null host hit arrays");
    if (!aligned(workspace, 256)) return fail(HT_ERR_ARG, "ht_run_event: workspace alignment");
    EventWs w = carve_event(g, workspace, n_hits, cap);
    if (workspace_bytes < w.total)
        return fail(HT_ERR_ARG, "ht_run_event: workspace %zu B < %zu B", workspace_bytes, w.total);
    cudaStream_t st = S(stream);
    const size_t hb = (size_t)n_hits * 4;
    cudaError_t e = cudaSuccess;
#define HT_TRY(call)                                           \
    do {                                                       \
        e = (call);                                            \
        if (e != cudaSuccess) return cuda_fail(e, #call);      \
    } while (0)
    if (n_hits > 0) {
        HT_TRY(cudaMemcpyAsync(w.x, hx, hb, cudaMemcpyHostToDevice, st));
        HT_TRY(cudaMemcpyAsync(w.y, hy, hb, cudaMemcpyHostToDevice, st));
        HT_TRY(cudaMemcpyAsync(w.z, hz, hb, cudaMemcpyHostToDevice, st));
    }
    ht_status s = ht_vote(g, w.x, w.y, n_hits, w.acc, w.stats, stream);
    if (s != HT_OK) return s;
    s = ht_find_peaks(g, w.acc, w.peaks, cap, w.count, w.scratch, w.scratch_bytes, stream);
    if (s != HT_OK) return s;
    s = ht_associate(g, w.x, w.y, n_hits, w.peaks, w.count, cap, w.assign, w.scratch,
                     w.scratch_bytes, stream);
    if (s != HT_OK) return s;
    s = ht_vote_z(g, w.x, w.y, w.z, n_hits, w.assign, w.peaks, w.count, cap, w.zres, w.scratch,
                  w.scratch_bytes, stream);
    if (s != HT_OK) return s;
    HT_TRY(cudaMemcpyAsync(h_count, w.count, 4, cudaMemcpyDeviceToHost, st));
    if (h_stats) HT_TRY(cudaMemcpyAsync(h_stats, w.stats, 16, cudaMemcpyDeviceToHost, st));
    if (n_hits > 0) HT_TRY(cudaMemcpyAsync(h_assign, w.assign, hb, cudaMemcpyDeviceToHost, st));
    HT_TRY(cudaStreamSynchronize(st));
    const int32_t np = *h_count < cap ? *h_count : cap;
    if (np > 0) {
        HT_TRY(cudaMemcpyAsync(h_peaks, w.peaks, (size_t)np * 16, cudaMemcpyDeviceToHost, st));
        HT_TRY(cudaMemcpyAsync(h_zres, w.zres, (size_t)np * 12, cudaMemcpyDeviceToHost, st));
        HT_TRY(cudaStreamSynchronize(st));
    }
#undef HT_TRY
    return HT_OK;
}

}  // extern "C"
