// mlp.cu -- the learned region proposal: a per-hit MLP 6 -> 128 -> 128 -> 64
// over (rho, d0) regions, its training kernels and the per-event region mask
// and per-hit region sets (ht_mlp_* in include/ht.h).  The paper has no
// learned part; this is the proposal's own reading.
//
// Numerics: BF16 weights and BF16 activations between layers, products of
// BF16 values exact in float32, float32 accumulation (tensor memory for the
// forward pass's 128-wide layers), float32 logits and softmax.  Features:
// x/110, y/110, z/(110 sinh 2.5), r/110, phi/pi, layer/9, each computed in
// float32 (no contraction) and rounded to BF16.
//
// Layout of the flat parameter array (float32 master and BF16 copy):
// W1[6][128] b1[128] W2[128][128] b2[128] W3[128][64] b3[64], W[i][o]
// multiplying input i into output o.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kIn = 6, kH = 128, kOut = 64;
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kOut, kParams = ob3 + kOut;
constexpr float kSinhEta = 6.0502044810397875f;   // sinh(2.5)

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Features of one hit, float32 operations in a fixed order, rounded to BF16.
__device__ __forceinline__ void hit_features(float x, float y, float z, int layer, float f[kIn])
{
    const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
    f[0] = bf(__fdiv_rn(x, 110.0f));
    f[1] = bf(__fdiv_rn(y, 110.0f));
    f[2] = bf(__fdiv_rn(z, __fmul_rn(110.0f, kSinhEta)));
    f[3] = bf(__fdiv_rn(r, 110.0f));
    f[4] = bf(__fdiv_rn(atan2f(y, x), 3.14159265358979f));
    f[5] = bf(__fdiv_rn((float)layer, 9.0f));
}

struct FwdOut {
    float *prob;             // n x 64 (or null)
    __nv_bfloat16 *h1, *h2;  // n x 128 each (or null)
    __nv_bfloat16 *feat;     // n x 8 (or null), features padded to 8
    float *mass;             // per-event region mass sums, [event][64] (or null)
    const int *off;          // event offsets when mass is set
    int n_ev;
    const int *d_n;          // (or null) device hit count, read instead of n
    unsigned long long *hmask;   // per-hit top-k region sets (or null)
    int topk;                    // regions per hit; >= 64: every region
    float pmin;                  // top-k mass below this: every region
};

__device__ __forceinline__ int event_of_hit(const int *off, int n_ev, int h)
{
    int lo = 0, hi = n_ev;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= h) lo = mid; else hi = mid;
    }
    return lo;
}

#include "mlp_tc.cuh"

// Split z of C[M][N] = sum_h A[h][M] B[h][N] (A BF16 with row stride lda,
// B float32 with row stride ldb) and, when bias is set, of bias[N] =
// sum_h B[h][N], on the CUDA cores, for the first layer (M = 6 inputs; the
// 128-row layers use k_wgrad_tc): the hits are split across gridDim.z and
// split z stores its partial sums at C + z pstride and bias + z pstride
// (plain stores: every entry of a split is written by exactly one CTA);
// k_wgrad_reduce adds the splits in a fixed order, so a training step is
// bit-reproducible.  CTA: 256 threads, a 64 x 64 output tile (4 x 4 per
// thread).
constexpr int kGT = 64, kGH = 32;
constexpr int kMaxSplits = 128;
__global__ void __launch_bounds__(256)
k_wgrad(const __nv_bfloat16 *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
        int n, int M, int N, float *__restrict__ C, float *__restrict__ bias, size_t pstride)
{
    C += (size_t)blockIdx.z * pstride;
    if (bias) bias += (size_t)blockIdx.z * pstride;
    __shared__ float sA[kGH][kGT], sB[kGH][kGT];
    const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    float bacc = 0.f;
    const int per = (n + gridDim.z - 1) / gridDim.z;
    const int h0 = blockIdx.z * per, h1 = min(n, h0 + per);
    for (int hb = h0; hb < h1; hb += kGH) {
        for (int t = threadIdx.x; t < kGH * kGT; t += 256) {
            const int r = t / kGT, c = t % kGT;
            const int hh = hb + r;
            sA[r][c] = (hh < h1 && m0 + c < M) ? __bfloat162float(A[(size_t)hh * lda + m0 + c]) : 0.f;
            sB[r][c] = (hh < h1 && n0 + c < N) ? B[(size_t)hh * ldb + n0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < kGH; ++r) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = sA[r][ty * 4 + u];
                b[u] = sB[r][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        if (bias && blockIdx.x == 0 && threadIdx.x < kGT)
            for (int r = 0; r < kGH; ++r) bacc += sB[r][threadIdx.x];
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int m = m0 + ty * 4 + u, nn = n0 + tx * 4 + v;
            if (m < M && nn < N) C[(size_t)m * N + nn] = acc[u][v];
        }
    if (bias && blockIdx.x == 0 && threadIdx.x < kGT && n0 + threadIdx.x < N)
        bias[n0 + threadIdx.x] = bacc;
}

// grad[i] += the splits' partial sums of parameter i, added in split order.
__global__ void k_wgrad_reduce(const float *__restrict__ part, int splits, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * kParams + i];
    grad[i] += s;
}

__global__ void k_count_labels(const int *__restrict__ labels, int n, int *__restrict__ nl)
{
    int c = 0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x)
        c += labels[h] >= 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nl, c);
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int np, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *__restrict__ pb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

// Per event: regions whose mean softmax mass is >= tau; with grow, also
// their 8 neighbours in the 8 x 8 region grid (no wrap); every region when
// more than fmax of the 64 are selected or the event has no hits.
__global__ void k_region_mask(const float *__restrict__ mass, const int *__restrict__ off,
                              int n_ev, float tau, float fmax, int grow,
                              unsigned long long *__restrict__ mask)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ev) return;
    const int n = off[e + 1] - off[e];
    unsigned long long bits = 0ull;
    for (int c = 0; c < kOut; ++c) {
        const float mm = n > 0 ? mass[(size_t)e * kOut + c] / (float)n : 0.f;
        if (mm >= tau) bits |= 1ull << c;
    }
    if (grow) {
        // bit 8 rb + db: neighbours in d0 are +-1 within a byte, in rho +-8
        const unsigned long long c0 = 0x0101010101010101ull, c7 = 0x8080808080808080ull;
        bits |= ((bits << 1) & ~c0) | ((bits >> 1) & ~c7);
        bits |= (bits << 8) | (bits >> 8);
    }
    mask[e] = ((float)__popcll(bits) > fmax * (float)kOut || n == 0) ? ~0ull : bits;
}


}  // namespace

cudaError_t prepare_mlp_kernels();

// The MLP calls need no geometry, so each device's kernel attributes are
// also set on the first MLP call made with that device current.
cudaError_t mlp_ready()
{
    constexpr int kMaxDev = 64;
    static std::once_flag once[kMaxDev];
    static cudaError_t status[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] { status[dev] = prepare_mlp_kernels(); });
    return status[dev];
}

// Region masses and masks of n_ev events whose hits sit at off[] (device);
// the hit total is read from off[n_ev] on the device, so a captured graph
// serves any batch of n_ev events with at most max_hits hits.
cudaError_t launch_region_mask(const void *params_bf16, const float *x, const float *y,
                               const float *z, const uint8_t *layer, const int *off, int n_ev,
                               int max_hits, float tau, float fmax, int grow, float *mass,
                               unsigned long long *masks, cudaStream_t st)
{
    cudaError_t e = mlp_ready();
    if (e == cudaSuccess) e = cudaMemsetAsync(mass, 0, (size_t)n_ev * kOut * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (max_hits > 0) {
        FwdOut o{nullptr, nullptr, nullptr, nullptr, mass, off, n_ev, off + n_ev};
        const int blocks = min((max_hits + kTcM - 1) / kTcM, device_sms() * 2);
        k_mlp_fwd_tc<<<blocks, kTcM, kTcSmem, st>>>((const __nv_bfloat16 *)params_bf16, x, y, z,
                                                    layer, max_hits, o);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_region_mask<<<(n_ev + 127) / 128, 128, 0, st>>>(mass, off, n_ev, tau, fmax, grow, masks);
    return cudaGetLastError();
}

// Per-hit region sets: the proposal network's top-k regions of every hit.
// n hits, or *d_n when d_n is set (n then bounds the grid).
cudaError_t launch_hit_masks(const void *params_bf16, const float *x, const float *y,
                             const float *z, const uint8_t *layer, int n, const int *d_n,
                             int topk, float pmin, unsigned long long *hit_masks, cudaStream_t st)
{
    cudaError_t e = mlp_ready();
    if (e != cudaSuccess || n <= 0) return e;
    FwdOut o{};
    o.d_n = d_n;
    o.hmask = hit_masks;
    o.topk = topk;
    o.pmin = pmin;
    const int blocks = min((n + kTcM - 1) / kTcM, device_sms() * 2);
    k_mlp_fwd_tc<<<blocks, kTcM, kTcSmem, st>>>((const __nv_bfloat16 *)params_bf16, x, y, z,
                                                layer, n, o);
    return cudaGetLastError();
}

cudaError_t prepare_mlp_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBwdTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kWgTcSmem);
    return e;
}

}  // namespace ht

using namespace ht;

extern "C" {

int32_t ht_mlp_param_count(void) { return kParams; }

int64_t ht_mlp_timeouts(void)
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_mlp_timeouts, sizeof v) != cudaSuccess) {
        set_error(HT_ERR_CUDA, "ht_mlp_timeouts: copy");
        return -1;
    }
    return (int64_t)v;
}

ht_status ht_mlp_forward(const void *params_bf16, const float *x, const float *y, const float *z,
                         const uint8_t *layer, int32_t n, float *prob, void *h1, void *h2,
                         void *feat, ht_stream stream)
{
    if (!params_bf16 || n < 0 || (n > 0 && (!x || !y || !z || !layer)))
        return set_error(HT_ERR_ARG, "ht_mlp_forward: bad argument");
    if (n == 0) return HT_OK;
    const cudaError_t pe = mlp_ready();
    if (pe != cudaSuccess) return set_error(HT_ERR_CUDA, cudaGetErrorString(pe));
    FwdOut o{prob, (__nv_bfloat16 *)h1, (__nv_bfloat16 *)h2, (__nv_bfloat16 *)feat, nullptr,
             nullptr, 0, nullptr};
    const int blocks = min((n + kTcM - 1) / kTcM, device_sms() * 2);
    k_mlp_fwd_tc<<<blocks, kTcM, kTcSmem, reinterpret_cast<cudaStream_t>(stream)>>>(
        (const __nv_bfloat16 *)params_bf16, x, y, z, layer, n, o);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HT_OK : set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

ht_status ht_mlp_region_mask(const void *params_bf16, const float *x, const float *y,
                             const float *z, const uint8_t *layer, const int32_t *off,
                             int32_t n_events, int32_t n_hits, float tau, float fmax, int32_t grow,
                             float *mass, uint64_t *masks, ht_stream stream)
{
    if (!params_bf16 || !off || !mass || !masks || n_events < 1 || n_hits < 0 ||
        (n_hits > 0 && (!x || !y || !z || !layer)))
        return set_error(HT_ERR_ARG, "ht_mlp_region_mask: bad argument");
    const cudaError_t e = launch_region_mask(params_bf16, x, y, z, layer, off, n_events, n_hits,
                                             tau, fmax, grow, mass,
                                             reinterpret_cast<unsigned long long *>(masks),
                                             reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HT_OK : set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

ht_status ht_mlp_hit_masks(const void *params_bf16, const float *x, const float *y,
                           const float *z, const uint8_t *layer, int32_t n_hits, int32_t topk,
                           float pmin, uint64_t *hit_masks, ht_stream stream)
{
    if (!params_bf16 || n_hits < 0 || topk < 1 ||
        (n_hits > 0 && (!x || !y || !z || !layer || !hit_masks)))
        return set_error(HT_ERR_ARG, "ht_mlp_hit_masks: bad argument");
    const cudaError_t e = launch_hit_masks(params_bf16, x, y, z, layer, n_hits, nullptr, topk,
                                           pmin,
                                           reinterpret_cast<unsigned long long *>(hit_masks),
                                           reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HT_OK : set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

size_t ht_mlp_backward_workspace_size(int32_t n)
{
    const size_t nh = (size_t)(n > 0 ? n : 1);
    return align256(nh * kOut * 4) + 2 * align256(nh * kH * 4) + 3 * align256(nh * kH * 2) + 256 +
           align256((size_t)kMaxSplits * kParams * 4);
}

// Gradients (added into grad, float32, kParams entries) of the mean cross
// entropy over labelled hits of one minibatch whose forward pass stored
// prob, h1, h2 and feat.
ht_status ht_mlp_backward(const void *params_bf16, const int32_t *labels, int32_t n,
                          const float *prob, const void *h1, const void *h2, const void *feat,
                          float *grad, void *workspace, size_t workspace_bytes, ht_stream stream)
{
    if (!params_bf16 || !labels || !prob || !h1 || !h2 || !feat || !grad || !workspace || n < 1)
        return set_error(HT_ERR_ARG, "ht_mlp_backward: bad argument");
    if (workspace_bytes < ht_mlp_backward_workspace_size(n))
        return set_error(HT_ERR_ARG, "ht_mlp_backward: workspace too small");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t pe = mlp_ready();
    if (pe != cudaSuccess) return set_error(HT_ERR_CUDA, cudaGetErrorString(pe));
    const size_t nh = (size_t)n;
    char *p = reinterpret_cast<char *>(workspace);
    float *dL = reinterpret_cast<float *>(p); p += align256(nh * kOut * 4);
    float *dH2 = reinterpret_cast<float *>(p); p += align256(nh * kH * 4);
    float *dH1 = reinterpret_cast<float *>(p); p += align256(nh * kH * 4);
    p += 3 * align256(nh * kH * 2);
    int *nl = reinterpret_cast<int *>(p);
    float *part = reinterpret_cast<float *>(p + 256);   // [splits][kParams]
    const int splits = max(1, min(kMaxSplits, n / 512));
    cudaError_t e = cudaMemsetAsync(nl, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(part, 0, (size_t)splits * kParams * 4, st);
    if (e != cudaSuccess) return set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    k_count_labels<<<min(1024, (n + 255) / 256), 256, 0, st>>>(labels, n, nl);
    const int blocks = min((n + kTcM - 1) / kTcM, device_sms() * 2);
    k_mlp_bwd_tc<<<blocks, kTcM, kBwdTcSmem, st>>>((const __nv_bfloat16 *)params_bf16, prob,
                                                   labels, (const __nv_bfloat16 *)h1,
                                                   (const __nv_bfloat16 *)h2, n, nl, dL, dH2, dH1);
    // dW3 = h2^T dL, db3 and dW2 = h1^T dH2, db2 on the tensor cores
    k_wgrad_tc<<<splits, kTcM, kWgTcSmem, st>>>((const __nv_bfloat16 *)h2, kH, dL, kOut, n, kOut,
                                                part + oW3, part + ob3, kParams);
    k_wgrad_tc<<<splits, kTcM, kWgTcSmem, st>>>((const __nv_bfloat16 *)h1, kH, dH2, kH, n, kH,
                                                part + oW2, part + ob2, kParams);
    // dW1 = f^T dH1, db1
    k_wgrad<<<dim3(1, kH / kGT, splits), 256, 0, st>>>((const __nv_bfloat16 *)feat, 8, dH1, kH, n,
                                                       kIn, kH, part + oW1, part + ob1, kParams);
    k_wgrad_reduce<<<(kParams + 255) / 256, 256, 0, st>>>(part, splits, grad);
    e = cudaGetLastError();
    return e == cudaSuccess ? HT_OK : set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

ht_status ht_mlp_adam(float *params, float *m, float *v, const float *grad, int32_t step, float lr,
                      float beta1, float beta2, float eps, void *params_bf16, ht_stream stream)
{
    if (!params || !m || !v || !grad || !params_bf16 || step < 1)
        return set_error(HT_ERR_ARG, "ht_mlp_adam: bad argument");
    const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
    k_adam<<<(kParams + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, m, v, grad, kParams, lr, beta1, beta2, eps, c1, c2, (__nv_bfloat16 *)params_bf16);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HT_OK : set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
